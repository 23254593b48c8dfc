"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lbks.h declares.  No compute call (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1507_07666_gb300 import build as build_mod

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbks.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbks_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = build_mod.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = _declared()
    for required in ("lbks_create_system", "lbks_set_geometry", "lbks_scf", "lbks_energy",
                     "lbks_relax_step", "lbks_hartree", "lbks_lda"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_1507_07666_gb300 import lbks
    assert set(_declared()) <= set(lbks.EXPORTED)


def test_host_only_calls(lib):
    from paper_1507_07666_gb300 import lbks
    p = lbks.lbks_params_default()
    assert (p.omega, p.theta, p.n_inner, p.precision) == (1.0, 0.5, 50, lbks.FP64)
    assert lbks.lbks_version().startswith("lbks")
    # invalid arguments are rejected on the host before any device work
    with pytest.raises(lbks.LbksError) as e:
        lbks.lbks_create_system(p, 1, 8, 8, 0.2, 1)
    assert e.value.code == lbks.EINVAL
    with pytest.raises(lbks.LbksError):
        lbks.lbks_create_system(p, 8, 8, 8, -0.2, 1)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_create_system(p, 8, 8, 8, 0.2, lbks.MAX_ORB + 1)
    bad = lbks.lbks_params_default(omega=2.5)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_create_system(bad, 8, 8, 8, 0.2, 1)
    assert "lbks_params" in lbks.last_error()


def test_fast_division_formula():
    """The library's index decoding divides by the grid extents with the
    multiply-high method; check the formula (as written in lbks_internal.cuh)
    exhaustively for the extents used and a sweep of numerators below 2^31."""
    def fastdiv(d):
        l = 0
        while (1 << l) < d:
            l += 1
        m = ((1 << 32) * ((1 << l) - d)) // d + 1
        return m & 0xFFFFFFFF, l

    import numpy as np
    ns = np.concatenate([np.arange(0, 200000, dtype=np.uint64),
                         np.random.default_rng(0).integers(0, 2 ** 31, 200000, dtype=np.uint64)])
    for d in list(range(1, 300)) + [384, 512, 1000, 1024, 1290]:
        m, l = fastdiv(d)
        q = ((((ns * np.uint64(m)) >> np.uint64(32)) + ns) & np.uint64(0xFFFFFFFF)) >> np.uint64(l)
        assert (q == ns // np.uint64(d)).all(), d


def _c_array(text, name):
    m = re.search(r"constexpr \w+ " + name + r"\[kPsiShapes\] = \{([^}]*)\};", text)
    assert m, name
    return [v.strip() for v in m.group(1).split(",")]


def test_binding_tile_shapes_match_the_library_tables():
    """The binding's tile-shape tables (index = lbks_set_psi_tile's shape)
    restate the library's: x and z extents, sites per thread, plane sums, and
    y = threads x sites per thread / x."""
    from paper_1507_07666_gb300 import lbks
    text = open(os.path.join(os.path.dirname(HEADER), os.pardir, "paper_1507_07666_gb300", "csrc",
                             "lbks_internal.cuh")).read()
    threads = int(re.search(r"constexpr int kThreads = (\d+);", text).group(1))
    tx = [int(v) for v in _c_array(text, "kPsiTileTX")]
    tz = [int(v) for v in _c_array(text, "kPsiTileTZ")]
    xw = [int(v) for v in _c_array(text, "kPsiTileXW")]
    pl = [v == "true" for v in _c_array(text, "kPsiTilePL")]
    assert len(lbks.PSI_TILES) == len(tx)
    assert [t[0] for t in lbks.PSI_TILES] == tx
    assert [t[2] for t in lbks.PSI_TILES] == tz
    assert [t[1] for t in lbks.PSI_TILES] == [threads * w // x for x, w in zip(tx, xw)]
    assert list(lbks.PSI_TILE_SITES_PER_THREAD) == xw
    assert list(lbks.PSI_TILE_PLANE_SUMS) == pl
