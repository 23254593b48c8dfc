"""Batched solves (lbks_create_batch / lbks_batch_scf): several geometries of
one shape relax in the same launches (system = blockIdx.y), each stopping on
its own |dE|.  Every system must match the same geometry solved alone and
the oracle; only the summation order of the reductions differs."""
import numpy as np
import pytest

import workloads as W
from oracle import scf

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _waters(count, seed):
    return W.water_scan(count, seed)


def test_batched_water_scan_matches_single_solves():
    """FP64: converged solves, batched and alone, agree to round-off."""
    torch, lbks = require_gpu()
    n, h = (28, 26, 30), 0.4
    mols = _waters(3, 1)
    # water at h = 0.4 has two occupied levels 0.01 Ha apart: long cycles converge in fewer of them
    b = lbks.Batch(n, h, 5, len(mols), precision=0, n_inner=100, max_cycles=400)
    b.set_geometries([(m.xyz, m.Z) for m in mols])
    res = b.scf()
    for i, m in enumerate(mols):
        s = lbks.System(n, h, 5, precision=0, n_inner=100, max_cycles=400)
        s.set_geometry(m.xyz, m.Z)
        ref = s.scf()
        assert res[i]["converged"] and res[i]["cycles"] == ref["cycles"]
        assert abs(res[i]["E_total"] - ref["E_total"]) <= 1e-9
        np.testing.assert_allclose(res[i]["eigenvalues"][:5], ref["eigenvalues"][:5], atol=1e-9)
        rho_b, rho_s = b.density(i), s.density()
        assert np.linalg.norm(rho_b - rho_s) / np.linalg.norm(rho_s) <= 1e-9
        s.close()
    b.close()


def test_batched_fp32_cycles_match_single_cycles():
    """FP32: the batched and the single launches may run different tuned
    kernels and sum overlaps in another order, so two solves stopped by
    |dE| can end a cycle apart; over a fixed number of cycles they agree to
    FP32 round-off."""
    torch, lbks = require_gpu()
    n, h = (28, 26, 30), 0.4
    mols = _waters(3, 1)
    b = lbks.Batch(n, h, 5, len(mols), precision=1, n_inner=25)
    b.set_geometries([(m.xyz, m.Z) for m in mols])
    res = b.scf_cycles(4)
    for i, m in enumerate(mols):
        s = lbks.System(n, h, 5, precision=1, n_inner=25)
        s.set_geometry(m.xyz, m.Z)
        ref = s.scf_cycles(4)
        assert abs(res[i]["E_total"] - ref["E_total"]) <= 2e-6
        np.testing.assert_allclose(res[i]["eigenvalues"][:5], ref["eigenvalues"][:5], atol=2e-6)
        rho_b, rho_s = b.density(i), s.density()
        assert np.linalg.norm(rho_b - rho_s) / np.linalg.norm(rho_s) <= 1e-5
        s.close()
    b.close()


def test_batched_trajectory_matches_oracle():
    """Three fixed cycles of two different geometries against the oracle."""
    torch, lbks = require_gpu()
    n, h = (24, 22, 26), 0.45
    mols = [W.water(1.7, 100.0), W.water(1.95, 112.0)]
    b = lbks.Batch(n, h, 5, 2, precision=0, n_inner=15, poisson_rtol=1e-12)
    b.set_geometries([(m.xyz, m.Z) for m in mols])
    res = b.scf_cycles(3)
    for i, m in enumerate(mols):
        st, ref = scf.scf(n, h, m.xyz, m.Z, 5, n_inner=15, poisson_rtol=1e-12, fixed_cycles=3)
        assert abs(res[i]["E_total"] - ref["E_total"]) <= 1e-8
        np.testing.assert_allclose(np.sort(res[i]["eigenvalues"][:5]), np.sort(ref["eigenvalues"]), atol=1e-8)
        rho = b.density(i)
        assert np.linalg.norm(rho - st.rho) / np.linalg.norm(st.rho) <= 1e-8
    b.close()


def test_batch_errors():
    torch, lbks = require_gpu()
    b = lbks.Batch((16, 16, 16), 0.4, 1, 2)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_batch_init(b.handle)  # no geometry yet
    with pytest.raises(lbks.LbksError):
        lbks.lbks_batch_set_geometry(b.handle, 2, [[0.0, 0.0, 0.0]], [2.0])  # index out of range
    with pytest.raises(lbks.LbksError):
        lbks.lbks_set_geometry(b.handle, [[0.0, 0.0, 0.0]], [2.0])  # single-system call on a batch
    b.close()
