"""Serving loop (lbks_server_create / lbks_submit / lbks_poll): requests of
different sizes admitted while others run give the same answer as the same
request solved alone, within the solve tolerance (here bit for bit, since
every system reduces in a fixed order on private scratch)."""
import time

import numpy as np
import pytest

import workloads as W

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

MIX = [
    ("He", W.helium(), (24, 24, 24), 0.4),
    ("H2", W.h2(1.4), (28, 24, 32), 0.35),
    ("LiH", W.lih(3.0), (30, 28, 36), 0.3),
    ("He", W.helium(), (20, 22, 24), 0.42),
    ("H2", W.h2(1.5), (24, 24, 24), 0.4),
]


def _alone(lbks, n, h, mol, prec):
    s = lbks.System(n, h, mol.n_orb, precision=prec, n_inner=20)
    s.set_geometry(mol.xyz, mol.Z)
    r = s.scf()
    s.close()
    return r


def _drain(lbks, srv, ids, timeout=300.0):
    out = {}
    t_end = time.time() + timeout
    while len(out) < len(ids):
        assert time.time() < t_end, "serving loop did not finish"
        for rid in ids:
            if rid in out:
                continue
            r = lbks.lbks_poll(srv, rid)
            if r is not None:
                out[rid] = r
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_results_in_the_mix_equal_results_alone(prec):
    torch, lbks = require_gpu()
    params = lbks.lbks_params_default(precision=prec, n_inner=20)
    srv = lbks.lbks_server_create(params, 0, 3)
    try:
        ids = []
        for _, mol, n, h in MIX * 2:  # ten requests, at most three at a time
            ids.append(lbks.lbks_submit(srv, n, h, mol.xyz, mol.Z))
        got = _drain(lbks, srv, ids)
        stats = lbks.lbks_server_get_stats(srv)
        assert stats["completed"] == len(ids) and stats["queued"] == 0 and stats["running"] == 0
    finally:
        lbks.lbks_server_destroy(srv)
    for k, rid in enumerate(ids):
        _, mol, n, h = (MIX * 2)[k]
        res, timing = got[rid]
        ref = _alone(lbks, n, h, mol, prec)
        assert res["converged"]
        assert abs(res["E_total"] - ref["E_total"]) <= 1e-10
        np.testing.assert_allclose(res["eigenvalues"][:mol.n_orb], ref["eigenvalues"][:mol.n_orb], atol=1e-10)
        assert timing["latency_s"] >= timing["run_s"] > 0


def test_serving_errors_are_reported_on_the_host():
    torch, lbks = require_gpu()
    srv = lbks.lbks_server_create(lbks.lbks_params_default(n_inner=20), 64 << 20, 1)
    try:
        with pytest.raises(lbks.LbksError) as e:  # can never fit the 64 MiB budget
            lbks.lbks_submit(srv, (128, 128, 128), 0.2, W.methane().xyz, W.methane().Z)
        assert e.value.code == lbks.ENOMEM
        with pytest.raises(lbks.LbksError) as e:
            lbks.lbks_poll(srv, 987654)
        assert e.value.code == lbks.ENOTFOUND
        mol = W.helium()
        a = lbks.lbks_submit(srv, (24, 24, 24), 0.4, mol.xyz, mol.Z)
        b = lbks.lbks_submit(srv, (24, 24, 24), 0.4, mol.xyz, mol.Z)
        with pytest.raises(lbks.LbksError) as e:  # one slot: b waits behind a
            lbks.lbks_server_wait(srv, b, 1e-4)
        assert e.value.code == lbks.ETIMEDOUT
        lbks.lbks_server_wait(srv, b, 120.0)
        ra, rb = lbks.lbks_poll(srv, a), lbks.lbks_poll(srv, b)
        assert ra[0]["E_total"] == rb[0]["E_total"]
        bad = lbks.lbks_submit(srv, (24, 24, 24), 0.4, [[9.0, 0.0, 0.0]], [2.0])  # atom outside the box
        lbks.lbks_server_wait(srv, bad, 60.0)
        with pytest.raises(lbks.LbksError) as e:
            lbks.lbks_poll(srv, bad)
        assert e.value.code == lbks.EINVAL
    finally:
        lbks.lbks_server_destroy(srv)


def test_new_handle_is_ready_while_the_legacy_stream_is_busy():
    """A handle zeroes its counters and flags on its own stream and waits for
    them.  Zeroing them with legacy-stream cudaMemset left them unordered
    with the solve's non-blocking streams: with the legacy stream held by a
    long kernel, the zeroing landed mid-solve (reset arrival counters and
    atom counts: failed Cholesky, energies without nuclear attraction)."""
    torch, lbks = require_gpu()
    _, mol, n, h = MIX[2]
    ref = _alone(lbks, n, h, mol, 1)
    torch.cuda._sleep(2_000_000_000)  # ~1 s spin on the legacy default stream
    s = lbks.System(n, h, mol.n_orb, precision=1, n_inner=20)
    s.set_geometry(mol.xyz, mol.Z)
    r = s.scf(stream=torch.cuda.Stream())
    s.close()
    torch.cuda.synchronize()
    assert r["converged"]
    assert abs(r["E_total"] - ref["E_total"]) <= 1e-10
