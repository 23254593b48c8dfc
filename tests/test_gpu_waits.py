"""Bounded device waits of the tensor-core overlap kernel: a wait that gives
up ends in an error the host sees, and the context stays usable.

lbks_set_wait_limit(0) makes every main mbarrier wait of the kernel give up
at once (a runtime override; nothing is broken on the device).  Each block
then counts a timeout, writes NaN partial sums, waits with the full bound for
its own tensor-core work, frees its tensor memory and returns.  The test
checks the NaN overlap and the counter, that a solve with more than eight
FP32 orbitals reports LBKS_ENOTCONV, and that with the default limit
restored the same calls give correct results again."""
import numpy as np
import pytest

import workloads as W

from gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _psi(n_sites, n_orb, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(n_orb, n_sites))


def test_overlap_wait_gives_up_and_recovers():
    torch, lbks = require_gpu()
    n_sites, n_orb, h = 40 * 40 * 40, 12, 0.3
    p = _psi(n_sites, n_orb, 5)
    pd = to_dev(torch, p, torch.float32)
    ref = h ** 3 * (pd.double().cpu().numpy() @ pd.double().cpu().numpy().T)
    S = torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda")
    t0 = lbks.lbks_wait_timeouts()
    prev = lbks.lbks_set_wait_limit(0)
    try:
        lbks.lbks_overlap(lbks.FP32, n_sites, n_orb, h, pd, S, tensor_cores=True)
        torch.cuda.synchronize()
        assert np.isnan(S.cpu().numpy()).all()
        assert lbks.lbks_wait_timeouts() > t0
    finally:
        assert lbks.lbks_set_wait_limit(prev) == 0
    lbks.lbks_overlap(lbks.FP32, n_sites, n_orb, h, pd, S, tensor_cores=True)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    d = np.sqrt(np.diag(ref))
    assert (np.abs(got - ref) / np.outer(d, d)).max() < 3e-6
    t1 = lbks.lbks_wait_timeouts()
    lbks.lbks_overlap(lbks.FP32, n_sites, n_orb, h, pd, S, tensor_cores=True)
    torch.cuda.synchronize()
    assert lbks.lbks_wait_timeouts() == t1  # no timeouts at the default limit


def test_solve_reports_the_failed_wait_and_the_next_solve_succeeds():
    torch, lbks = require_gpu()
    mol = W.water_cluster(2, seed=3, box=11.0, min_oo=5.0, margin=2.5)
    n, h = (36, 32, 34), 0.35
    prev = lbks.lbks_set_wait_limit(0)
    try:
        s = lbks.System(n, h, 10, precision=lbks.FP32, n_inner=10, max_cycles=3)
        s.set_geometry(mol.xyz, mol.Z)  # the start uses the exact overlap: no tensor-core waits yet
        with pytest.raises(lbks.LbksError) as e:
            s.scf()
        assert e.value.code == lbks.ENOTCONV
        s.close()
    finally:
        lbks.lbks_set_wait_limit(prev)
    s = lbks.System(n, h, 10, precision=lbks.FP32, n_inner=10, max_cycles=3)
    s.set_geometry(mol.xyz, mol.Z)
    r = s.scf_cycles(2)
    assert np.isfinite(r["E_total"]) and np.isfinite(r["eigenvalues"][:10]).all()
    s.close()
