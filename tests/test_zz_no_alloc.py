"""lbks_relax_step_noalloc, the variant for callers that may not allocate GPU
memory (their memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is off-limits to them), must give what lbks_relax_step
gives, for every precision and every stream-collide variant, and must not
change the device's free memory.  Two calls in a row check that the fixed
scratch array carries nothing from one call into the next.  Collected last
on purpose."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice

from gpu_util import rel_err, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 2e-5, 2: 2e-5}


def _buffers(torch, prec, n, n_orb, seed):
    TS = {0: torch.float64, 1: torch.float32, 2: torch.bfloat16}[prec]
    T = torch.float64 if prec == 0 else torch.float32
    nx, ny, nz = n
    f, V, sigma, _, u = W.random_state(n, n_orb, seed)
    return {
        "f_in": to_dev(torch, f, TS), "u_in": to_dev(torch, u[1:], T) if n_orb > 1 else None,
        "V": to_dev(torch, V, torch.float64), "sigma": to_dev(torch, sigma, torch.float64),
        "f_out": torch.empty((n_orb, 19, nz, ny, nx), dtype=TS, device="cuda"),
        "psi": torch.empty((n_orb, nz, ny, nx), dtype=T, device="cuda"),
        "S": torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda"),
        "lam": torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda"),
        "sig_out": torch.empty((n_orb,), dtype=torch.float64, device="cuda"),
    }


def _call(fn, prec, n, n_orb, b):
    omega, theta, h = 1.0, 0.5, 0.3
    dt = lattice.time_step(theta, omega, h)
    fn(prec, *n, n_orb, h, omega, theta, dt, b["f_in"], b["u_in"], b["V"], b["sigma"], b["f_out"], b["psi"], b["S"],
       b["lam"], b["sig_out"])


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4], ids=["tuned", "sites", "pairs", "prefetch", "bulk"])
@pytest.mark.parametrize("prec", [0, 1, 2], ids=["fp64", "fp32", "bf16"])
def test_noalloc_step_matches_allocating_step_twice(prec, variant):
    torch, lbks = require_gpu()
    prev = lbks.lbks_set_relax_variant(variant)
    try:
        # other sizes, other contents in each call; the odd nx runs the one-site
        # kernel where a variant needs even rows or 8-site multiples
        cases = [((32, 20, 17), 5, 21), ((64, 48, 40), 3, 22), ((33, 21, 17), 4, 23)]
        for n, n_orb, seed in cases:
            ref = _buffers(torch, prec, n, n_orb, seed)
            _call(lbks.lbks_relax_step, prec, n, n_orb, ref)
            got = _buffers(torch, prec, n, n_orb, seed)
            _call(lbks.lbks_relax_step_noalloc, prec, n, n_orb, got)  # warm-up: resolves the array's address
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            _call(lbks.lbks_relax_step_noalloc, prec, n, n_orb, got)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0, "the allocation-free step changed the free memory"
            for k in ("f_out", "psi", "S", "lam", "sig_out"):
                a, b = to_np(got[k]), to_np(ref[k])
                assert rel_err(a, b) <= TOL[prec], (n, k)
    finally:
        lbks.lbks_set_relax_variant(prev)


def test_noalloc_rejects_more_orbitals_than_its_scratch_holds():
    torch, lbks = require_gpu()
    b = _buffers(torch, 0, (4, 4, 4), 2, 0)
    with pytest.raises(lbks.LbksError) as e:
        _call(lbks.lbks_relax_step_noalloc, 0, (4, 4, 4), 9, b)
    assert e.value.code == lbks.EINVAL
    assert "8 orbitals" in str(e.value)
