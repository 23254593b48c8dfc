"""GPU parity of the FP64 field kernels: Hartree (lattice Poisson with
multipole boundary values) and LDA exchange-correlation, against the oracle
on the same inputs, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import lda, poisson

from gpu_util import rel_err, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,h,c", [((24, 24, 24), 0.5, (0.0, 0.0, 0.0)),
                                   ((33, 27, 30), 0.4, (0.7, -0.5, 0.3)),
                                   ((64, 64, 64), 0.25, (0.2, 0.1, -0.4))])
def test_hartree_matches_oracle(n, h, c):
    torch, lbks = require_gpu()
    nx, ny, nz = n
    X, Y, Z = poisson.coords(n, h)
    s = 1.1
    rho = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    rho += 0.3 * np.exp(-((X + 1.0) ** 2 + Y ** 2 + (Z - 0.5) ** 2) / 0.8)
    ref, _, _ = poisson.hartree(rho, h, rtol=1e-13)
    v = torch.zeros((nz, ny, nx), dtype=torch.float64, device="cuda")
    it, rr = lbks.lbks_hartree(nx, ny, nz, h, to_dev(torch, rho, torch.float64), v, rtol=1e-13)
    assert rr <= 1e-13 and it > 0
    # both at relative residual 1e-13; the condition number grows like (n+1)^2
    assert rel_err(to_np(v), ref) < 1e-9
    # warm start from the solution converges at once
    it2, _ = lbks.lbks_hartree(nx, ny, nz, h, to_dev(torch, rho, torch.float64), v, rtol=1e-12)
    assert it2 <= 2


def test_hartree_reports_non_convergence():
    torch, lbks = require_gpu()
    n, h = (20, 20, 20), 0.5
    X, Y, Z = poisson.coords(n, h)
    rho = np.exp(-(X * X + Y * Y + Z * Z))
    v = torch.zeros((20, 20, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(lbks.LbksError) as e:
        lbks.lbks_hartree(20, 20, 20, h, to_dev(torch, rho, torch.float64), v, rtol=1e-14, max_iter=3)
    assert e.value.code == lbks.ENOTCONV


def test_hartree_ignores_an_earlier_solves_direction():
    """The first PCG direction is the preconditioned residual itself.  A
    direction left non-finite in the shared scratch by an earlier solve (a NaN
    density, stopped after two iterations) must not leak into the next one:
    p = z + 0 * p would be NaN."""
    torch, lbks = require_gpu()
    n, h = (22, 18, 20), 0.45
    nx, ny, nz = n
    X, Y, Z = poisson.coords(n, h)
    rho = np.exp(-(X * X + 0.5 * Y * Y + (Z - 0.3) ** 2))
    stream = torch.cuda.Stream()  # one workspace for both solves
    bad = torch.full((nz, ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(bad)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_hartree(nx, ny, nz, h, bad, v, rtol=1e-12, max_iter=2, stream=stream)
    v.zero_()
    it, rr = lbks.lbks_hartree(nx, ny, nz, h, to_dev(torch, rho, torch.float64), v, rtol=1e-12, stream=stream)
    stream.synchronize()
    ref, _, _ = poisson.hartree(rho, h, rtol=1e-13)
    assert rr <= 1e-12 and np.isfinite(to_np(v)).all()
    assert rel_err(to_np(v), ref) < 1e-9


def test_lda_matches_oracle():
    torch, lbks = require_gpu()
    rng = np.random.default_rng(0)
    rho = np.concatenate([[0.0, 1e-20, 5e-15, 1e-14, 3.0 / (4 * math.pi)],
                          10.0 ** rng.uniform(-16, 3, size=100000)])
    eps_ref, v_ref = lda.lda_xc(rho)
    d = to_dev(torch, rho, torch.float64)
    eps = torch.empty_like(d)
    v = torch.empty_like(d)
    lbks.lbks_lda(len(rho), d, eps, v)
    torch.cuda.synchronize()
    np.testing.assert_allclose(to_np(eps), eps_ref, rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(to_np(v), v_ref, rtol=1e-13, atol=1e-300)
