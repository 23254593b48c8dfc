"""Overlap matrix S = h^3 Psi Psi^T through lbks_overlap against an FP64
product of the same stored values.

The tensor-core kernel (the solver's per-step overlap of more than eight FP32
orbitals) splits each value into bf16 hi + lo, which leaves a 2^-17-relative,
sign-random error per product, and accumulates in tensor memory in FP32 over
at most 512 sites.  That accumulation truncates: the diagonal carries a
negative relative bias of about 1e-6, which the test bounds; the solver uses
this kernel only for sigma and Lambda, which every step measures again.  The
SIMT kernels (FP64, and the orthonormalising overlap) sum in FP64."""
import numpy as np
import pytest

from gpu_util import require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu


def _orbitals(n, n_orb, seed, smooth):
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = n
    if not smooth:
        return rng.uniform(-1.0, 1.0, size=(n_orb, nz, ny, nx))
    z, y, x = np.meshgrid(np.linspace(-1, 1, nz), np.linspace(-1, 1, ny), np.linspace(-1, 1, nx), indexing="ij")
    out = np.empty((n_orb, nz, ny, nx))
    for j in range(n_orb):
        c = rng.uniform(-0.5, 0.5, size=3)
        w = rng.uniform(0.2, 0.6)
        poly = 1.0 + rng.uniform(-1, 1) * x + rng.uniform(-1, 1) * y * z
        out[j] = poly * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * w * w))
    return out


def _scaled_err(S, ref):
    d = np.sqrt(np.abs(np.diag(ref)))
    return np.abs(S - ref) / np.outer(d, d)


@pytest.mark.parametrize("n,n_orb,smooth", [
    ((40, 40, 40), 9, True),     # N % 4 == 0: vector loads
    ((40, 40, 40), 40, True),
    ((64, 48, 40), 64, True),
    ((23, 19, 17), 16, False),   # ragged N: scalar loads, partial last tile
    ((31, 7, 5), 33, False),
    ((24, 20, 16), 20, False),   # each compile-time bound of the kernel: <= 16, 32, 40 (ten warps), 48, 64 orbitals
    ((21, 17, 15), 45, False),
    ((32, 16, 12), 36, True),
    ((12, 10, 8), 3, True),
])
def test_fp32_overlap_tensor_cores(n, n_orb, smooth):
    torch, lbks = require_gpu()
    h = 0.3
    psi = _orbitals(n, n_orb, 7 + n_orb, smooth).astype(np.float32).astype(np.float64)
    N = int(np.prod(n))
    S = torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda")
    lbks.lbks_overlap(lbks.FP32, N, n_orb, h, to_dev(torch, psi, torch.float32), S, tensor_cores=True)
    torch.cuda.synchronize()
    flat = psi.reshape(n_orb, N)
    ref = h ** 3 * (flat @ flat.T)
    g = to_np(S)
    np.testing.assert_array_equal(g, g.T)
    err = _scaled_err(g, ref)
    assert err.max() < 3e-6, err.max()
    bias = np.mean((np.diag(g) - np.diag(ref)) / np.diag(ref))
    assert -1.5e-6 < bias <= 1e-7, bias


@pytest.mark.parametrize("n,n_orb", [((40, 40, 40), 40), ((23, 19, 17), 9), ((5, 3, 2), 2)])
def test_fp32_overlap_simt_is_unbiased(n, n_orb):
    torch, lbks = require_gpu()
    h = 0.3
    psi = _orbitals(n, n_orb, 5 + n_orb, True).astype(np.float32).astype(np.float64)
    N = int(np.prod(n))
    S = torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda")
    lbks.lbks_overlap(lbks.FP32, N, n_orb, h, to_dev(torch, psi, torch.float32), S)
    torch.cuda.synchronize()
    flat = psi.reshape(n_orb, N)
    ref = h ** 3 * (flat @ flat.T)
    g = to_np(S)
    assert _scaled_err(g, ref).max() < 2e-7
    assert abs(np.mean((np.diag(g) - np.diag(ref)) / np.diag(ref))) < 2e-8


@pytest.mark.parametrize("n_orb", [3, 8, 12, 64])
def test_fp64_overlap(n_orb):
    torch, lbks = require_gpu()
    n, h = (21, 18, 13), 0.25
    psi = _orbitals(n, n_orb, 3, True)
    N = int(np.prod(n))
    S = torch.empty((n_orb, n_orb), dtype=torch.float64, device="cuda")
    lbks.lbks_overlap(lbks.FP64, N, n_orb, h, to_dev(torch, psi, torch.float64), S)
    torch.cuda.synchronize()
    flat = psi.reshape(n_orb, N)
    assert _scaled_err(to_np(S), h ** 3 * (flat @ flat.T)).max() < 1e-13


def test_overlap_single_site_and_errors():
    torch, lbks = require_gpu()
    psi = torch.tensor([[2.0], [3.0]] * 5, dtype=torch.float32, device="cuda")  # 10 orbitals, one site
    S = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    v = np.array([2.0, 3.0] * 5)
    for tc in (False, True):
        S.fill_(np.nan)
        lbks.lbks_overlap(lbks.FP32, 1, 10, 1.0, psi, S, tensor_cores=tc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(to_np(S), np.outer(v, v), rtol=1e-7)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_overlap(lbks.FP32, 0, 10, 1.0, psi, S)
    with pytest.raises(lbks.LbksError):
        lbks.lbks_overlap(lbks.FP32, 1, 65, 1.0, psi, S)
