"""The relaxation step at the 8-water cluster's full size (256^3 grid, 40
orbitals, FP32) in the launch configuration the bench times, checked on sampled
sites that the oracle's definition gives one by one: the orbital at r is the
scaled sum of the populations arriving from r - v_p (Eq. KSLB, pull
streaming, nothing from outside the box), plus the W source xi_p u(r - v_p).
The overlap is checked through properties that hold at any size (symmetry,
the diagonal against an FP64 sum of the returned orbitals)."""
import numpy as np
import pytest

from oracle import lattice

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

N3, NO, H, THETA = (256, 256, 256), 40, 0.2, 0.5


def _sample_sites(rng, n, count):
    nx, ny, nz = n
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny // 2, nz - 1), (nx - 1, 0, nz // 3)]  # faces and corners
    while len(pts) < count:
        pts.append(tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))))
    return pts


def _pulled(torch, arr, n, pts, p):
    """Values arr[..., z - vz, y - vy, x - vx] for each sampled site (0 outside)."""
    nx, ny, nz = n
    vx, vy, vz = lattice.VELOCITIES[p]
    out = []
    for (x, y, z) in pts:
        sx, sy, sz = x - vx, y - vy, z - vz
        if 0 <= sx < nx and 0 <= sy < ny and 0 <= sz < nz:
            out.append(arr[..., sz, sy, sx])
        else:
            out.append(torch.zeros(arr.shape[:-3], dtype=arr.dtype, device=arr.device))
    return torch.stack(out, dim=-1)  # [..., site]


@pytest.mark.parametrize("storage", ["populations", "psi"])
def test_cluster_step_on_sampled_sites(storage):
    torch, lbks = require_gpu()
    nx, ny, nz = N3
    rng = np.random.Generator(np.random.PCG64(17))
    gen = torch.Generator(device="cuda").manual_seed(17)
    xi = lattice.xi(THETA)
    chi = lattice.chi()
    dt = lattice.time_step(THETA, 1.0, H)
    V = -3.0 * torch.rand((nz, ny, nx), generator=gen, dtype=torch.float64, device="cuda")
    sig = torch.from_numpy(rng.uniform(0.5, 2.0, NO)).cuda()
    S = torch.empty((NO, NO), dtype=torch.float64, device="cuda")
    lam, sig2 = torch.empty_like(S), torch.empty_like(sig)
    pts = _sample_sites(rng, N3, 48)
    if storage == "populations":
        f = torch.rand((NO, 19, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        u = 0.1 * torch.rand((NO - 1, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        fo = torch.empty_like(f)
        psi = torch.empty((NO, nz, ny, nx), dtype=torch.float32, device="cuda")
        lbks.lbks_relax_step(lbks.FP32, nx, ny, nz, NO, H, 1.0, THETA, dt, f, u, V, sig, fo, psi, S, lam, sig2)
        torch.cuda.synchronize()
        ref = torch.zeros((NO, len(pts)), dtype=torch.float64, device="cuda")
        for p in range(19):
            ref += _pulled(torch, f[:, p], N3, pts, p).double()
            ref[1:] += xi[p] * _pulled(torch, u, N3, pts, p).double()
        del f, fo, u
    else:
        pin = torch.rand((NO, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        lam_in = torch.from_numpy(np.tril(rng.uniform(-0.3, 0.3, (NO, NO)), -1)).cuda()
        psi = torch.empty_like(pin)
        lbks.lbks_relax_step_psi(lbks.FP32, nx, ny, nz, NO, H, THETA, dt, pin, lam_in, V, sig, psi, S, lam, sig2)
        torch.cuda.synchronize()
        # populations the state stands for: xi_p psi - dt chi_p V psi + xi_p u, u_j = -sum_k Lambda_jk psi_k
        ref = torch.zeros((NO, len(pts)), dtype=torch.float64, device="cuda")
        for p in range(19):
            pp = _pulled(torch, pin, N3, pts, p).double()
            vv = _pulled(torch, V, N3, pts, p)
            uu = -(lam_in @ pp)
            ref += (xi[p] - dt * chi[p] * vv)[None] * pp + xi[p] * uu
        del pin
    ref *= sig[:, None]
    got = torch.stack([psi[:, z, y, x] for (x, y, z) in pts], dim=-1).double()
    err = (got - ref).abs().max().item() / ref.abs().max().item()
    assert err < 2e-5, err
    # overlap: symmetric, diagonal = h^3 sum psi_j^2 (FP64 over the returned orbitals)
    Sd = S.cpu().numpy()
    np.testing.assert_array_equal(Sd, Sd.T)
    diag = H ** 3 * (psi.double() ** 2).sum(dim=(1, 2, 3)).cpu().numpy()
    np.testing.assert_allclose(np.diag(Sd), diag, rtol=3e-6)  # tensor-core overlap: bias below 1.5e-6
    np.testing.assert_allclose(sig2.cpu().numpy(), 1.0 / np.sqrt(np.diag(Sd)), rtol=1e-12)
    del psi
    torch.cuda.empty_cache()
