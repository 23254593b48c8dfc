"""The relaxation step at the 8-water cluster's full size (256^3 grid, 40
orbitals, FP32) in the launch configuration the bench times, checked on sampled
sites against the oracle: each sampled site's 3 x 3 x 3 neighbourhood (zeros
outside the box) goes through the oracle's own step -- ``lb.pull_stream`` and
``lb.collide`` for populations (Eq. KSLB), ``psi.step`` for orbital storage --
and its centre must equal the GPU's orbitals and, for populations, all 19
post-collision populations.  The overlap is checked through properties that
hold at any size (symmetry, the diagonal against an FP64 sum of the returned
orbitals)."""
import numpy as np
import pytest

from oracle import lattice, lb
from oracle import psi as opsi

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

N3, NO, H, THETA = (256, 256, 256), 40, 0.2, 0.5


def _sample_sites(rng, n, count):
    nx, ny, nz = n
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny // 2, nz - 1), (nx - 1, 0, nz // 3)]  # faces and corners
    while len(pts) < count:
        pts.append(tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))))
    return pts


def _patch(arr, pt, n):
    """arr[..., z-1:z+2, y-1:y+2, x-1:x+2] in FP64 on the host, zero outside the box."""
    lo = [c - 1 for c in pt[::-1]]  # z, y, x
    a = [max(l, 0) for l in lo]
    b = [min(l + 3, m) for l, m in zip(lo, n[::-1])]
    out = np.zeros(tuple(arr.shape[:-3]) + (3, 3, 3))
    sub = arr[..., a[0]:b[0], a[1]:b[1], a[2]:b[2]].double().cpu().numpy()
    out[..., a[0] - lo[0]:b[0] - lo[0], a[1] - lo[1]:b[1] - lo[1], a[2] - lo[2]:b[2] - lo[2]] = sub
    return out


@pytest.mark.parametrize("storage", ["populations", "psi"])
def test_cluster_step_on_sampled_sites(storage):
    torch, lbks = require_gpu()
    nx, ny, nz = N3
    rng = np.random.Generator(np.random.PCG64(17))
    gen = torch.Generator(device="cuda").manual_seed(17)
    xi = lattice.xi(THETA)
    dt = lattice.time_step(THETA, 1.0, H)
    V = -3.0 * torch.rand((nz, ny, nx), generator=gen, dtype=torch.float64, device="cuda")
    sig = torch.from_numpy(rng.uniform(0.5, 2.0, NO)).cuda()
    S = torch.empty((NO, NO), dtype=torch.float64, device="cuda")
    lam, sig2 = torch.empty_like(S), torch.empty_like(sig)
    pts = _sample_sites(rng, N3, 48)
    xi_b = xi[None, :, None, None, None]
    sig_np = sig.cpu().numpy()
    if storage == "populations":
        f = torch.rand((NO, 19, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        u = 0.1 * torch.rand((NO - 1, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        fo = torch.empty_like(f)
        psi = torch.empty((NO, nz, ny, nx), dtype=torch.float32, device="cuda")
        lbks.lbks_relax_step(lbks.FP32, nx, ny, nz, NO, H, 1.0, THETA, dt, f, u, V, sig, fo, psi, S, lam, sig2)
        torch.cuda.synchronize()
        ref_psi, ref_f, got_f = [], [], []
        for (x, y, z) in pts:
            # the populations the (split) state stands for: f + xi_p u for orbitals 1..
            fs = _patch(f, (x, y, z), N3)
            fs[1:] += xi_b * _patch(u, (x, y, z), N3)[:, None]
            arr = lb.pull_stream(fs)[:, :, 1:2, 1:2, 1:2] * sig_np[:, None, None, None, None]
            ps = arr.sum(axis=1)
            ref_psi.append(ps[:, 0, 0, 0])
            ref_f.append(lb.collide(arr, ps, _patch(V, (x, y, z), N3)[1:2, 1:2, 1:2], 1.0, THETA, dt)[..., 0, 0, 0])
            got_f.append(fo[:, :, z, y, x].double().cpu().numpy())
        ref_f, got_f = np.stack(ref_f, axis=-1), np.stack(got_f, axis=-1)
        assert np.abs(got_f - ref_f).max() / np.abs(ref_f).max() < 2e-5
        del f, fo, u
    else:
        pin = torch.rand((NO, nz, ny, nx), generator=gen, dtype=torch.float32, device="cuda")
        lam_np = np.tril(rng.uniform(-0.3, 0.3, (NO, NO)), -1)
        lam_in = torch.from_numpy(lam_np).cuda()
        psi = torch.empty_like(pin)
        lbks.lbks_relax_step_psi(lbks.FP32, nx, ny, nz, NO, H, THETA, dt, pin, lam_in, V, sig, psi, S, lam, sig2)
        torch.cuda.synchronize()
        ref_psi = []
        for (x, y, z) in pts:
            st = opsi.PsiState(_patch(pin, (x, y, z), N3))
            st.lam, st.vc = lam_np, _patch(V, (x, y, z), N3)
            ref_psi.append(opsi.step(st, sig_np, st.vc, THETA, dt, H)["psi"][:, 1, 1, 1])
        del pin
    ref = np.stack(ref_psi, axis=-1)
    got = torch.stack([psi[:, z, y, x] for (x, y, z) in pts], dim=-1).double().cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-5, err
    # overlap: symmetric, diagonal = h^3 sum psi_j^2 (FP64 over the returned orbitals)
    Sd = S.cpu().numpy()
    np.testing.assert_array_equal(Sd, Sd.T)
    diag = H ** 3 * (psi.double() ** 2).sum(dim=(1, 2, 3)).cpu().numpy()
    np.testing.assert_allclose(np.diag(Sd), diag, rtol=3e-6)  # tensor-core overlap: bias below 1.5e-6
    np.testing.assert_allclose(sig2.cpu().numpy(), 1.0 / np.sqrt(np.diag(Sd)), rtol=1e-12)
    del psi
    torch.cuda.empty_cache()
