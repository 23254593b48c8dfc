"""Helpers shared by the GPU parity tests (device transfer, the xi weights for
rebuilding the paper's post-collision state from the split GPU outputs)."""
import numpy as np

from oracle import lattice


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA; run them with -m gpu on a GPU machine")
    from paper_1507_07666_gb300 import build
    build.build()
    from paper_1507_07666_gb300 import lbks
    return torch, lbks


def to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_np(t):
    return t.detach().double().cpu().numpy()


def paper_state(f_split, u, theta):
    """f* = f_split + xi_p u_{j-1} for j >= 1 (the W source carried by u)."""
    xi = lattice.xi(theta)
    out = f_split.copy()
    for j in range(1, f_split.shape[0]):
        out[j] += xi[:, None, None, None] * u[j - 1][None]
    return out


def rel_err(a, b):
    """max |a - b| / max |b|"""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
