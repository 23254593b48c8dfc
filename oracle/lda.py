"""Local density approximation for exchange-correlation (oracle; test
infrastructure only).

Sec. 2 writes V_xc[rho] without fixing a functional (the paper's own runs
use B88 exchange and LYP correlation, Sec. 4).  The functional here is the
spin-unpolarised LDA: Slater exchange and the Perdew-Zunger 1981
parametrisation of the Ceperley-Alder correlation energy (Phys. Rev. B 23,
5048, Appendix C).

    r_s = (3 / (4 pi rho))^(1/3)
    eps_x = -(3/4) (3/pi)^(1/3) rho^(1/3),     v_x = (4/3) eps_x
    r_s >= 1: eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
              v_c   = eps_c (1 + 7/6 beta1 sqrt(r_s) + 4/3 beta2 r_s)
                            / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s
              v_c   = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2D - C)/3 r_s

The potential is v = d(rho eps)/d rho = eps - (r_s/3) d eps/d r_s.
Below RHO_FLOOR both eps_xc and v_xc are taken as zero.
"""
import numpy as np

RHO_FLOOR = 1e-14

GAMMA, BETA1, BETA2 = -0.1423, 1.0529, 0.3334
A_PZ, B_PZ, C_PZ, D_PZ = 0.0311, -0.048, 0.0020, -0.0116


def exchange(rho):
    ex = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * np.cbrt(rho)
    return ex, (4.0 / 3.0) * ex


def correlation(rs):
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    hi = rs >= 1.0
    lo = ~hi
    s = np.sqrt(rs[hi])
    den = 1.0 + BETA1 * s + BETA2 * rs[hi]
    ec[hi] = GAMMA / den
    vc[hi] = ec[hi] * (1.0 + (7.0 / 6.0) * BETA1 * s + (4.0 / 3.0) * BETA2 * rs[hi]) / den
    r = rs[lo]
    lr = np.log(r)
    ec[lo] = A_PZ * lr + B_PZ + C_PZ * r * lr + D_PZ * r
    vc[lo] = A_PZ * lr + (B_PZ - A_PZ / 3.0) + (2.0 / 3.0) * C_PZ * r * lr + (2.0 * D_PZ - C_PZ) / 3.0 * r
    return ec, vc


def lda_xc(rho):
    """(eps_xc, v_xc) per site, both zero where rho < RHO_FLOOR."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho >= RHO_FLOOR
    r = rho[m]
    ex, vx = exchange(r)
    rs = np.cbrt(3.0 / (4.0 * np.pi * r))
    ec, vc = correlation(rs)
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v
