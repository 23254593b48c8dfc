"""Converged solves against the oracle's fixed point, through the C ABI.

The self-consistent loop of the Born-Oppenheimer scenario (Sec. 3.1) stops
by the rule of include/lbks.h (changes of the energy, the eigenvalues and
the density, each with its geometric tail).  Each case here runs the GPU
solve to that rule with the default tolerances and compares the delivered
result with the oracle's solution of the same case converged far tighter
(tests/golden/converged_<case>.npz, written by make_goldens.py from oracle/
alone):

    |Delta E_total| <= 1e-5 Ha,  eigenvalues <= 1e-5 Ha,
    relative density L2 <= 1e-5 (of 4^3-site block sums on the 96^3 and
    128^3 grids, whose full density is not stored).

Cases: He, H2, LiH, H2O and CH4 (1, 1, 2, 5 and 5 orbitals) and a water
dimer (10 orbitals: the wide path, tensor-core overlap), in FP64, FP32 and
BF16 populations with the FP32 polish, FP32 orbital storage; the served mix
of five molecules in BF16 + polish and in FP32 orbital storage; the 128^3
methane and 96^3 water bench workloads in FP32."""
import json
import os
import time

import numpy as np
import pytest

import workloads as W

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

E_TOL, EIG_TOL, RHO_TOL = 1e-5, 1e-5, 1e-5
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SMALL = ["he_24", "h2_24", "lih_28", "h2o_38", "ch4_32", "dimer_36"]
MODES = {"fp64": (0, 0), "fp32": (1, 0), "bf16_polish": (2, 0), "fp32_psi": (1, 1)}


def golden(name):
    z = np.load(os.path.join(GOLDEN, f"converged_{name}.npz"))
    return {"E_total": float(z["E_total"]), "eigenvalues": np.asarray(z["eigenvalues"]), "rho": z["rho"],
            "block": int(z["block"]), "meta": json.loads(str(z["meta"]))}


def block_sums(rho, b):
    if b == 1:
        return rho
    nz, ny, nx = rho.shape
    r = rho[: nz - nz % b, : ny - ny % b, : nx - nx % b]
    return r.reshape(nz // b, b, ny // b, b, nx // b, b).sum(axis=(1, 3, 5))


def check(res, rho, ref, label):
    no = len(ref["eigenvalues"])
    dE = abs(res["E_total"] - ref["E_total"])
    dEig = float(np.abs(np.sort(res["eigenvalues"][:no]) - ref["eigenvalues"]).max())
    r = block_sums(rho, ref["block"])
    dRho = float(np.linalg.norm(r - ref["rho"]) / np.linalg.norm(ref["rho"]))
    print(f"{label}: cycles {res['cycles']}, |dE| {dE:.2e}, eig {dEig:.2e}, rho L2 {dRho:.2e}")
    assert res["converged"], label
    assert dE <= E_TOL, (label, dE)
    assert dEig <= EIG_TOL, (label, dEig)
    assert dRho <= RHO_TOL, (label, dRho)


def solve(lbks, w, prec, storage, **extra):
    s = lbks.System(w.n, w.h, w.n_orb, precision=prec, n_inner=w.n_inner, theta=w.theta, omega=w.omega,
                    mix=w.mix, max_cycles=400, poisson_rtol=1e-12, storage=storage, **extra)
    s.set_geometry(w.molecule.xyz, w.molecule.Z)
    res = s.scf()
    rho = s.density()
    s.close()
    return res, rho


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("case", SMALL)
def test_converged_solve_matches_oracle_fixed_point(case, mode):
    torch, lbks = require_gpu()
    w = W.converged_cases()[case]
    prec, storage = MODES[mode]
    res, rho = solve(lbks, w, prec, storage)
    check(res, rho, golden(case), f"{case} {mode}")


@pytest.mark.parametrize("case", ["ch4_128", "h2o_96"])
def test_bench_workload_solve_matches_oracle_fixed_point(case):
    """The 128^3 methane and 96^3 water workloads of the bench, FP32
    populations, in the bench's launch configuration (tuned kernels)."""
    torch, lbks = require_gpu()
    w = W.converged_cases()[case]
    res, rho = solve(lbks, w, 1, 0)
    check(res, rho, golden(case), f"{case} fp32")


SERVED = ["he_24", "h2_24", "lih_28", "h2o_38", "ch4_32"]


@pytest.mark.parametrize("mode", ["bf16_polish", "fp32_psi"])
def test_served_mix_matches_oracle_fixed_points(mode):
    """Five molecules submitted at once (twice each) to a server with three
    slots; every served result is within the stated tolerances of its
    oracle fixed point."""
    torch, lbks = require_gpu()
    prec, storage = MODES[mode]
    cases = W.converged_cases()
    srv = lbks.lbks_server_create(lbks.lbks_params_default(precision=prec, storage=storage, max_cycles=400,
                                                           poisson_rtol=1e-12), 0, 3)
    order = SERVED * 2
    try:
        ids = [lbks.lbks_submit(srv, cases[c].n, cases[c].h, cases[c].molecule.xyz, cases[c].molecule.Z,
                                n_inner=cases[c].n_inner) for c in order]
        out, t_end = {}, time.time() + 600.0
        while len(out) < len(ids):
            assert time.time() < t_end, "serving loop did not finish"
            for rid in ids:
                if rid not in out:
                    r = lbks.lbks_poll(srv, rid)
                    if r is not None:
                        out[rid] = r
            time.sleep(0.002)
    finally:
        lbks.lbks_server_destroy(srv)
    for c, rid in zip(order, ids):
        res, _ = out[rid]
        ref = golden(c)
        no = len(ref["eigenvalues"])
        assert res["converged"], c
        assert abs(res["E_total"] - ref["E_total"]) <= E_TOL, (c, res["E_total"], ref["E_total"])
        np.testing.assert_allclose(np.sort(res["eigenvalues"][:no]), ref["eigenvalues"], atol=EIG_TOL)


def test_converged_state_does_not_depend_on_the_start():
    """Two seeded starts (and the fixed start) of CH4 reach the same fixed
    point within the tolerances: the stop rule's bound holds from any start."""
    torch, lbks = require_gpu()
    w = W.converged_cases()["ch4_32"]
    ref = golden("ch4_32")
    for seed in (0, 7, 2024):
        s = lbks.System(w.n, w.h, w.n_orb, precision=1, n_inner=w.n_inner, max_cycles=400, poisson_rtol=1e-12,
                        seed=seed)
        s.set_geometry(w.molecule.xyz, w.molecule.Z)
        res = s.scf()
        check(res, s.density(), ref, f"ch4_32 fp32 seed {seed}")
        s.close()


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_psi"])
@pytest.mark.parametrize("case", ["lih_28", "ch4_32", "dimer_36"])
def test_inexact_hartree_solves_reach_the_same_fixed_point(case, mode):
    """lbks_params.poisson_adapt: each cycle's Hartree solve stops at a
    tolerance tied to the previous density change (1e-4 at most); the solve
    still ends within the tolerances of the oracle's fixed point, with fewer
    CG iterations than at the fixed tolerance."""
    torch, lbks = require_gpu()
    w = W.converged_cases()[case]
    prec, storage = MODES[mode]
    res, rho = solve(lbks, w, prec, storage, poisson_adapt=1e-3)
    check(res, rho, golden(case), f"{case} {mode} inexact Hartree")
    fixed, _ = solve(lbks, w, prec, storage)
    per = lambda r: r["poisson_iters"] / r["cycles"]
    print(f"CG iterations per cycle: {per(res):.2f} inexact, {per(fixed):.2f} fixed")
    assert per(res) < per(fixed)
