"""Writes the oracle's converged solutions of workloads.converged_cases()
into this folder (converged_<case>.npz), for the GPU parity tests of
converged solves.

Calls only the oracle (and the seeded inputs of `workloads`): nothing here
comes from the CUDA path.  Each case runs the oracle's self-consistent loop
(oracle.scf.scf) with tolerances far below the tests' (E 1e-10 Ha,
eigenvalues and density 1e-8), i.e. to the fixed point of the scheme; grids
above 64^3 sites run the orbital-storage form of the same steps (oracle.psi,
identical up to rounding at omega = 1).

Stored per case: E_total, the ascending eigenvalues, the electron count, the
cycles and steps taken, the changes and tails of the last cycle, and the
density -- in full up to 64^3 sites, else as sums over 4 x 4 x 4 blocks of
sites (with the block size stored).

    python tests/golden/make_goldens.py [case ...]     (default: all)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import scf  # noqa: E402

TOLS = {"e_tol": 1e-10, "eig_tol": 1e-8, "rho_tol": 1e-8}
FULL_RHO_SITES = 64 ** 3
BLOCK = 4


def block_sums(rho, b):
    nz, ny, nx = rho.shape
    r = rho[: nz - nz % b, : ny - ny % b, : nx - nx % b]
    return r.reshape(nz // b, b, ny // b, b, nx // b, b).sum(axis=(1, 3, 5))


def run(name, w):
    storage = "psi" if w.sites > FULL_RHO_SITES else "populations"
    t0 = time.time()
    st, res = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, w.n_orb, n_inner=w.n_inner, max_cycles=2000,
                      mix=w.mix, theta=w.theta, omega=w.omega, storage=storage, **TOLS)
    secs = time.time() - t0
    if not res["converged"]:
        raise RuntimeError(f"{name}: oracle did not converge in {res['cycles']} cycles")
    full = w.sites <= FULL_RHO_SITES
    meta = {"case": name, "workload": w.name, "grid": list(w.n), "h": w.h, "n_orb": w.n_orb,
            "n_inner": w.n_inner, "mix": w.mix, "theta": w.theta, "omega": w.omega, "storage": storage,
            "tolerances": TOLS, "cycles": res["cycles"], "steps": res["steps"], "dE": res["dE"],
            "d_eig": res["d_eig"], "d_rho": res["d_rho"], "err_E": res["err_E"], "err_eig": res["err_eig"],
            "err_rho": res["err_rho"], "oracle_seconds": round(secs, 1),
            "rho": "full" if full else f"sums over {BLOCK}^3 blocks"}
    np.savez_compressed(os.path.join(HERE, f"converged_{name}.npz"), E_total=np.float64(res["E_total"]),
                        eigenvalues=np.asarray(res["eigenvalues"]), n_electrons=np.float64(res["n_electrons"]),
                        rho=st.rho if full else block_sums(st.rho, BLOCK), block=np.int64(1 if full else BLOCK),
                        meta=np.array(json.dumps(meta)))
    print(json.dumps(meta), flush=True)


def main(names):
    cases = W.converged_cases()
    for name in names or list(cases):
        run(name, cases[name])


if __name__ == "__main__":
    main(sys.argv[1:])
