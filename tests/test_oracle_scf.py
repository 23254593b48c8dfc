"""Pins of the oracle's self-consistent loop.

* At self-consistency the output potential equals the input potential, the
  density integrates to the electron count, the orbitals are orthonormal.
* The converged single-orbital state is the dominant eigenvector of the
  step operator T(V) = K_xi - dt M_chi V of the final potential, i.e. the
  lowest eigenvector of the equivalent discretised Hamiltonian
  (1 - T(V)) / dt, found here by dense diagonalisation (Sec. 3,
  eigen-expansion argument).  With two orbitals the occupied span matches
  T's dominant two-dimensional invariant subspace.
* The converged answer does not depend on the potential mixing, or (for one
  orbital, whose fixed point is an eigenvector) on the cycle length.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lb, scf

from test_oracle_operators import _angle, _dense_T


def _orthonormal(psi, h):
    S = lb.gram(psi, h)
    return np.abs(S - np.eye(len(S))).max()


def test_helium_converges_with_invariants():
    w = W.he_24()
    st, res = scf.scf(w.n, w.h, w.molecule.xyz, w.molecule.Z, 1, n_inner=w.n_inner, e_tol=1e-6)
    assert res["converged"] and res["cycles"] < 30
    assert res["n_electrons"] == pytest.approx(2.0, abs=1e-12)
    assert _orthonormal(st.psi, w.h) < 1e-12
    # energies fall towards the variational minimum
    hist = np.array(res["history"])
    assert (np.diff(hist) < 1e-9).all()
    # the parts add up, the potential terms have the physical signs
    assert res["E_ext"] < 0 < res["E_H"] and res["E_xc"] < 0 < res["T_s"]
    assert res["eigenvalues"][0] < 0


def test_converged_energy_independent_of_mixing_and_cycle_length():
    w = W.he_24()
    args = (w.n, w.h, w.molecule.xyz, w.molecule.Z, 1)
    _, a = scf.scf(*args, n_inner=20, e_tol=1e-10, mix=0.5)
    _, b = scf.scf(*args, n_inner=20, e_tol=1e-10, mix=0.3)
    _, c = scf.scf(*args, n_inner=35, e_tol=1e-10, mix=0.5)
    assert a["E_total"] == pytest.approx(b["E_total"], abs=1e-8)
    assert a["E_total"] == pytest.approx(c["E_total"], abs=1e-8)
    assert a["eigenvalues"][0] == pytest.approx(c["eigenvalues"][0], abs=1e-7)


def test_single_orbital_fixed_point_is_dense_eigenvector():
    mol, n, h = W.helium(), (9, 10, 11), 0.6
    st, res = scf.scf(n, h, mol.xyz, mol.Z, 1, n_inner=30, e_tol=1e-12, max_cycles=400)
    assert res["converged"]
    assert np.abs(st.v_out - st.v_in).max() < 1e-7
    T = _dense_T(n, st.v_in, st.theta, st.dt)
    w, U = np.linalg.eig(T)
    k = int(np.argmax(w.real))
    assert _angle(st.psi[0], U[:, k].real) < 1e-9
    assert np.sqrt(st.last_S[0, 0]) == pytest.approx(float(w[k].real), abs=1e-10)


def test_two_orbital_span_is_dominant_invariant_subspace():
    mol, n, h = W.lih(2.0), (10, 10, 12), 0.6
    st, res = scf.scf(n, h, mol.xyz, mol.Z, 2, n_inner=30, e_tol=1e-12, max_cycles=400)
    assert res["converged"]
    T = _dense_T(n, st.v_in, st.theta, st.dt)
    w, U = np.linalg.eig(T)
    o = np.argsort(-w.real)
    Q, _ = np.linalg.qr(U[:, o[:2]].real)
    P, _ = np.linalg.qr(st.psi.reshape(2, -1).T)
    cosines = np.linalg.svd(Q.T @ P)[1]
    assert (1 - cosines).max() < 1e-7  # subspace angle below ~4e-4 rad
    # the lowest orbital is the dominant eigenvector itself
    assert _angle(st.psi[0], U[:, o[0]].real) < 1e-9
    assert _orthonormal(st.psi, h) < 1e-12
