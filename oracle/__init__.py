"""FP64 CPU oracle for the lattice-kinetic Kohn-Sham method (Mendoza, Herrmann,
Succi, "Lattice Boltzmann Model for Electronic Structure Simulations").

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The CUDA library never calls it and shares no code, tables or
constants with it; both sides are fed the same inputs from ``workloads``.

Everything here is plain numpy in float64, written to be read against the
paper: each function names the section / equation it follows.  There is no
blocking, fusion or reordering beyond what the equations state.

Modules
-------
lattice  D3Q19 velocities and weights; equilibrium weights xi_p and source
         weights chi_p (Sec. 3, equilibrium and source definitions).
lb       pull streaming, BGK collision with potential and orthogonalisation
         sources (Eqs. LBeq, KSLB, W_jp), per-step normalisation and the
         Gram/Lambda reduction; Cholesky orthonormalisation.
poisson  Hartree potential: 7-point lattice Poisson with multipole
         boundary values, solved by conjugate gradients (Sec. 2, Hartree
         integral of H_KS; the paper gives no algorithm).
lda      Slater exchange + Perdew-Zunger-81 correlation, spin-unpolarised
         (Sec. 2, V_xc[rho]; the paper's own runs used B88/LYP).
energy   kinetic operator of the equilibrium stencil, total energy terms and
         orbital eigenvalues (Rayleigh quotients).
scf      initial orbitals, external potential, the self-consistent loop
         (Born-Oppenheimer ground state at fixed nuclei, Sec. 3.1).

Parity pins: every function above is pinned by the ``-m "not gpu"`` tests
against closed forms, exact lattice identities, brute-force dense operators
or physical limits.  Absolute total energies of softened-nucleus LDA atoms
at these grid spacings have no published closed form: for the full SCF the
pins are its invariants and the pinned pieces it is built from.
"""
