/*
 * lbks.h -- C ABI of the GB300 lattice-kinetic Kohn-Sham solver.
 *
 * Method: Mendoza, Herrmann, Succi, "Lattice Boltzmann Model for Electronic
 * Structure Simulations".  Each occupied Kohn-Sham orbital j carries D3Q19
 * populations f_jp that relax in imaginary time by Eq. KSLB (Sec. 3):
 *
 *   f_jp(r + v_p, t+1) = f_jp - omega (f_jp - xi_p psi_j) - dt chi_p V psi_j
 *                        - omega xi_p sum_{k<j} Lambda_jk psi_k,
 *   psi_j = sum_p f_jp,  Lambda_jk = <psi_j|psi_k> / <psi_k|psi_k>,
 *
 * inside a self-consistent loop that rebuilds the density, the Hartree
 * potential (lattice Poisson), the LDA exchange-correlation potential, the
 * Cholesky orthonormalisation of the orbitals and the total energy.
 *
 * Conventions (every entry point):
 *  - Return value: LBKS_OK (0) or a positive LBKS_E* code; lbks_last_error()
 *    gives a one-line message for the calling thread.  No C++ exception
 *    crosses this boundary.
 *  - Units: atomic units (bohr, Hartree).  Grid site (i, j, k) of an
 *    nx x ny x nz grid at spacing h sits at ((i-(nx-1)/2) h, (j-(ny-1)/2) h,
 *    (k-(nz-1)/2) h): the box centre is the origin.
 *  - Grid arrays are x-fastest: index s = x + nx (y + ny z), N = nx ny nz.
 *  - Population arrays are f[j][p][z][y][x] (orbital, velocity, grid);
 *    orbital arrays psi[j][z][y][x]; the W field u[j-1][z][y][x] for
 *    j = 1 .. n_orb-1 (orbital 0 has none).
 *  - "dev" pointers are CUDA device pointers of the current device, owned by
 *    the caller; "host" pointers are host memory owned by the caller.
 *    Handles own their device memory.  A `stream` argument is a borrowed
 *    cudaStream_t (NULL = legacy default stream); the library never
 *    destroys it.  Device-pointer entry points are asynchronous on that
 *    stream unless stated otherwise.
 *  - Element type of population arrays follows `precision`: LBKS_FP64 ->
 *    double, LBKS_FP32 -> float, LBKS_BF16 -> bfloat16 (__nv_bfloat16);
 *    orbital and W-field arrays are double for LBKS_FP64, float otherwise.
 *    Potentials, densities, overlaps and energies are always double.
 *
 * D3Q19 velocity order (a data layout shared with callers):
 *    p:  0 ( 0, 0, 0)
 *        1 (+1, 0, 0)   2 (-1, 0, 0)   3 ( 0,+1, 0)   4 ( 0,-1, 0)
 *        5 ( 0, 0,+1)   6 ( 0, 0,-1)
 *        7 (+1,+1, 0)   8 (-1,-1, 0)   9 (+1,-1, 0)  10 (-1,+1, 0)
 *       11 (+1, 0,+1)  12 (-1, 0,-1)  13 (+1, 0,-1)  14 (-1, 0,+1)
 *       15 ( 0,+1,+1)  16 ( 0,-1,-1)  17 ( 0,+1,-1)  18 ( 0,-1,+1)
 *    lattice weights w = 1/3 (rest), 1/18 (axis), 1/36 (diagonal), c_s^2 = 1/3.
 */
#ifndef LBKS_H
#define LBKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBKS_MAX_ORB 64 /* orbitals per system handled by this build (above 8: separate Gram kernel) */

enum lbks_status {
    LBKS_OK = 0,
    LBKS_EINVAL = 1,    /* bad argument: sizes <= 0, h <= 0, n_orb out of range, null pointer */
    LBKS_ENOMEM = 2,    /* device allocation failed or byte budget exceeded */
    LBKS_ENOTCONV = 3,  /* max_cycles reached (results still filled) or overlap not positive definite */
    LBKS_ETIMEDOUT = 4, /* a bounded wait expired */
    LBKS_EBUSY = 5,     /* resource in use */
    LBKS_ECUDA = 6,     /* a CUDA runtime call failed; message has the CUDA error string */
    LBKS_ENOTFOUND = 7  /* unknown request id */
};

enum lbks_precision {
    LBKS_FP64 = 0, /* populations, collide and orbitals in double: the plain path */
    LBKS_FP32 = 1, /* populations, collide and orbitals in float; overlaps, energies, Poisson in double */
    LBKS_BF16 = 2  /* populations stored as bfloat16; collide, orbitals and W field in float;
                      overlaps, energies, Poisson in double */
};

/* What a relaxation step stores between steps.
 * LBKS_STORE_POPULATIONS: the 19 post-collision populations of every orbital
 *   (Eq. KSLB as written; any omega).
 * LBKS_STORE_PSI: omega = 1 only.  There the collision forgets the arriving
 *   populations and every post-collision population is xi_p psi - chi_p dt V psi
 *   + xi_p u (Sec. 3), a fixed combination of the orbital, the potential and
 *   the W field at its site.  The step keeps psi alone and applies the same
 *   pull-and-sum as a 19-point stencil:
 *     psi'(r) = sigma sum_p [(xi_p - dt chi_p Vc(r - v_p)) psi(r - v_p) + xi_p u(r - v_p)],
 *   Vc the potential of the collision that produced psi.  Identical results up
 *   to rounding; 2 orbital arrays instead of 38 population arrays.  FP64 or FP32. */
enum lbks_storage {
    LBKS_STORE_POPULATIONS = 0,
    LBKS_STORE_PSI = 1
};

/* Solver controls.  lbks_params_default() fills the defaults in brackets. */
typedef struct lbks_params {
    double omega;        /* BGK relaxation frequency, 0 < omega < 2 [1.0]; Sec. 3, Eq. LBeq */
    double theta;        /* second moment of the equilibrium xi_p psi [0.5]; sets
                            dt = theta h^2 (2 - omega) / omega (Sec. 3, D relation) */
    int n_inner;         /* relaxation steps per self-consistent cycle, >= 2 [50] */
    double mix;          /* linear potential mixing V <- mix V_out + (1-mix) V [0.5] */
    double e_tol;        /* stop rule on the total energy (below), Hartree, > 0 [1e-6] */
    int max_cycles;      /* [200] */
    int precision;       /* enum lbks_precision [LBKS_FP64] */
    double softening;    /* nuclear softening a (bohr); <= 0 means a = h [0] */
    double poisson_rtol; /* CG relative residual target [1e-11] */
    int poisson_max_iter;/* [20000] */
    double polish_tol;   /* LBKS_BF16 only: once every running system's |dE| < polish_tol, or
                            has stalled below 100 polish_tol (no longer halving over two cycles:
                            the bfloat16 noise floor), the populations are widened to FP32 and the
                            solve finishes in FP32, converging only after two FP32 cycles
                            (bfloat16 rounding would otherwise bound the accuracy); <= 0 never [1e-4] */
    int storage;         /* enum lbks_storage [LBKS_STORE_POPULATIONS]; LBKS_STORE_PSI needs omega = 1
                            and LBKS_FP64 or LBKS_FP32 */
    double eig_tol;      /* stop rule on the eigenvalues (largest change), Hartree; <= 0: not watched [2e-6] */
    double rho_tol;      /* stop rule on the density (relative L2 change); <= 0: not watched [2e-6] */
    uint64_t seed;       /* start orbitals: 0 the fixed offsets of lbks_set_geometry, else seeded offsets
                            (SplitMix64) [0]; the converged state does not depend on it */
    double poisson_adapt;/* > 0: each cycle's Hartree solve stops at the relative residual
                            max(poisson_rtol, min(1e-4, poisson_adapt * D)), D the relative density
                            change of the previous evaluation (an inexact solve while the density
                            still moves; at the stop rule's D <= rho_tol it is poisson_adapt * rho_tol
                            or tighter); 0: poisson_rtol always [0] */
} lbks_params;

/* Stop rule of lbks_scf and lbks_batch_scf (the paper stops once the orbital
 * energies no longer change, Sec. 4; the bound is this library's reading).
 * Cycles are grouped in blocks of 4.  At the end of block m three changes
 * since the end of block m-1 are watched: D_E = |E_m - E_(m-1)|, D_eig =
 * max_j |eps_j,m - eps_j,(m-1)| and D_rho = ||rho_m - rho_(m-1)|| / ||rho_m||.
 * Each is extended by its geometric tail D r / (1 - r), r the larger of the
 * last two ratios D_m / D_(m-1), D_(m-1) / D_(m-2), capped at 0.92 (0.98 per
 * cycle: a change that does not shrink counts as shrinking at that rate).  A
 * system has converged once, for each quantity with a positive tolerance
 * (e_tol, eig_tol, rho_tol), both its change and its tail are within the
 * tolerance, or its change is below the rounding floor 8 u s: u the unit
 * roundoff of the orbital values (2^-53 for LBKS_FP64, 2^-24 otherwise), s =
 * |E|, max_j |eps_j| and 1 for the three quantities; at least three blocks
 * run.  The tail estimates the distance left to the fixed point: a change
 * alone does not bound it when a cycle contracts the error slowly (the
 * Gram-Schmidt source of Eq. KSLB separates occupied orbitals of close
 * eigenvalues slowly, and that rotation leaks into the density); blocks let
 * a slow drift stand out of single-precision rounding noise, which does not
 * grow with the block length. */

void lbks_params_default(lbks_params* p);

/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to cap).  Returns the full message length. */
int lbks_last_error(char* buf, size_t cap);

/* Library version string, static storage. */
const char* lbks_version(void);

/* Number of kernels this library has enqueued in this process (a CUDA-graph
 * replay counts each of its kernel nodes).  Bookkeeping only. */
uint64_t lbks_kernel_launches(void);

/* Bounded device waits.  The tensor-core overlap kernel (more than eight FP32
 * orbitals) waits on mbarriers for its own tensor-core work; every such wait
 * gives up after a number of polls (default 2^22, far beyond any normal
 * completion).  A block whose wait gave up counts a timeout, writes NaN
 * partial sums -- the overlap, and with it the solve, becomes non-finite and
 * lbks_scf returns LBKS_ENOTCONV -- waits for its own tensor-core work
 * (2^22 polls at most, whatever the limit), frees its tensor memory and
 * returns, leaving the context usable.
 * lbks_set_wait_limit sets the polls of these waits for launches enqueued
 * afterwards (0: every wait gives up at once; a handle's captured cycle graph
 * keeps the value it was captured with) and returns the previous value;
 * process-wide, meant for tests of the failure path.  lbks_wait_timeouts
 * returns the number of blocks whose wait gave up on the current device
 * since the library was loaded (synchronous). */
uint32_t lbks_set_wait_limit(uint32_t polls);
uint64_t lbks_wait_timeouts(void);

/* ------------------------------------------------------------------ systems */
typedef struct lbks_system lbks_system;

/* A system is the paper's problem statement (Sec. 2: nuclei and electrons ->
 * Kohn-Sham orbitals, density and energies) on one grid: n_orb doubly occupied
 * orbitals, each carrying the D3Q19 populations of Eq. KSLB (Sec. 3).
 * Allocates all device state of one system on the current device: two
 * population buffers of n_orb*19*N elements, orbitals, W field, potentials,
 * CG vectors and reduction scratch.  Up to 8 orbitals the overlap products
 * are fused into the stream-collide kernel; above, a separate tiled Gram
 * kernel forms them.  EINVAL: nx, ny, nz < 2, h <= 0, n_orb < 1 or >
 * LBKS_MAX_ORB, bad params.  ENOMEM: cudaMalloc failed. */
int lbks_create_system(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb,
                       lbks_system** out);
int lbks_destroy_system(lbks_system* sys);

/* Bytes of device memory lbks_create_system would allocate. */
size_t lbks_system_bytes(const lbks_params* p, int nx, int ny, int nz, int n_orb);

/* Sets the nuclei (xyz: 3*n_atoms bohr relative to the box centre; Z: charges)
 * and resets the orbitals to the Gaussian start (orbital j on nucleus
 * order[j mod n_atoms] by decreasing Z, width 1.2 (1 + 0.35 (j div n_atoms))
 * bohr, offset 0.25 (sin(1+2.1j), sin(2+3.3j), sin(3+4.7j)) bohr,
 * Cholesky-orthonormalised; f* = xi psi).  Evaluates the starting density,
 * potentials and energy.  Synchronous.  EINVAL: atom outside the box,
 * n_atoms < 1, sum Z != 2 n_orb (closed-shell neutral only). */
int lbks_set_geometry(lbks_system* sys, int n_atoms, const double* xyz, const double* Z);

typedef struct lbks_result {
    double E_total;                   /* Hartree */
    double dE;                        /* |E_c - E_{c-1}| of the last cycle */
    double eigenvalues[LBKS_MAX_ORB]; /* Ritz values of the occupied subspace, ascending */
    double n_electrons;               /* h^3 sum rho */
    int cycles;
    int steps;                        /* relaxation steps (orbital-site updates = steps*n_orb*N) */
    int converged;
    int poisson_iters;                /* CG iterations, all cycles */
    double wall_s;
    double d_eig;                     /* D_eig of the last block of the stop rule */
    double d_rho;                     /* D_rho of the last block */
    double err_E, err_eig, err_rho;   /* geometric tails of the three block changes (the stop
                                         rule's estimates of the distance left); INFINITY before
                                         three blocks */
    double poisson_s;                 /* device time of the Hartree solves (CUDA events), all cycles */
} lbks_result;

/* The self-consistent loop of the Born-Oppenheimer scenario (Sec. 3.1: nuclei
 * fixed, orbitals relaxed by Eq. KSLB while the density, the Hartree and the
 * exchange-correlation potentials are rebuilt from them; Sec. 4 stops once
 * the orbital energies settle).  Each cycle runs n_inner - 1 relaxation
 * steps at fixed potential, one step that orthonormalises the orbitals
 * (Cholesky), then rebuilds density, potentials and energies and mixes the
 * potential.  Runs from the current state until the stop rule above holds
 * or max_cycles (ENOTCONV, result filled).  Blocking; all GPU work is queued
 * on `stream`.  ENOTCONV also when the overlap is not positive definite or
 * an energy is not finite; ECUDA on a CUDA failure. */
int lbks_scf(lbks_system* sys, void* stream, lbks_result* out);

/* Runs exactly n cycles (no convergence test); result as lbks_scf (one
 * result per system of a batched handle). */
int lbks_scf_cycles(lbks_system* sys, int n, void* stream, lbks_result* out);



typedef struct lbks_energy_terms {
    double T_s, E_ext, E_H, E_xc, E_nn, E_total;
    double eigenvalues[LBKS_MAX_ORB];      /* Ritz values, ascending */
    double orbital_energies[LBKS_MAX_ORB]; /* <psi_j|H|psi_j> per orbital */
    double n_electrons;
} lbks_energy_terms;

/* Stream-collide kernel variant (up to 8 orbitals; more use one kernel):
 *   0  one site per thread;
 *   1  two x-neighbouring sites per thread, two-element loads, x-shifted
 *      populations by warp shuffle (nx even and arrays 16-byte aligned, else 0);
 *   2  one site per thread, the next orbital's populations loaded before the
 *      current orbital collides (more loads in flight, fewer threads);
 *   3  omega = 1, FP32 or bfloat16 populations, any orbital count: the pulled
 *      populations of each (256-site tile, orbital) copied into a ring of
 *      shared-memory slots by the tensor memory accelerator (bulk copies, one
 *      producer warp, mbarriers), consumer warps collide one site each, and
 *      the overlap of the step is summed from the tile's orbitals in shared
 *      memory (no separate overlap kernel; N a multiple of 8 and 16-byte
 *      aligned arrays, else 0).
 * More than 8 orbitals: 0 is the one-orbital-per-thread kernel followed by the
 * tensor-core overlap; 1 and 2 are taken as 0.
 * In orbital storage (LBKS_STORE_PSI) the variants are 0: the stencil staged
 * in shared memory by tiles, 1: one site per thread from L1, 2: the stencil's
 * boxes copied into shared memory by the tensor memory accelerator, which also
 * forms the W source at any orbital count (nx a multiple of 16 / the orbital
 * value's bytes and 16-byte aligned arrays, else 0), 3: up to 8 orbitals, a
 * 32 x 8 column of sites marching along z with a ring of four planes in
 * shared memory, the next plane's loads in flight while a plane is summed
 * (more orbitals: 0).  More than 8 orbitals in orbital storage: 2 where it
 * applies, else 0.
 * mode 0 (default), tuned: the first lbks_set_geometry of each shape
 * (precision, orbitals, omega == 1 or not, grid, systems) times every
 * variant on the handle's buffers (a few launches, before they hold state)
 * and keeps the fastest for every later handle of that shape and for
 * lbks_relax_step of that shape (untuned shapes: variant 0).  mode 1 + v:
 * variant v forced.  Process-wide.  Returns the previous mode, or -1 for a
 * bad mode. */
int lbks_set_relax_variant(int mode);

/* Variant the handle's stream-collide runs, and the tuner's ms per launch of
 * each variant in ms[0..3] (may be NULL; negative: not measured by this
 * handle). */
int lbks_get_relax_variant(const lbks_system* sys, int* variant, double* ms);

/* Orbital storage, up to 8 orbitals: the tile shape of the staged stencil
 * (the box of every orbital's psi and of Vc that a block sums from shared
 * memory).  Shapes (x by y by z sites): 0 32 x 8 x 4 (the default),
 * 1 32 x 8 x 8, 2 64 x 4 x 4, 3 32 x 8 x 2, one site per thread; 4 64 x 8 x 4
 * and 5 64 x 8 x 2, two x-neighbouring sites per thread; 6 32 x 8 x 8 and
 * 7 32 x 8 x 4, one site per thread summing by velocity class from each
 * plane's in-plane sums (plane sums).  Shapes 1-7 need rows of whole 16-byte
 * pieces, 16-byte aligned psi in and out and Vc, and a box that fits a
 * block's shared memory; shapes 4 and 5 take FP32, or FP64 up to three
 * orbitals; shapes 6 and 7 FP32 up to six orbitals, or FP64 up to three;
 * elsewhere shape 0 runs.
 * The tuner times every shape that runs as itself on the first handle of a
 * grid shape and keeps the fastest with the staged kernel (then compares the
 * staged kernel with the others).  lbks_set_psi_tile(-1) restores that; 0..7
 * forces the shape for later handles and lbks_relax_step_psi calls.  Returns
 * the previous setting, or -2 for a bad shape (lbks_last_error says why).
 * lbks_get_psi_tile: the handle's shape and the tuner's ms per step of each
 * shape in ms[0..7] (may be NULL; negative: not timed). */
int lbks_set_psi_tile(int shape);
int lbks_get_psi_tile(const lbks_system* sys, int* shape, double* ms);

/* Energy terms of the last evaluation (after lbks_set_geometry or a cycle).
 * Sec. 2 states that the ground-state energy is a functional of the density
 * (Kohn-Sham formulation) but prints no expression; the standard Kohn-Sham
 * one is taken, with the terms of H_KS (Sec. 2): T_s + E_ext + E_H + E_xc
 * plus the nucleus-nucleus repulsion E_nn, T_s = 2 sum_j <psi_j|T_h|psi_j>,
 * T_h = (1 - K_xi) / (theta h^2) the kinetic operator of the equilibrium
 * stencil (Sec. 3).  The eigenvalues are the orbital energies E_j of Eq. KSE,
 * taken as Ritz values of the occupied subspace (the quantity Sec. 4's stop
 * rule watches).  Host copy; synchronous. */
int lbks_energy(const lbks_system* sys, lbks_energy_terms* out);

/* Hellmann-Feynman forces on the nuclei (Born-Oppenheimer, Sec. 3.1 with the
 * nuclei then moved): minus the explicit derivative of the total energy,
 *   F_I = Z_I h^3 sum_r rho(r) (r - R_I) / (|r - R_I|^2 + a^2)^(3/2)
 *         + sum_{J != I} Z_I Z_J (R_I - R_J) / |R_I - R_J|^3     (Ha/bohr),
 * at the density of the last evaluation (a is the softening).  At
 * self-consistency this is -dE_total/dR_I up to the scheme's
 * non-variational terms.  forces: host, 3 * n_atoms doubles (x, y, z per
 * nucleus, the order of lbks_set_geometry); EINVAL when cap is smaller or no
 * geometry is set.  The electron-nucleus sum runs on the device (one
 * deterministic grid reduction), the nucleus-nucleus sum on the host.
 * Synchronous. */
int lbks_forces(lbks_system* sys, double* forces, size_t cap);
int lbks_batch_forces(lbks_system* sys, int system, double* forces, size_t cap);

/* Moves the nuclei of a single-system handle (same count and charges) and
 * keeps the orbitals as the start of the next lbks_scf (warm start):
 * rebuilds V_ext, and the potential and energies of the current orbitals at
 * the new positions (unmixed).  xyz: 3 * n_atoms doubles, inside the box
 * (EINVAL otherwise).  Synchronous. */
int lbks_move_atoms(lbks_system* sys, const double* xyz);

/* Born-Oppenheimer molecular dynamics of a single-system handle (the nuclei
 * moved on the SCF ground-state surface, Sec. 3.1): velocity Verlet,
 *   R <- R + dt v + dt^2 F / (2 m),  SCF at R (warm start),  v <- v + dt (F + F') / (2 m),
 * with the Hellmann-Feynman forces of lbks_forces.  Atomic units: dt in
 * hbar/Ha, masses in electron masses (n_atoms doubles), velocities in
 * bohr hbar^-1 Ha (3 n_atoms, in: initial, out: final).  energies (may be
 * NULL): (n_steps + 1) x 2 doubles, E_total of the electrons and nuclei and
 * the nuclear kinetic energy at each step (step 0: the start).  xyz_traj (may
 * be NULL): (n_steps + 1) x 3 n_atoms positions.  Every step's SCF must
 * converge (LBKS_ENOTCONV otherwise, the arrays filled up to that step). */
int lbks_md(lbks_system* sys, int n_steps, double dt, const double* masses, double* velocities, void* stream,
            double* energies, double* xyz_traj);

/* Born-Oppenheimer geometry relaxation of a single-system handle: SCF, forces,
 * then quasi-Newton moves R <- R + alpha H F (H: BFGS estimate of the inverse
 * Hessian, starting from step * I; no nucleus moved more than 0.2 bohr per
 * move), each followed by a warm-started SCF.  A move that lowers E_total is
 * kept (H updated from the change of R and F, alpha back towards 1);
 * otherwise it is undone and alpha halves.  Stops when the largest
 * |F_I| < fmax (Ha/bohr): LBKS_OK; after max_steps moves: LBKS_ENOTCONV with
 * the results filled.  step: the initial inverse-Hessian scale (bohr^2/Ha).
 * fixed: n_atoms flags (non-zero: the nucleus stays where it is and its force
 * is not counted), or NULL for none.  out: the SCF result at the returned geometry, with
 * cycles, steps, poisson_iters and wall_s summed over every SCF run; xyz_out:
 * 3 * n_atoms doubles (may be NULL); steps_out: moves tried (may be NULL).
 * The handle is left at the returned geometry, relaxed there. */
int lbks_relax_geometry(lbks_system* sys, int max_steps, double fmax, double step, const int* fixed,
                        void* stream, lbks_result* out, double* xyz_out, int* steps_out);

/* ---------------------------------------------------------------------------
 * Concurrent dynamics (Sec. 3, "Concurrent Dynamics", Eq. KSLBCD): electrons
 * and nuclei moved together.  The paper prints the two-step, time-centred
 * update f(r + v h; t + h) = f(r - v h; t - h) + 2h (U + iV + iW) with
 * U_jp = kappa w_p q_p E_j phi_j, but no kinetic term, no rule for kappa and
 * no start.  It is read here as the real-time counterpart of the omega = 1
 * ground-state step (Wick rotation of Sec. 3's first equation), with the
 * complex orbitals phi_j as state and its own step tau:
 *   phi_j(t + tau) = phi_j(t - tau) + 2i (tau/dt) D_j(phi(t)) + 2 tau kappa E_j (K_q phi_j)(t),
 *   D_j(r) = sum_p [xi_p a_j - dt chi_p V phi_j](r - v_p) - phi_j(r),   zero outside the box,
 *   a_j = phi_j - sum_{k<j} Lambda_jk phi_k,  Lambda_jk = <phi_k|phi_j> / <phi_k|phi_k>,
 *   K_q phi(r) = sum_p w_p q_p phi(r - v_p),  dt = theta h^2.
 * D_j = -dt H phi_j (+ the W source) with H = (1 - K_xi)/dt + K_chi V; an
 * eigenvector of H with eigenvalue eps rotates at Omega, sin(Omega tau) =
 * eps tau, and the scheme is stable while tau |eps| < 1 over the spectrum of
 * H (tau = dt / 2 by default).  Every n_pot steps the nuclei make a
 * velocity-Verlet step of n_pot tau under the Hellmann-Feynman forces of
 * rho = 2 sum_j |phi_j|^2 (Ehrenfest form), and V = V_ext + V_H + v_xc is
 * rebuilt from rho (no mixing).  Up to 8 orbitals; omega = 1 handles.
 * A level is [j][part][z][y][x]: part 0 real, 1 imaginary values of orbital j,
 * in the compute type (double for LBKS_FP64, float otherwise).  Lambda and
 * S are [j][k][2] doubles (real, imaginary). */
typedef struct lbks_cd_params {
    double tau;   /* real-time step (hbar/Ha), at most theta h^2; 0: theta h^2 / 2 */
    double kappa; /* gain of the U source (dimensionless); 0: no U source */
    int n_pot;    /* electron steps per potential rebuild and nuclear move; 0: 10 */
} lbks_cd_params;

/* Starts the dynamics of a single-system handle from its current orbitals
 * (normally an SCF ground state): level 0 = the orbitals (imaginary parts
 * zero), the potential rebuilt from them, the forces, and the second level by
 * Taylor expansion to second order, phi(tau) = phi + i s D(phi) -
 * s^2 D0(D0(phi)) / 2 + tau kappa E K_q phi (s = tau/dt, D0 without the W
 * source).  E_target: n_orb orbital energies (Ha) of the U source, or NULL
 * with kappa = 0.  energy (may be NULL): E_total and the electron count of the
 * start.  The handle's potential is replaced (a later lbks_scf restarts from
 * it).  Allocates the three levels on first use (6 n_orb N values).
 * Synchronous on the handle's stream. */
int lbks_cd_start(lbks_system* sys, const lbks_cd_params* p, const double* E_target, void* stream, double* energy);

/* n_blocks blocks of n_pot steps.  masses: n_atoms nuclear masses (electron
 * masses) and velocities: 3 n_atoms (bohr Ha/hbar; in: initial, out: final),
 * or masses NULL for fixed nuclei.  energies (may be NULL): n_blocks x 3
 * doubles after each block: E_total of the orbitals at the nuclei, the
 * nuclear kinetic energy and the electron count.  xyz_traj (may be NULL):
 * n_blocks x 3 n_atoms positions.  EINVAL if a nucleus leaves the box.
 * Synchronous. */
int lbks_cd_run(lbks_system* sys, int n_blocks, const double* masses, double* velocities, void* stream,
                double* energies, double* xyz_traj);

/* Host copy of a level (0: the older, 1: the current): 2 n_orb N doubles,
 * layout [j][part][z][y][x]. */
int lbks_cd_get_orbitals(const lbks_system* sys, int level, double* host, size_t cap);

/* Time since the start (hbar/Ha), steps taken (the start counts one) and the
 * forces at the current level (3 n_atoms doubles, may be NULL). */
int lbks_cd_get_state(const lbks_system* sys, double* time, int64_t* steps, double* forces, size_t cap);

/* One step of the dynamics on device arrays (the update above):
 * phi_next = phi_prev + 2i (tau/dt) D(phi) + u_j K_q phi_j with u_coef[j] =
 * 2 tau kappa E_j (device, n_orb doubles, or NULL: no U source).  phi_prev
 * may be NULL (taken as zero).  lambda: Lambda of phi (device, n_orb^2 x 2
 * doubles, strictly lower part used) or NULL: no W source.  S_next (may be
 * NULL): the overlap S[i][j] = <phi_next_i|phi_next_j> = h^3 sum conj(phi_i) phi_j;
 * lambda_next (with S_next, may be NULL): Lambda of phi_next.  phi_next must
 * not alias phi or phi_prev.  precision LBKS_FP64 or LBKS_FP32.  Up to 8
 * orbitals.  Asynchronous on stream. */
int lbks_cd_step(int precision, int nx, int ny, int nz, int n_orb, double h, double theta, double tau,
                 const void* phi_prev_dev, const void* phi_dev, const double* V_dev, const double* lambda_dev,
                 const double* u_coef_dev, void* phi_next_dev, double* S_next_dev, double* lambda_next_dev,
                 void* stream);

/* Kernel of later dynamics steps: -1 (default) the staged kernel (every
 * orbital's box with a one-site halo in shared memory) where the box leaves
 * two blocks per SM, else one site per thread from L1; 0 one site per thread;
 * 1 staged where it applies.  Returns the previous mode, or -2 for a bad mode
 * (lbks_last_error says why). */
int lbks_set_cd_kernel(int mode);

/* Overlap S and (lambda may be NULL) Lambda of one level of n_sites sites. */
int lbks_cd_overlap(int precision, size_t n_sites, int n_orb, double h, const void* phi_dev, double* S_dev,
                    double* lambda_dev, void* stream);

/* Host copies (synchronous) of the last evaluation's density rho (N doubles),
 * orthonormal orbitals (n_orb*N doubles) and potentials (N doubles each).
 * EINVAL if cap (elements) is too small. */
int lbks_get_density(const lbks_system* sys, double* host, size_t cap);
int lbks_get_orbitals(const lbks_system* sys, double* host, size_t cap);
int lbks_get_potential(const lbks_system* sys, int which /*0 V_in,1 V_out,2 V_H,3 V_ext*/,
                       double* host, size_t cap);

/* ---------------------------------------------------------------- batching
 * A batched handle holds n_systems systems of one grid shape, orbital count
 * and parameter set (e.g. a scan over geometries).  Every kernel of the
 * relaxation cycle, the Hartree solve and the reductions covers all systems
 * in one launch (system = blockIdx.y), and each relaxation cycle is one
 * CUDA-graph replay.  Systems advance in lock step; one whose |dE| drops
 * below e_tol stops and is skipped by every later launch.  Per-system
 * results equal those of single-system handles up to the summation order of
 * the reductions (block counts differ). */
int lbks_create_batch(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb, int n_systems,
                      lbks_system** out);
size_t lbks_batch_bytes(const lbks_params* p, int nx, int ny, int nz, int n_orb, int n_systems);
/* Stores system `system`'s nuclei (checks as lbks_set_geometry); nothing runs. */
int lbks_batch_set_geometry(lbks_system* sys, int system, int n_atoms, const double* xyz, const double* Z);
/* Gaussian starts and the first evaluation of every system (all must have
 * geometry).  Synchronous. */
int lbks_batch_init(lbks_system* sys);
/* Self-consistent loop of all systems; out[n_systems].  ENOTCONV if some
 * system did not converge within max_cycles (results still filled). */
int lbks_batch_scf(lbks_system* sys, void* stream, lbks_result* out);
int lbks_batch_energy(const lbks_system* sys, int system, lbks_energy_terms* out);
int lbks_batch_get_density(const lbks_system* sys, int system, double* host, size_t cap);

/* ------------------------------------------------------------------ serving
 * A request loop with continuous batching.  Each request is one closed-shell
 * single-point solve (grid, spacing, nuclei).  Worker slots (host threads,
 * each with its own CUDA stream on the server's device) take queued requests
 * in arrival order, skipping ahead to the first one whose device memory
 * (lbks_system_bytes) fits in the free budget; a request whose shape matches
 * an idle pooled system reuses it, so populations and potentials stay
 * resident between requests; idle pooled systems are freed, oldest first,
 * when a new shape needs the room.  Slots run concurrently, so the kernels
 * of different requests overlap on the GPU.  A request's result does not
 * depend on what else runs (fixed-order reductions, private scratch). */
typedef struct lbks_server lbks_server;

typedef struct lbks_request {
    int nx, ny, nz;     /* grid */
    double h;           /* spacing, bohr */
    int n_orb;          /* doubly occupied orbitals; sum Z must be 2 n_orb */
    int n_atoms;
    const double* xyz;  /* 3*n_atoms, bohr, box-centre origin; copied by lbks_submit */
    const double* Z;    /* n_atoms; copied */
    int precision;      /* < 0: server default */
    int n_inner;        /* <= 0: server default */
    double e_tol;       /* <= 0: server default */
    int max_cycles;     /* <= 0: server default */
} lbks_request;

typedef struct lbks_timing {
    double queue_s;   /* submit -> slot start */
    double run_s;     /* slot start -> result */
    double latency_s; /* submit -> result */
} lbks_timing;

typedef struct lbks_server_stats {
    int queued, running, pooled;
    uint64_t completed;
    size_t bytes_in_use, budget_bytes;
} lbks_server_stats;

/* budget_bytes = 0: 85 % of the device's free memory at creation.
 * defaults = NULL: lbks_params_default().  EINVAL: max_slots not in [1, 64]. */
int lbks_server_create(const lbks_params* defaults, size_t budget_bytes, int max_slots, lbks_server** out);
/* Stops the slots after their current requests, frees pooled systems. */
int lbks_server_destroy(lbks_server* srv);
/* Queues a copy of the request and returns its id at once.  EINVAL for a
 * malformed request, ENOMEM when it can never fit the budget. */
int lbks_submit(lbks_server* srv, const lbks_request* req, uint64_t* id);
/* *done = 1 once the request finished; then `out` (and `timing`, if not
 * NULL) are filled, the id is released and the return value is the solve's
 * status (LBKS_OK, LBKS_ENOTCONV, ...).  ENOTFOUND for an unknown id. */
int lbks_poll(lbks_server* srv, uint64_t id, lbks_result* out, lbks_timing* timing, int* done);
/* Blocks until the request finished (without releasing it) or timeout_s
 * passed (ETIMEDOUT). */
int lbks_server_wait(lbks_server* srv, uint64_t id, double timeout_s);
int lbks_server_get_stats(lbks_server* srv, lbks_server_stats* out);

/* ------------------------------------------------- step-level device kernels
 * These expose the kernels the solver is built from, on caller-owned device
 * buffers, so that each step can be checked on its own.                    */

/* One relaxation step (Eq. KSLB with the normalisation of Sec. 3) for
 * n_orb orbitals on an nx x ny x nz grid:
 *   f_jp(r)   = f_in_jp(r - v_p) + xi_p u_(j-1)(r - v_p)  (zero outside)
 *   f_jp     *= sigma_in[j];  psi_j = sum_p f_jp
 *   f_out_jp  = f_jp - omega (f_jp - xi_p psi_j) - dt chi_p V psi_j
 *   S         = h^3 psi psi^T;  lambda_jk = S_jk/S_kk (k<j);  sigma_out_j = 1/sqrt(S_jj)
 * f_out holds the collision WITHOUT the orthogonalisation source; that
 * source, -omega xi_p sum_k lambda_jk psi_k, is carried by the W field that
 * lbks_w_field writes from psi_out and lambda_out and the next step pulls
 * in.  f_in + xi u is the paper's post-collision state.
 * u_in: (n_orb-1)*N elements or NULL for u = 0.  V: N doubles.
 * sigma_in / sigma_out: n_orb doubles (may alias).  S_out, lambda_out:
 * n_orb^2 doubles (row-major, lambda strictly lower).  psi_out: n_orb*N.
 * f_in and f_out must not alias.  Scratch is library-managed device memory
 * (allocated once per device and size, reused).  Asynchronous on stream. */
int lbks_relax_step(int precision, int nx, int ny, int nz, int n_orb, double h,
                    double omega, double theta, double dt,
                    const void* f_in_dev, const void* u_in_dev, const double* V_dev,
                    const double* sigma_in_dev, void* f_out_dev, void* psi_out_dev,
                    double* S_out_dev, double* lambda_out_dev, double* sigma_out_dev,
                    void* stream);

/* The step of lbks_relax_step for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is an interface convenience.
 *
 * Who needs it: code that already owns every byte it may touch on the GPU --
 * a host application whose memory is fully carved up by another framework's
 * pool allocator, a plug-in that is not allowed to call cudaMalloc, or a
 * latency-critical server that cannot afford the implicit device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  Such a caller still
 * provides every input and output buffer; only the reduction scratch that
 * lbks_relax_step would allocate moves into a fixed array of this library.
 *
 * The scratch is a file-scope __device__ array of 2048 blocks x 36 doubles
 * plus a counter (about 590 KB); every GPU that loads the library holds it
 * until the process exits.  On the first call on a device (with that device
 * current) the library looks up the array's device address; make that
 * first call before starting any stream capture.  Nothing is allocated or
 * freed: no cudaMalloc, cudaFree or allocating library routine is called.
 * Each call clears the arrival counter and overwrites the partials before
 * reading them; the array otherwise keeps the last call's contents.  All
 * calls share the one array, so calls that overlap on the GPU (different
 * streams, or different host threads without ordering) race and give wrong
 * overlaps: order them on one stream.  EINVAL for n_orb > 8 (the array's
 * limit) and for every argument lbks_relax_step rejects; all three
 * precisions (LBKS_FP64, LBKS_FP32, LBKS_BF16) are accepted.  Arguments and
 * results are exactly those of lbks_relax_step, and so is the stream-collide
 * variant it runs (lbks_set_relax_variant). */
int lbks_relax_step_noalloc(int precision, int nx, int ny, int nz, int n_orb, double h,
                            double omega, double theta, double dt,
                            const void* f_in_dev, const void* u_in_dev, const double* V_dev,
                            const double* sigma_in_dev, void* f_out_dev, void* psi_out_dev,
                            double* S_out_dev, double* lambda_out_dev, double* sigma_out_dev,
                            void* stream);

/* One relaxation step in orbital storage (LBKS_STORE_PSI, omega = 1; Sec. 3,
 * Eq. KSLB with the populations written as xi_p psi - chi_p dt Vc psi + xi_p u):
 *   psi_out_j(r) = sigma_in_j sum_p [(xi_p - dt chi_p Vc(r - v_p)) psi_in_j(r - v_p)
 *                                    + xi_p u_j(r - v_p)],   zero outside the box,
 *   u_j = -sum_{k<j} lambda_in_jk psi_in_k   (the W source; omega = 1),
 * and, as lbks_relax_step, S = h^3 psi_out psi_out^T, lambda_out and sigma_out.
 * precision: LBKS_FP64 (psi double) or LBKS_FP32 (float).  psi_in, psi_out:
 * n_orb*N values, orbital-major, must not alias.  lambda_in: n_orb^2 doubles
 * (strictly lower part used; may alias lambda_out) or NULL for no W source.
 * Vc: N doubles, the potential of the collision that produced psi_in (zeros
 * when psi_in is a start orbital: f = xi psi has no potential term).
 * sigma_in may alias sigma_out.  Kernel: the one lbks_set_relax_variant
 * forces, else the TMA kernel where it applies (nx a multiple of 16 / the
 * value's bytes, psi_in and Vc 16-byte aligned), else the tiled one.  The TMA
 * kernel, and any kernel up to 8 orbitals, forms the W source inside the
 * step; otherwise more than 8 orbitals use library-managed scratch for u.
 * Asynchronous on stream. */
int lbks_relax_step_psi(int precision, int nx, int ny, int nz, int n_orb, double h, double theta, double dt,
                        const void* psi_in_dev, const double* lambda_in_dev, const double* Vc_dev,
                        const double* sigma_in_dev, void* psi_out_dev, double* S_out_dev,
                        double* lambda_out_dev, double* sigma_out_dev, void* stream);

/* Energy matrix of n_orb orbitals in the potential V (the orbital energies of
 * Eq. KSE as a Ritz problem; kinetic operator of the equilibrium stencil,
 * Sec. 3): out[j*n_orb + k] = H_jk = h^3 sum_r psi_j (T_h + V) psi_k and
 * out[n_orb^2 + j] = h^3 sum_r psi_j T_h psi_j, T_h psi = (psi - K_xi psi) /
 * (theta h^2), K_xi psi(r) = sum_p xi_p psi(r - v_p), psi = 0 outside the box.
 * psi: n_orb*N values (double for LBKS_FP64, float otherwise), orbital-major;
 * V: N doubles; out: n_orb^2 + n_orb doubles.  The solver's own kernel (FP32
 * orbitals: FP32 neighbour differences and products, FP64 sums over sites).
 * Asynchronous on stream. */
int lbks_energy_matrix(int precision, int nx, int ny, int nz, int n_orb, double h, double theta,
                       const void* psi_dev, const double* V_dev, double* out_dev, void* stream);

/* W field of the orthogonalisation source (Sec. 3, W_jp):
 * u_(j-1)(r) = -omega sum_{k<j} lambda_jk psi_k(r), j = 1..n_orb-1. */
int lbks_w_field(int precision, size_t n_sites, int n_orb, double omega,
                 const void* psi_dev, const double* lambda_dev, void* u_out_dev, void* stream);

/* Overlap matrix S = h^3 psi psi^T (the inner products behind sigma_j and
 * lambda_jk of Sec. 3 and behind the orthonormalisation), FP64 result.
 * psi: n_orb * n_sites values (FP64 for LBKS_FP64, else FP32), orbital-major.
 * S: n_orb^2 doubles, row-major, both triangles written.
 * tensor_cores = 0: SIMT products summed in FP64 (the orthonormalising
 * overlap of the solver).  tensor_cores = 1 and FP32 orbitals: the tcgen05
 * kernel of the solver's per-step overlap for more than eight orbitals --
 * each value split into bf16 hi + lo, FP32 accumulation in tensor memory over
 * at most 512 sites (truncating: a relative bias below ~1.5e-6 on S_jj), FP64
 * beyond; ignored for LBKS_FP64.  Asynchronous on stream. */
int lbks_overlap(int precision, size_t n_sites, int n_orb, double h, const void* psi_dev,
                 double* S_dev, int tensor_cores, void* stream);

/* Cholesky S = L L^T of an n x n SPD matrix on the device (FP64, one CTA),
 * writes L^{-1} (lower, row-major).  Sets *status_dev = 0, or j+1 if the
 * j-th pivot is not positive. */
int lbks_cholesky_inverse(int n, const double* S_dev, double* Linv_dev, int* status_dev, void* stream);

/* In-place orthonormalisation at every site: f_jp <- sum_k Linv_jk f_kp and
 * psi_j <- sum_k Linv_jk psi_k (either pointer may be NULL). */
int lbks_orth_apply(int precision, size_t n_sites, int n_orb, const double* Linv_dev,
                    void* f_dev, void* psi_dev, void* stream);

/* Hartree potential: solves (6 V - sum of face neighbours) = 4 pi h^2 rho
 * with ghost values from the monopole+dipole+quadrupole of rho about the box
 * centre (Sec. 2, Hartree integral).  v_dev holds the warm start on entry
 * and the solution on exit.  Conjugate gradients in FP64 until relative
 * residual <= rtol or max_iter.  Synchronous (reads back the iteration count
 * and residual).  ENOTCONV if max_iter is reached. */
int lbks_hartree(int nx, int ny, int nz, double h, const double* rho_dev, double* v_dev,
                 double rtol, int max_iter, int* iters_out, double* relres_out, void* stream);

/* Spin-unpolarised LDA per site: Slater exchange + Perdew-Zunger-81
 * correlation; eps and v zero where rho < 1e-14 (Sec. 2, V_xc). */
int lbks_lda(size_t n_sites, const double* rho_dev, double* eps_dev, double* v_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBKS_H */
