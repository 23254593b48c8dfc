// Internal declarations shared by the translation units of liblbks.
// Not part of the public ABI (see include/lbks.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace lbks {

constexpr int kThreads = 256;  // block size of every grid kernel
constexpr int kMaxOrb = 8;       // orbitals handled by the fused stream-collide kernel
constexpr int kMaxOrbWide = 64;  // orbitals handled at all (wide kernels above kMaxOrb)
constexpr int kEmatWideStride = kMaxOrbWide * kMaxOrbWide + kMaxOrbWide;
constexpr int kMpStride = 16;    // doubles per system: multipoles of rho
constexpr int kEmatStride = 80;  // doubles per system: H (NO^2) and kinetic (NO) terms
constexpr int kE4Stride = 4;     // doubles per system: energy integrals

// D3Q19 velocity components in the order of include/lbks.h.
__host__ __device__ constexpr int vel(int p, int a) {
    constexpr int t[19][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[p][a];
}
// |v_p|^2: 0 rest, 1 axis, 2 face diagonal.
__host__ __device__ constexpr int vclass(int p) {
    return vel(p, 0) * vel(p, 0) + vel(p, 1) * vel(p, 1) + vel(p, 2) * vel(p, 2);
}

// Unsigned 32-bit division by a runtime constant d >= 1 for n < 2^31:
// q = (umulhi(n, m) + n) >> l with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994).
struct FastDiv {
    uint32_t d, m, l;
    FastDiv() : d(1), m(1), l(0) {}
    explicit FastDiv(uint32_t dd) : d(dd) {
        l = 0;
        while ((1ull << l) < dd) ++l;
        m = (uint32_t)(((1ull << 32) * ((1ull << l) - dd)) / dd + 1);
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
        return (__umulhi(n, m) + n) >> l;
#else
        return (uint32_t)((((uint64_t)n * m) >> 32) + n) >> l;
#endif
    }
};

// Lattice coefficients of one relaxation, per velocity class.
struct Coef {
    double omega, dt, theta, h;
    double xi[3];   // w_p (1 + (theta - 1/3) q_p)
    double chi[3];  // w_p [1 - (v^2 - 1) * 3/2]
};
Coef make_coef(double omega, double theta, double dt, double h);

// One grid shape; a launch covers gridDim.y systems of this shape (system =
// blockIdx.y, arrays of consecutive systems at fixed strides).  `active`
// (optional, one flag per system) lets finished systems skip a launch.
struct Grid {
    int nx, ny, nz;
    uint32_t N;
    FastDiv divx, divy;
    const int* active = nullptr;
};
Grid make_grid(int nx, int ny, int nz);

// Reduction scratch: per-block partial sums and one arrival counter that the
// last block resets, one region of each per system of a batched launch.
// Kernels sharing a Scratch must be stream-ordered.
struct Scratch {
    double* partial = nullptr;  // systems * max_blocks * max_vals doubles
    unsigned* counter = nullptr;  // one per system
    int max_blocks = 0;           // blocks per system
    int max_vals = 0;
    int systems = 1;
};

// Overlap S = h^3 Psi Psi^T of N_O FP32 orbitals per system (N_O <= kMaxOrbWide)
// on the tensor cores (bf16 hi/lo split, FP64 block and grid sums); with lam
// also Lambda and sigma as the relaxation step needs them.  drain_tiles: tiles
// of 64 sites summed in TMEM before the FP64 fold (0: the default, 8; the
// 33..40-orbital kernel drains after whole pairs of tiles).
cudaError_t launch_gram_tc(int NO, const Grid& g, double h, const float* psi, double* S, double* lam,
                           double* sigma, const Scratch& sc, int B, cudaStream_t st, int drain_tiles = 0);
// Blocks of the tensor-core Gram kernel whose bounded mbarrier waits expired
// (device counter since the library was loaded; 0 unless the hardware stalled).
unsigned gram_tc_timeouts();
// Polls of the tensor-core Gram kernel's mbarrier waits for later launches;
// returns the previous value.
uint32_t set_gram_tc_wait_limit(uint32_t polls);
// The current limit (polls) for the main mbarrier waits of later launches.
uint32_t device_wait_limit();

// Launch bookkeeping.
void count_launches(uint64_t n);
// Records the calling thread's error message (returned by lbks_last_error); returns code.
int set_last_error(int code, const char* msg);
int num_sms();

// Stream-collide variants (up to kMaxOrb orbitals): one site per thread; two
// x-neighbouring sites per thread with two-element loads (needs an even nx
// and aligned arrays, else the one-site kernel runs); one site per thread
// with the next orbital's populations loaded before the current one collides.
constexpr int kRelaxSites = 0;
constexpr int kRelaxPairs = 1;
constexpr int kRelaxPrefetch = 2;
constexpr int kRelaxBulk = 3;  // omega = 1: populations copied into shared memory by the tensor memory
                               // accelerator, overlap fused (lbks_bulk.cuh)
constexpr int kRelaxVariants = 4;
constexpr int kRelaxVariantMask = 3;
// In orbital storage the same ids pick the stencil kernel: staged in shared
// memory by the threads, one site per thread from L1, or staged by the tensor
// memory accelerator (psi_tma_applies; forms the W source itself at any
// orbital count, so no W field runs with it).
constexpr int kPsiKernelTiled = kRelaxSites;
constexpr int kPsiKernelDirect = kRelaxPairs;
constexpr int kPsiKernelTma = kRelaxPrefetch;
constexpr int kPsiKernelZ = kRelaxBulk;  // up to kMaxOrb orbitals: marching along z, a ring of planes
// The staged kernel (up to kMaxOrb orbitals) takes its tile shape from the
// kernel id's bits from kPsiShapeShift on (0: the default 32 x 8 x 4).
constexpr int kPsiShapeShift = 8;
constexpr int kPsiShapes = 8;
// The shapes: TX x (kThreads XW / TX) x TZ sites, XW x-neighbouring sites per
// thread.  XW = 2 sums two sites from 8- or 16-byte shared-memory loads (half
// the load instructions of the 19-point sums).  PL: plane sums -- the pulled
// sums by velocity class (rest, faces, edges) from each plane's in-plane face
// and diagonal sums, carried along the thread's z-column.
constexpr int kPsiTileTX[kPsiShapes] = {32, 32, 64, 32, 64, 64, 32, 32};
constexpr int kPsiTileTZ[kPsiShapes] = {4, 8, 4, 2, 4, 2, 8, 4};
constexpr int kPsiTileXW[kPsiShapes] = {1, 1, 1, 1, 2, 2, 1, 1};
constexpr bool kPsiTilePL[kPsiShapes] = {false, false, false, false, false, false, true, true};
// Whether shape k runs as itself for no orbitals of elem bytes (else the
// default shape runs): its box of the no orbitals and Vc, rows padded by 16
// bytes on each side, fits a block's 227 KB of shared memory, and at two
// sites per thread or with plane sums the accumulators fit the registers
// (FP32 -- up to six orbitals with plane sums -- or FP64 up to three).
constexpr bool psi_tile_runs(int elem, int no, int k) {
    return k >= 0 && k < kPsiShapes &&
           (size_t)(no + 1) * (size_t)(kPsiTileTX[k] + 2 * (16 / elem)) * (size_t)(kThreads * kPsiTileXW[k] / kPsiTileTX[k] + 2) *
                   (size_t)(kPsiTileTZ[k] + 2) * (size_t)elem <=
               227 * 1024 &&
           (kPsiTileXW[k] == 1 || elem <= 4 || no <= 3) &&
           (!kPsiTilePL[k] || (elem <= 4 && no <= 6) || no <= 3);
}
// The TMA kernel's tensor maps need rows of whole 16-byte units (nx a
// multiple of 16 / elem, elem the bytes of an orbital value) and 16-byte
// aligned orbitals and potential.
inline bool psi_tma_applies(int nx, const void* psi, const void* V, size_t elem) {
    auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    return elem > 0 && elem <= 16 && nx % (int)(16 / elem) == 0 && al(psi) && al(V);
}
// Flag or-ed into the variant by the cycle-ending step: its overlap feeds the
// Cholesky orthonormalisation, which fixes the orbital norms that density and
// energies see, so it is summed exactly (FP64) even where the per-step
// overlap runs on the tensor cores (more than kMaxOrb FP32 orbitals).
constexpr int kRelaxExactOverlap = 4;

// Variant for a stream-collide launch outside a handle: forced by
// lbks_set_relax_variant, else the tuned choice for the shape, else one site.
int relax_variant_for(int precision, int n_orb, double omega, int nx, int ny, int nz);

// ------------------------------------------------------------------ relax ops
// Implemented per precision (lbks_relax_f64.cu, lbks_relax_f32.cu).
struct RelaxIO {
    const void* f_in;
    const void* u_in;  // may be null
    const double* V;
    const double* sigma_in;
    void* f_out;
    void* psi_out;
    double* S_out;
    double* lambda_out;
    double* sigma_out;
    // orbital storage, up to kMaxOrb orbitals: the W source from Lambda of the
    // step that produced f_in (null: no W source), instead of the field u_in
    const double* lambda_in = nullptr;
};

struct OrbitalStart {  // Gaussian start of one orbital
    double cx, cy, cz, width;
};

// Launchers of one precision; each covers B systems of the grid's shape,
// arrays of consecutive systems at fixed strides (populations NO*19*N,
// orbitals NO*N, W field max(NO-1,1)*N, potentials N, NO x NO matrices,
// NO scales, kMpStride multipoles, kEmatStride energy-matrix entries).
struct PrecisionOps {
    cudaError_t (*relax)(int n_orb, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int B, int variant,
                         cudaStream_t);
    // omega = 1 only: the step in orbital storage (f_in / f_out hold psi in the
    // compute type, V is the potential of the collision that produced f_in)
    cudaError_t (*relax_psi)(int n_orb, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int B,
                             int variant, cudaStream_t);
    cudaError_t (*w_field)(int n_orb, const Grid&, double omega, const void* psi, const double* lam, void* u, int B,
                           cudaStream_t);
    cudaError_t (*orth_apply)(int n_orb, const Grid&, const double* Linv, void* f, void* psi, int B, cudaStream_t);
    cudaError_t (*gram)(int n_orb, const Grid&, double h, const void* psi, double* S, const Scratch&, int B,
                        cudaStream_t);
    // starts: device array [B][n_orb]
    cudaError_t (*init_orbitals)(int n_orb, const Grid&, double h, const OrbitalStart* starts, void* psi, int B,
                                 cudaStream_t);
    cudaError_t (*equilibrium)(int n_orb, const Grid&, const Coef&, const void* psi, void* f, int B, cudaStream_t);
    // rho = 2 sum psi^2 and its multipoles mp[0..9] = {q, p_x, p_y, p_z, Q_xx,
    // Q_yy, Q_zz, Q_xy, Q_xz, Q_yz}; mp[10] = h^3 sum (rho - rho_ref)^2 and
    // mp[11] = h^3 sum rho^2 (the stop rule's density change; rho_ref may alias rho)
    cudaError_t (*density)(int n_orb, const Grid&, double h, const void* psi, double* rho, const double* rho_ref,
                           double* mp, const Scratch&, int B, cudaStream_t);
    // H[j][k] = <psi_j|T_h + V|psi_k>, kin[j] = <psi_j|T_h|psi_j>  (n_orb^2 + n_orb doubles per system)
    cudaError_t (*energy_matrix)(int n_orb, const Grid&, const Coef&, const void* psi, const double* V,
                                 double* out, const Scratch&, int B, cudaStream_t);
    size_t elem;      // bytes of a stored population
    size_t psi_elem;  // bytes of an orbital / W-field value (the compute type)
};
const PrecisionOps& ops_f64();
const PrecisionOps& ops_f32();
const PrecisionOps& ops_bf16();  // bfloat16 populations, float arithmetic and orbitals
// Widens n bfloat16 populations to float (the switch to the FP32 polish phase).
cudaError_t launch_bf16_to_f32(const void* src, void* dst, size_t n, cudaStream_t);

// ----------------------------------------------------------------- field ops
// lbks_fields.cu (always FP64)
constexpr int kMaxAtoms = 256;
// counts[B] atoms per system, atoms[B][kMaxAtoms][4] = (x, y, z, Z)
cudaError_t launch_vext(const Grid&, double h, const int* counts, const double* atoms, double a, double* v, int B,
                        cudaStream_t);
// Electron-nucleus Hellmann-Feynman forces at density rho: out[B][kMaxAtoms][3]
// (rows 0 .. counts[b] - 1 written); max_atoms bounds counts[].
cudaError_t launch_forces(const Grid&, double h, const int* counts, const double* atoms, double a, const double* rho,
                          double* out, int max_atoms, const Scratch& sc, int B, cudaStream_t);
cudaError_t launch_cholesky(int n, const double* S, double* Linv, int* status, const int* active, int B,
                            cudaStream_t);
cudaError_t launch_fill(double* p, size_t n, double value, cudaStream_t);
cudaError_t launch_lda(size_t n, const double* rho, double* eps, double* v, cudaStream_t);
// V_out = V_ext + V_H + v_xc(rho); V_in = first ? V_out : mix V_out + (1 - mix) V_in;
// e4 = h^3 {sum V_ext rho, sum V_H rho, sum rho eps_xc, sum rho}
cudaError_t launch_potential(const Grid&, double h, const double* rho, const double* vext,
                             const double* vh, double* vout, double* vin, int first, double mix,
                             double* e4, const Scratch&, int B, cudaStream_t);

// ------------------------------------------------------ concurrent dynamics
// lbks_cd_f64.cu, lbks_cd_f32.cu (up to kMaxOrb complex orbitals).  A level
// is [system][j][part][z][y][x], part 0 real and 1 imaginary.
struct CdIO {
    const void* prev;    // may be null (alpha = 0)
    const void* extra;   // may be null (beta = 0)
    const void* cur;
    void* out;
    const double* V;      // [system][N]
    const double* lam;    // [system][NO][NO][2] of cur, or null: no W source
    const double* ucoef;  // [system][NO], or null: no U source
    double* S_out;        // [system][NO][NO][2] of out, or null: no overlap
    double* lam_out;      // [system][NO][NO][2] of out (with S_out), may be null
    double alpha, beta, c_re, c_im, h;
};
// Lattice weights per velocity class: xi_p, chi_p and the U source's w_p q_p.
struct CdCoef {
    double dt;  // the ground-state step theta h^2 of the pulled populations
    double xi[3], chi[3], wq[3];
};
// out_j = alpha prev_j + beta extra_j + c D_j(cur) + u_j (K_q cur_j), with the
// overlap (and Lambda) of out when io.S_out is set.
template <typename T>
cudaError_t launch_cd_step(int NO, const Grid&, const CdCoef&, const CdIO&, const Scratch&, int B, cudaStream_t);
// Kernel of the step: -1 the staged one wherever its box leaves two blocks per
// SM (else one site per thread), 0 one site per thread, 1 staged where it applies.
int cd_kernel_mode();
// Overlap S[i][j] = <phi_i|phi_j> and Lambda of one level.
template <typename T>
cudaError_t launch_cd_overlap(int NO, const Grid&, const void* phi, double h, double* S, double* lam,
                              const Scratch&, int B, cudaStream_t);

struct CGState {  // device-resident scalars of the preconditioned CG
    double bb, rr, rz, pap, alpha, beta, relres;
    double rtol;  // the solve's relative residual target (set by the start kernel)
    int iters, done;
};
struct PoissonBufs {
    double *b, *r, *p, *ap, *z, *tmp;  // fine-grid vectors (tmp: spare)
    CGState* cg;
    double* mp;  // multipoles of rho (10 doubles)
    float* r32 = nullptr;  // the residual in single precision: the preconditioner's right-hand side
    float* x32 = nullptr;  // the preconditioner's result (the finest level's x)
};
constexpr int kMaxLevels = 10;
struct MGLevel {  // single-precision arrays of the preconditioner (level 0 included)
    Grid g;
    float *x = nullptr, *b = nullptr, *r = nullptr;
};
struct MGHierarchy {
    int nlev = 0;
    MGLevel lev[kMaxLevels];
};
// lbks_poisson.cu
int mg_levels(int nx, int ny, int nz);
size_t mg_coarse_doubles(int nx, int ny, int nz);  // doubles that hold x, b, r (FP32) of every level, one system
// Carves `coarse` (B * mg_coarse_doubles) into the levels; level arrays hold
// the B systems consecutively.
MGHierarchy make_hierarchy(const Grid& fine, double* coarse, int B);
// Builds the right-hand side (4 pi h^2 rho + ghost values) and r = b - A x.
cudaError_t launch_poisson_start(const Grid&, double h, const double* rho, double* x, double rtol,
                                 const PoissonBufs&, const Scratch&, int B, cudaStream_t);
// `iters` preconditioned CG iterations (no-ops once converged), to the
// tolerance the start kernel recorded (rtol is that of the start).
cudaError_t launch_poisson_iterate(const Grid&, double* x, double rtol, int iters, const PoissonBufs&,
                                   const MGHierarchy&, const Scratch&, int B, cudaStream_t);
cudaError_t launch_multipoles_from_rho(const Grid&, double h, const double* rho, double* mp,
                                       const Scratch&, int B, cudaStream_t);

}  // namespace lbks
