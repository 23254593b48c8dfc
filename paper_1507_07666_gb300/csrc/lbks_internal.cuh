// Internal declarations shared by the translation units of liblbks.
// Not part of the public ABI (see include/lbks.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace lbks {

constexpr int kThreads = 256;  // block size of every grid kernel
constexpr int kMaxOrb = 8;

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

struct Grid {
    int nx, ny, nz;
    uint32_t N;
    FastDiv divx, divy;
};
Grid make_grid(int nx, int ny, int nz);

// Reduction scratch: per-block partial sums and one arrival counter that the
// last block resets.  Kernels sharing a Scratch must be stream-ordered.
struct Scratch {
    double* partial = nullptr;  // max_blocks * max_vals doubles
    unsigned* counter = nullptr;
    int max_blocks = 0;
    int max_vals = 0;
};

// Launch bookkeeping.
void count_launches(uint64_t n);
// Records the calling thread's error message (returned by lbks_last_error); returns code.
int set_last_error(int code, const char* msg);
int num_sms();

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
};

struct OrbitalStart {  // Gaussian start of one orbital
    double cx, cy, cz, width;
};

struct PrecisionOps {
    cudaError_t (*relax)(int n_orb, const Grid&, const Coef&, const RelaxIO&, const Scratch&, cudaStream_t);
    cudaError_t (*w_field)(int n_orb, size_t n_sites, double omega, const void* psi, const double* lam,
                           void* u, cudaStream_t);
    cudaError_t (*orth_apply)(int n_orb, size_t n_sites, const double* Linv, void* f, void* psi,
                              cudaStream_t);
    cudaError_t (*gram)(int n_orb, const Grid&, double h, const void* psi, double* S, const Scratch&,
                        cudaStream_t);
    cudaError_t (*init_orbitals)(int n_orb, const Grid&, double h, const OrbitalStart* starts, void* psi,
                                 cudaStream_t);
    cudaError_t (*equilibrium)(int n_orb, size_t n_sites, const Coef&, const void* psi, void* f,
                               cudaStream_t);
    // rho = 2 sum psi^2 and its multipoles mp[10] = {q, p_x, p_y, p_z, Q_xx, Q_yy, Q_zz, Q_xy, Q_xz, Q_yz}
    cudaError_t (*density)(int n_orb, const Grid&, double h, const void* psi, double* rho, double* mp,
                           const Scratch&, cudaStream_t);
    // H[j][k] = <psi_j|T_h + V|psi_k>, kin[j] = <psi_j|T_h|psi_j>  (out: n_orb^2 + n_orb doubles)
    cudaError_t (*energy_matrix)(int n_orb, const Grid&, const Coef&, const void* psi, const double* V,
                                 double* out, const Scratch&, cudaStream_t);
    size_t elem;
};
const PrecisionOps& ops_f64();
const PrecisionOps& ops_f32();

// ----------------------------------------------------------------- field ops
// lbks_fields.cu (always FP64)
cudaError_t launch_vext(const Grid&, double h, int n_atoms, const double* atoms_dev /*4 per atom*/,
                        double a, double* v, cudaStream_t);
cudaError_t launch_cholesky(int n, const double* S, double* Linv, int* status, cudaStream_t);
cudaError_t launch_fill(double* p, size_t n, double value, cudaStream_t);
cudaError_t launch_lda(size_t n, const double* rho, double* eps, double* v, cudaStream_t);
// V_out = V_ext + V_H + v_xc(rho); V_in = first ? V_out : mix V_out + (1 - mix) V_in;
// e4 = h^3 {sum V_ext rho, sum V_H rho, sum rho eps_xc, sum rho}
cudaError_t launch_potential(const Grid&, double h, const double* rho, const double* vext,
                             const double* vh, double* vout, double* vin, int first, double mix,
                             double* e4, const Scratch&, cudaStream_t);

struct CGState {  // device-resident scalars of the preconditioned CG
    double bb, rr, rz, pap, alpha, beta, relres;
    int iters, done;
};
struct PoissonBufs {
    double *b, *r, *p, *ap, *z, *tmp;  // fine-grid vectors
    CGState* cg;
    double* mp;  // multipoles of rho (10 doubles)
};
constexpr int kMaxLevels = 10;
struct MGLevel {
    Grid g;
    double *x = nullptr, *b = nullptr, *r = nullptr;
};
struct MGHierarchy {
    int nlev = 0;
    MGLevel lev[kMaxLevels];
};
// lbks_poisson.cu
int mg_levels(int nx, int ny, int nz);
size_t mg_coarse_doubles(int nx, int ny, int nz);           // x, b, r of every level below the finest
MGHierarchy make_hierarchy(const Grid& fine, double* coarse);  // carves `coarse` into the levels
// Builds the right-hand side (4 pi h^2 rho + ghost values) and r = b - A x.
cudaError_t launch_poisson_start(const Grid&, double h, const double* rho, double* x, double rtol,
                                 const PoissonBufs&, const Scratch&, cudaStream_t);
// `iters` preconditioned CG iterations (no-ops once converged).
cudaError_t launch_poisson_iterate(const Grid&, double* x, double rtol, int iters, const PoissonBufs&,
                                   const MGHierarchy&, const Scratch&, cudaStream_t);
cudaError_t launch_multipoles_from_rho(const Grid&, double h, const double* rho, double* mp,
                                       const Scratch&, cudaStream_t);

}  // namespace lbks
