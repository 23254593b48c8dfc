// Grid fields of the self-consistent loop, all in FP64: external potential,
// Cholesky of the overlap, LDA exchange-correlation, potential assembly with
// mixing and energy integrals, multipoles of the density (the Hartree solve
// itself is in lbks_poisson.cu).
#include "lbks_internal.cuh"
#include "lbks_reduce.cuh"

#include <algorithm>

namespace lbks {

namespace {

__device__ __forceinline__ void coords(const Grid& g, double h, uint32_t s, int& x, int& y, int& z, double& rx,
                                       double& ry, double& rz) {
    const uint32_t q = g.divx.div(s);
    x = (int)(s - q * (uint32_t)g.nx);
    const uint32_t zz = g.divy.div(q);
    y = (int)(q - zz * (uint32_t)g.ny);
    z = (int)zz;
    rx = (x - 0.5 * (g.nx - 1)) * h;
    ry = (y - 0.5 * (g.ny - 1)) * h;
    rz = (z - 0.5 * (g.nz - 1)) * h;
}

int grid_for(size_t n, int cap_blocks) {
    const size_t need = (n + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)cap_blocks));
}

// Blocks per system of a reduction kernel over B systems.
int red_cap(const Scratch& sc, int vals, int B) {
    if (sc.max_vals < vals || sc.systems < B) return 0;
    return std::max(1, std::min(sc.max_blocks, num_sms() * 4 / std::max(B, 1)));
}

// ------------------------------------------------------------ external potential
// V_ext(r) = -sum_I Z_I / sqrt(|r - R_I|^2 + a^2)   (softened nuclei)
__global__ void __launch_bounds__(kThreads) k_vext(Grid g, double h, const int* __restrict__ counts,
                                                   const double* __restrict__ atoms, double a2, double* __restrict__ v) {
    if (inactive(g)) return;
    const int n_atoms = counts[sys_id()];
    atoms += (size_t)sys_id() * kMaxAtoms * 4;
    v += (size_t)sys_id() * g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        int x, y, z;
        double rx, ry, rz;
        coords(g, h, s, x, y, z, rx, ry, rz);
        double acc = 0.0;
        for (int I = 0; I < n_atoms; ++I) {
            const double dx = rx - atoms[4 * I], dy = ry - atoms[4 * I + 1], dz = rz - atoms[4 * I + 2];
            acc -= atoms[4 * I + 3] / sqrt(dx * dx + dy * dy + dz * dz + a2);
        }
        v[s] = acc;
    }
}

// ------------------------------------------------------- Hellmann-Feynman forces
// Electron-nucleus part of the force on each nucleus at the density rho,
// F_I = Z_I h^3 sum_r rho(r) (r - R_I) / (|r - R_I|^2 + a^2)^(3/2)
// (minus the derivative of h^3 sum rho V_ext with respect to R_I).  Nuclei in
// chunks of kForceChunk, one pass over rho per chunk; per-thread FP64 sums,
// block sums into a flat partial array (row pitch kp = 3 * nuclei rounded up
// to whole chunks), the last block sums the rows in a fixed order and writes
// out[3 I + c] (times h^3).
constexpr int kForceChunk = 8;

__host__ __device__ inline int force_pitch(int n_atoms) {
    return 3 * ((n_atoms + kForceChunk - 1) / kForceChunk) * kForceChunk;
}

__global__ void __launch_bounds__(kThreads) k_forces(Grid g, double h, const int* __restrict__ counts,
                                                     const double* __restrict__ atoms, double a2,
                                                     const double* __restrict__ rho, double* __restrict__ out,
                                                     Scratch sc) {
    if (inactive(g)) return;
    const int na = counts[sys_id()];
    const int kp = force_pitch(na);
    atoms += (size_t)sys_id() * kMaxAtoms * 4;
    rho += (size_t)sys_id() * g.N;
    out += (size_t)sys_id() * 3 * kMaxAtoms;
    double* partial = sys_partial(sc);
    for (int a0 = 0; a0 < na; a0 += kForceChunk) {
        double acc[3 * kForceChunk];
#pragma unroll
        for (int k = 0; k < 3 * kForceChunk; ++k) acc[k] = 0.0;
        for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
            int x, y, z;
            double rx, ry, rz;
            coords(g, h, s, x, y, z, rx, ry, rz);
            const double r = rho[s];
#pragma unroll
            for (int c = 0; c < kForceChunk; ++c) {
                const int I = a0 + c;
                if (I >= na) break;
                const double dx = rx - atoms[4 * I], dy = ry - atoms[4 * I + 1], dz = rz - atoms[4 * I + 2];
                const double d2 = dx * dx + dy * dy + dz * dz + a2;
                const double w = r * atoms[4 * I + 3] / (d2 * sqrt(d2));
                acc[3 * c] += w * dx;
                acc[3 * c + 1] += w * dy;
                acc[3 * c + 2] += w * dz;
            }
        }
        block_sum_store<3 * kForceChunk>(acc, partial + (size_t)blockIdx.x * kp + 3 * a0);
        __syncthreads();  // the block sums' shared rows are reused by the next chunk
    }
    __shared__ double tot[3 * kMaxAtoms];
    if (grid_total_rt(partial, sys_counter(sc), tot, kp)) {
        const double h3 = h * h * h;
        for (int k = threadIdx.x; k < 3 * na; k += blockDim.x) out[k] = h3 * tot[k];
    }
}


// --------------------------------------------------------------------- Cholesky
// S = L L^T (one CTA), then L^{-1} by forward substitution, one column per thread.
__global__ void k_cholesky(int n, const double* __restrict__ S, double* __restrict__ Linv, int* status,
                           const int* active) {
    if (active && !active[blockIdx.y]) return;
    S += (size_t)blockIdx.y * n * n;
    Linv += (size_t)blockIdx.y * n * n;
    status += blockIdx.y;
    __shared__ double L[kMaxOrbWide * kMaxOrbWide];
    __shared__ int bad;
    if (threadIdx.x == 0) {
        bad = 0;
        for (int i = 0; i < n * n; ++i) L[i] = 0.0;
        for (int j = 0; j < n && !bad; ++j) {
            double d = S[j * n + j];
            for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
            if (!(d > 0.0)) {
                bad = j + 1;
                break;
            }
            const double ljj = sqrt(d);
            L[j * n + j] = ljj;
            for (int i = j + 1; i < n; ++i) {
                double t = S[i * n + j];
                for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
                L[i * n + j] = t / ljj;
            }
        }
        *status = bad;
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k < n) {
        for (int i = 0; i < n; ++i) {
            double t;
            if (bad) {
                t = (i == k) ? 1.0 : 0.0;  // identity when S is not positive definite
            } else if (i < k) {
                t = 0.0;
            } else {
                t = (i == k) ? 1.0 : 0.0;
                for (int m = k; m < i; ++m) t -= L[i * n + m] * Linv[m * n + k];
                t /= L[i * n + i];
            }
            Linv[i * n + k] = t;
        }
    }
}

__global__ void k_fill(double* p, size_t n, double value) {
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) p[s] = value;
}

// --------------------------------------------------------------------------- LDA
// Spin-unpolarised Slater exchange + Perdew-Zunger 1981 correlation
// (Phys. Rev. B 23, 5048, Appendix C).  v = d(rho eps)/d rho.
__device__ __forceinline__ void lda_point(double rho, double& eps, double& v) {
    if (!(rho >= 1e-14)) {
        eps = 0.0;
        v = 0.0;
        return;
    }
    const double kPi = 3.141592653589793238462643383279502884;
    const double cx = -0.75 * cbrt(3.0 / kPi);
    const double ex = cx * cbrt(rho);
    const double vx = (4.0 / 3.0) * ex;
    const double rs = cbrt(3.0 / (4.0 * kPi * rho));
    double ec, vc;
    if (rs >= 1.0) {
        const double gam = -0.1423, b1 = 1.0529, b2 = 0.3334;
        const double sr = sqrt(rs);
        const double den = 1.0 + b1 * sr + b2 * rs;
        ec = gam / den;
        vc = ec * (1.0 + (7.0 / 6.0) * b1 * sr + (4.0 / 3.0) * b2 * rs) / den;
    } else {
        const double A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
        const double lr = log(rs);
        ec = A * lr + B + C * rs * lr + D * rs;
        vc = A * lr + (B - A / 3.0) + (2.0 / 3.0) * C * rs * lr + (2.0 * D - C) / 3.0 * rs;
    }
    eps = ex + ec;
    v = vx + vc;
}

__global__ void __launch_bounds__(kThreads) k_lda(size_t n, const double* __restrict__ rho, double* __restrict__ eps,
                                                  double* __restrict__ v) {
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        double e, w;
        lda_point(rho[s], e, w);
        eps[s] = e;
        v[s] = w;
    }
}

// V_out = V_ext + V_H + v_xc; mixing; energy integrals.
__global__ void __launch_bounds__(kThreads) k_potential(Grid g, double h, const double* __restrict__ rho,
                                                        const double* __restrict__ vext,
                                                        const double* __restrict__ vh, double* __restrict__ vout,
                                                        double* __restrict__ vin, int first, double mix, double* e4,
                                                        Scratch sc) {
    if (inactive(g)) return;
    {
        const size_t o = (size_t)sys_id() * g.N;
        rho += o; vext += o; vh += o; vout += o; vin += o;
        e4 += (size_t)sys_id() * kE4Stride;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        const double r = rho[s];
        double e, w;
        lda_point(r, e, w);
        const double vo = vext[s] + vh[s] + w;
        vout[s] = vo;
        vin[s] = first ? vo : mix * vo + (1.0 - mix) * vin[s];
        acc[0] += vext[s] * r;
        acc[1] += vh[s] * r;
        acc[2] += r * e;
        acc[3] += r;
    }
    double* partial = sys_partial(sc);
    block_sum_store<4>(acc, partial + (size_t)blockIdx.x * 4);
    __shared__ double tot[4];
    if (grid_total<4>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        for (int k = 0; k < 4; ++k) e4[k] = h3 * tot[k];
    }
}

// ------------------------------------------------------------------- multipoles
// Multipoles {q, p_x, p_y, p_z, Q_xx, Q_yy, Q_zz, Q_xy, Q_xz, Q_yz} of rho.
__global__ void __launch_bounds__(kThreads) k_multipoles(Grid g, double h, const double* __restrict__ rho, double* mp,
                                                         Scratch sc) {
    if (inactive(g)) return;
    rho += (size_t)sys_id() * g.N;
    mp += (size_t)sys_id() * kMpStride;
    double acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        int x, y, z;
        double rx, ry, rz;
        coords(g, h, s, x, y, z, rx, ry, rz);
        const double r = rho[s];
        acc[0] += r;
        acc[1] += r * rx; acc[2] += r * ry; acc[3] += r * rz;
        acc[4] += r * rx * rx; acc[5] += r * ry * ry; acc[6] += r * rz * rz;
        acc[7] += r * rx * ry; acc[8] += r * rx * rz; acc[9] += r * ry * rz;
    }
    double* partial = sys_partial(sc);
    block_sum_store<10>(acc, partial + (size_t)blockIdx.x * 10);
    __shared__ double tot[10];
    if (grid_total<10>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        const double tr = tot[4] + tot[5] + tot[6];
        mp[0] = h3 * tot[0];
        mp[1] = h3 * tot[1]; mp[2] = h3 * tot[2]; mp[3] = h3 * tot[3];
        mp[4] = h3 * (3.0 * tot[4] - tr); mp[5] = h3 * (3.0 * tot[5] - tr); mp[6] = h3 * (3.0 * tot[6] - tr);
        mp[7] = h3 * 3.0 * tot[7]; mp[8] = h3 * 3.0 * tot[8]; mp[9] = h3 * 3.0 * tot[9];
    }
}

}  // namespace

// ---------------------------------------------------------------------- launchers
cudaError_t launch_forces(const Grid& g, double h, const int* counts, const double* atoms, double a, const double* rho,
                          double* out, int max_atoms, const Scratch& sc, int B, cudaStream_t st) {
    if (max_atoms < 1 || max_atoms > kMaxAtoms || sc.systems < B) return cudaErrorInvalidValue;
    // every block's row of the flat partial array fits the system's scratch region
    const int rows = (int)std::min<size_t>((size_t)sc.max_blocks * sc.max_vals / force_pitch(max_atoms),
                                           (size_t)num_sms() * 2 / std::max(B, 1));
    if (rows < 1) return cudaErrorInvalidValue;
    k_forces<<<dim3(grid_for(g.N, rows), B), kThreads, 0, st>>>(g, h, counts, atoms, a * a, rho, out, sc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_vext(const Grid& g, double h, const int* counts, const double* atoms, double a, double* v, int B,
                        cudaStream_t st) {
    k_vext<<<dim3(grid_for(g.N, std::max(1, num_sms() * 8 / B)), B), kThreads, 0, st>>>(g, h, counts, atoms, a * a, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cholesky(int n, const double* S, double* Linv, int* status, const int* active, int B,
                            cudaStream_t st) {
    if (n < 1 || n > kMaxOrbWide) return cudaErrorInvalidValue;
    k_cholesky<<<dim3(1, B), 64, 0, st>>>(n, S, Linv, status, active);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(double* p, size_t n, double value, cudaStream_t st) {
    k_fill<<<grid_for(n, num_sms() * 8), kThreads, 0, st>>>(p, n, value);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lda(size_t n, const double* rho, double* eps, double* v, cudaStream_t st) {
    k_lda<<<grid_for(n, num_sms() * 8), kThreads, 0, st>>>(n, rho, eps, v);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_potential(const Grid& g, double h, const double* rho, const double* vext, const double* vh,
                             double* vout, double* vin, int first, double mix, double* e4, const Scratch& sc, int B,
                             cudaStream_t st) {
    const int cap = red_cap(sc, 4, B);
    if (cap < 1) return cudaErrorInvalidValue;
    k_potential<<<dim3(grid_for(g.N, cap), B), kThreads, 0, st>>>(g, h, rho, vext, vh, vout, vin, first, mix, e4, sc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_multipoles_from_rho(const Grid& g, double h, const double* rho, double* mp, const Scratch& sc,
                                       int B, cudaStream_t st) {
    const int cap = red_cap(sc, 10, B);
    if (cap < 1) return cudaErrorInvalidValue;
    k_multipoles<<<dim3(grid_for(g.N, cap), B), kThreads, 0, st>>>(g, h, rho, mp, sc);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lbks
