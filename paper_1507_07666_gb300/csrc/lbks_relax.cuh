// Relaxation kernels of the lattice-kinetic Kohn-Sham solver, templated on
// the population element type T (double or float) and the orbital count NO.
// Included by lbks_relax_f64.cu and lbks_relax_f32.cu, each of which
// instantiates one T.
//
// Method (Sec. 3 of Mendoza, Herrmann, Succi):
//   Eq. LBeq / KSLB  f_jp(r + v_p, t+1) = f_jp - omega (f_jp - xi_p psi_j)
//                                        - dt chi_p V psi_j + W_jp
//   W_jp = -omega xi_p sum_{k<j} Lambda_jk psi_k,  Lambda_jk = <psi_j|psi_k>/<psi_k|psi_k>
// The W source is applied one kernel later: the stream-collide kernel writes
// the collision without it (f_out) plus psi and the overlap S; k_w_field
// writes u_j = -omega sum_{k<j} Lambda_jk psi_k; the next stream-collide
// pulls f_out + xi_p u.  The sum is exactly the paper's post-collision state.
#pragma once

#include "lbks_internal.cuh"
#include "lbks_reduce.cuh"

#include <algorithm>

// Minimum resident blocks per SM requested from the register allocator for
// the stream-collide kernel (a tuning knob; 1 lets it use up to 255 registers).
#ifndef LBKS_RELAX_MIN_BLOCKS
#define LBKS_RELAX_MIN_BLOCKS 1
#endif

namespace lbks {

template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// Index of pair (j, i), i <= j, in the packed lower triangle.
__host__ __device__ constexpr int tri(int j, int i) { return j * (j + 1) / 2 + i; }

// Neighbour bookkeeping of one site for pull streaming.
struct Site {
    uint32_t s;
    bool xm, xp, ym, yp, zm, zp;  // a source exists at x-1, x+1, ...
};

__device__ __forceinline__ Site decode(const Grid& g, uint32_t s) {
    Site t;
    t.s = s;
    const uint32_t q = g.divx.div(s);
    const int x = (int)(s - q * (uint32_t)g.nx);
    const uint32_t zz = g.divy.div(q);
    const int y = (int)(q - zz * (uint32_t)g.ny);
    const int z = (int)zz;
    t.xm = x > 0; t.xp = x < g.nx - 1;
    t.ym = y > 0; t.yp = y < g.ny - 1;
    t.zm = z > 0; t.zp = z < g.nz - 1;
    return t;
}

// Does the source site r - v_p exist?
__device__ __forceinline__ bool has_source(const Site& t, int p) {
    const int vx = vel(p, 0), vy = vel(p, 1), vz = vel(p, 2);
    return (vx == 0 || (vx > 0 ? t.xm : t.xp)) && (vy == 0 || (vy > 0 ? t.ym : t.yp)) &&
           (vz == 0 || (vz > 0 ? t.zm : t.zp));
}

// Linear index of r - v_p (valid only when has_source).
__device__ __forceinline__ uint32_t source_index(const Grid& g, uint32_t s, int p) {
    const int off = vel(p, 0) + vel(p, 1) * g.nx + vel(p, 2) * g.nx * g.ny;
    return (uint32_t)((int)s - off);
}

// ---------------------------------------------------------------------------
// Fused pull-stream + normalisation + BGK collision + potential source for
// all NO orbitals of a site; psi epilogue; overlap partials; the last block
// turns S into Lambda and the next step's scale sigma.
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads, LBKS_RELAX_MIN_BLOCKS) k_stream_collide(Grid g, Coef c, RelaxIO io,
                                                                                  Scratch sc) {
    constexpr int NP = NO * (NO + 1) / 2;
    const T* __restrict__ fin = static_cast<const T*>(io.f_in);
    const T* __restrict__ uin = static_cast<const T*>(io.u_in);
    T* __restrict__ fout = static_cast<T*>(io.f_out);
    T* __restrict__ psio = static_cast<T*>(io.psi_out);
    const uint32_t N = g.N;

    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[j];
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};

    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        const T vr = (T)__ldg(io.V + s);
        T psi[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const T* fj = fin + (size_t)j * 19 * N;
            T gp[19];
#pragma unroll
            for (int p = 0; p < 19; ++p)
                gp[p] = has_source(t, p) ? ld_ro(fj + (size_t)p * N + source_index(g, s, p)) : T(0);
            if (j > 0 && uin != nullptr) {
                const T* uj = uin + (size_t)(j - 1) * N;
#pragma unroll
                for (int p = 0; p < 19; ++p)
                    if (has_source(t, p)) gp[p] += xi[vclass(p)] * ld_ro(uj + source_index(g, s, p));
            }
            T ps = T(0);
#pragma unroll
            for (int p = 0; p < 19; ++p) ps += gp[p];
            ps *= sig[j];
            const T A = om * ps, B = dt * vr * ps;
            const T e[3] = {xi[0] * A - chi[0] * B, xi[1] * A - chi[1] * B, xi[2] * A - chi[2] * B};
            const T c1 = om1 * sig[j];
            T* oj = fout + (size_t)j * 19 * N;
#pragma unroll
            for (int p = 0; p < 19; ++p) st_stream(oj + (size_t)p * N + s, c1 * gp[p] + e[vclass(p)]);
            psio[(size_t)j * N + s] = ps;
            psi[j] = ps;
        }
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) acc[tri(j, i)] += psi[j] * psi[i];
    }

    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    block_sum_store<NP>(v, sc.partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(sc.partial, sc.counter, tot) && threadIdx.x == 0) {
        const double h3 = c.h * c.h * c.h;
        for (int j = 0; j < NO; ++j)
            for (int i = 0; i <= j; ++i) {
                const double sji = h3 * tot[tri(j, i)];
                io.S_out[j * NO + i] = sji;
                io.S_out[i * NO + j] = sji;
            }
        for (int j = 0; j < NO; ++j) {
            for (int k = 0; k < NO; ++k)
                io.lambda_out[j * NO + k] = (k < j) ? io.S_out[j * NO + k] / io.S_out[k * NO + k] : 0.0;
            io.sigma_out[j] = 1.0 / sqrt(io.S_out[j * NO + j]);
        }
    }
}

// u_(j-1)(r) = -omega sum_{k<j} Lambda_jk psi_k(r)
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_w_field(size_t n, double omega, const T* __restrict__ psi,
                                                      const double* __restrict__ lam, T* __restrict__ u) {
    T l[NO][NO];
#pragma unroll
    for (int j = 0; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < NO; ++k) l[j][k] = (T)(-omega * lam[j * NO + k]);
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        T ps[NO];
#pragma unroll
        for (int k = 0; k < NO - 1; ++k) ps[k] = ld_ro(psi + k * n + s);
#pragma unroll
        for (int j = 1; j < NO; ++j) {
            T w = T(0);
#pragma unroll
            for (int k = 0; k < j; ++k) w += l[j][k] * ps[k];
            u[(j - 1) * n + s] = w;
        }
    }
}

// f_jp <- sum_k Linv_jk f_kp, psi_j <- sum_k Linv_jk psi_k, in place per site.
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_orth_apply(size_t n, const double* __restrict__ Linv,
                                                         T* __restrict__ f, T* __restrict__ psi) {
    T L[NO][NO];
#pragma unroll
    for (int j = 0; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < NO; ++k) L[j][k] = (T)Linv[j * NO + k];
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        if (f != nullptr) {
#pragma unroll 1
            for (int p = 0; p < 19; ++p) {
                T a[NO];
#pragma unroll
                for (int k = 0; k < NO; ++k) a[k] = f[((size_t)k * 19 + p) * n + s];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    T o = T(0);
#pragma unroll
                    for (int k = 0; k <= j; ++k) o += L[j][k] * a[k];
                    f[((size_t)j * 19 + p) * n + s] = o;
                }
            }
        }
        if (psi != nullptr) {
            T a[NO];
#pragma unroll
            for (int k = 0; k < NO; ++k) a[k] = psi[(size_t)k * n + s];
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                T o = T(0);
#pragma unroll
                for (int k = 0; k <= j; ++k) o += L[j][k] * a[k];
                psi[(size_t)j * n + s] = o;
            }
        }
    }
}

// S = h^3 psi psi^T
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_gram(Grid g, double h, const T* __restrict__ psi, double* S,
                                                   Scratch sc) {
    constexpr int NP = NO * (NO + 1) / 2;
    double acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.0;
    const uint32_t N = g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        double a[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) a[j] = (double)psi[(size_t)j * N + s];
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) acc[tri(j, i)] += a[j] * a[i];
    }
    block_sum_store<NP>(acc, sc.partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(sc.partial, sc.counter, tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        for (int j = 0; j < NO; ++j)
            for (int i = 0; i <= j; ++i) {
                S[j * NO + i] = h3 * tot[tri(j, i)];
                S[i * NO + j] = h3 * tot[tri(j, i)];
            }
    }
}

struct StartsArg {
    OrbitalStart o[kMaxOrb];
};

// psi0_j(r) = exp(-|r - c_j|^2 / (2 w_j^2))
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_init_orbitals(Grid g, double h, StartsArg st, T* __restrict__ psi) {
    const uint32_t N = g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const uint32_t q = g.divx.div(s);
        const int x = (int)(s - q * (uint32_t)g.nx);
        const uint32_t z = g.divy.div(q);
        const int y = (int)(q - z * (uint32_t)g.ny);
        const double rx = (x - 0.5 * (g.nx - 1)) * h, ry = (y - 0.5 * (g.ny - 1)) * h,
                     rz = ((int)z - 0.5 * (g.nz - 1)) * h;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const double dx = rx - st.o[j].cx, dy = ry - st.o[j].cy, dz = rz - st.o[j].cz;
            const double w = st.o[j].width;
            psi[(size_t)j * N + s] = (T)exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * w * w));
        }
    }
}

// f_jp = xi_p psi_j
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_equilibrium(size_t n, Coef c, const T* __restrict__ psi,
                                                          T* __restrict__ f) {
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const T a = psi[(size_t)j * n + s];
#pragma unroll
            for (int p = 0; p < 19; ++p) f[((size_t)j * 19 + p) * n + s] = xi[vclass(p)] * a;
        }
    }
}

// rho = 2 sum_j psi_j^2 and its moments about the box centre.
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_density(Grid g, double h, const T* __restrict__ psi,
                                                      double* __restrict__ rho, double* mp, Scratch sc) {
    double acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.0;
    const uint32_t N = g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const double a = (double)psi[(size_t)j * N + s];
            r += a * a;
        }
        r *= 2.0;
        rho[s] = r;
        const uint32_t q = g.divx.div(s);
        const int x = (int)(s - q * (uint32_t)g.nx);
        const uint32_t z = g.divy.div(q);
        const int y = (int)(q - z * (uint32_t)g.ny);
        const double rx = (x - 0.5 * (g.nx - 1)) * h, ry = (y - 0.5 * (g.ny - 1)) * h,
                     rz = ((int)z - 0.5 * (g.nz - 1)) * h;
        acc[0] += r;
        acc[1] += r * rx; acc[2] += r * ry; acc[3] += r * rz;
        acc[4] += r * rx * rx; acc[5] += r * ry * ry; acc[6] += r * rz * rz;
        acc[7] += r * rx * ry; acc[8] += r * rx * rz; acc[9] += r * ry * rz;
    }
    block_sum_store<10>(acc, sc.partial + (size_t)blockIdx.x * 10);
    __shared__ double tot[10];
    if (grid_total<10>(sc.partial, sc.counter, tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        const double tr = tot[4] + tot[5] + tot[6];
        mp[0] = h3 * tot[0];
        mp[1] = h3 * tot[1]; mp[2] = h3 * tot[2]; mp[3] = h3 * tot[3];
        mp[4] = h3 * (3.0 * tot[4] - tr); mp[5] = h3 * (3.0 * tot[5] - tr); mp[6] = h3 * (3.0 * tot[6] - tr);
        mp[7] = h3 * 3.0 * tot[7]; mp[8] = h3 * 3.0 * tot[8]; mp[9] = h3 * 3.0 * tot[9];
    }
}

// H_jk = h^3 sum psi_j (T_h + V) psi_k, kin_j = h^3 sum psi_j T_h psi_j,
// T_h = (1 - K_xi) / (theta h^2), K_xi psi(r) = sum_p xi_p psi(r - v_p).
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_energy_matrix(Grid g, Coef c, const T* __restrict__ psi,
                                                            const double* __restrict__ V, double* out,
                                                            Scratch sc) {
    constexpr int K = NO * NO + NO;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const uint32_t N = g.N;
    const double inv = 1.0 / (c.theta * c.h * c.h);
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        const double vr = V[s];
        double a[NO], hp[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const T* pj = psi + (size_t)j * N;
            double kx = 0.0;
#pragma unroll
            for (int p = 0; p < 19; ++p)
                if (has_source(t, p)) kx += c.xi[vclass(p)] * (double)pj[source_index(g, s, p)];
            a[j] = (double)pj[s];
            const double tp = (a[j] - kx) * inv;
            acc[NO * NO + j] += a[j] * tp;
            hp[j] = tp + vr * a[j];
        }
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int k = 0; k < NO; ++k) acc[j * NO + k] += a[j] * hp[k];
    }
    block_sum_store<K>(acc, sc.partial + (size_t)blockIdx.x * K);
    __shared__ double tot[K];
    if (grid_total<K>(sc.partial, sc.counter, tot) && threadIdx.x == 0) {
        const double h3 = c.h * c.h * c.h;
        for (int k = 0; k < K; ++k) out[k] = h3 * tot[k];
    }
}

// ----------------------------------------------------------------- launchers
template <typename Kern>
int blocks_per_sm(Kern kern) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

inline int elementwise_grid(size_t n) {
    const size_t need = (n + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)num_sms() * 8));
}

template <typename Kern>
int reduction_grid(Kern kern, size_t n, const Scratch& sc, int vals) {
    static_assert(sizeof(Kern) > 0, "");
    int cap = blocks_per_sm(kern) * num_sms();
    const int by_scratch = sc.max_vals >= vals ? sc.max_blocks : 0;
    cap = std::min(cap, by_scratch);
    const size_t need = (n + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)cap));
}

template <typename T>
struct Ops {
    template <int NO>
    static cudaError_t relax_n(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, cudaStream_t st) {
        auto kern = k_stream_collide<T, NO>;
        static const int nb = blocks_per_sm(kern);
        const int cap = std::min(nb * num_sms(), sc.max_blocks);
        const size_t need = (g.N + kThreads - 1) / kThreads;
        const int grid = (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)cap));
        if (sc.max_vals < NO * (NO + 1) / 2 || grid < 1) return cudaErrorInvalidValue;
        kern<<<grid, kThreads, 0, st>>>(g, c, io, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t wfield_n(size_t n, double omega, const void* psi, const double* lam, void* u, cudaStream_t st) {
        if (NO < 2) return cudaSuccess;
        k_w_field<T, NO><<<elementwise_grid(n), kThreads, 0, st>>>(n, omega, (const T*)psi, lam, (T*)u);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t orth_n(size_t n, const double* Linv, void* f, void* psi, cudaStream_t st) {
        k_orth_apply<T, NO><<<elementwise_grid(n), kThreads, 0, st>>>(n, Linv, (T*)f, (T*)psi);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t gram_n(const Grid& g, double h, const void* psi, double* S, const Scratch& sc, cudaStream_t st) {
        auto kern = k_gram<T, NO>;
        const int grid = reduction_grid(kern, g.N, sc, NO * (NO + 1) / 2);
        kern<<<grid, kThreads, 0, st>>>(g, h, (const T*)psi, S, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t init_n(const Grid& g, double h, const OrbitalStart* starts, void* psi, cudaStream_t st) {
        StartsArg a;
        for (int j = 0; j < NO; ++j) a.o[j] = starts[j];
        k_init_orbitals<T, NO><<<elementwise_grid(g.N), kThreads, 0, st>>>(g, h, a, (T*)psi);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t eq_n(size_t n, const Coef& c, const void* psi, void* f, cudaStream_t st) {
        k_equilibrium<T, NO><<<elementwise_grid(n), kThreads, 0, st>>>(n, c, (const T*)psi, (T*)f);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t density_n(const Grid& g, double h, const void* psi, double* rho, double* mp,
                                 const Scratch& sc, cudaStream_t st) {
        auto kern = k_density<T, NO>;
        const int grid = reduction_grid(kern, g.N, sc, 10);
        kern<<<grid, kThreads, 0, st>>>(g, h, (const T*)psi, rho, mp, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t energy_n(const Grid& g, const Coef& c, const void* psi, const double* V, double* out,
                                const Scratch& sc, cudaStream_t st) {
        auto kern = k_energy_matrix<T, NO>;
        const int grid = reduction_grid(kern, g.N, sc, NO * NO + NO);
        kern<<<grid, kThreads, 0, st>>>(g, c, (const T*)psi, V, out, sc);
        count_launches(1);
        return cudaGetLastError();
    }

    static cudaError_t relax(int n_orb, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc,
                             cudaStream_t st) {
        switch (n_orb) {
            case 1: return relax_n<1>(g, c, io, sc, st);
            case 2: return relax_n<2>(g, c, io, sc, st);
            case 3: return relax_n<3>(g, c, io, sc, st);
            case 4: return relax_n<4>(g, c, io, sc, st);
            case 5: return relax_n<5>(g, c, io, sc, st);
            case 6: return relax_n<6>(g, c, io, sc, st);
            case 7: return relax_n<7>(g, c, io, sc, st);
            case 8: return relax_n<8>(g, c, io, sc, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t w_field(int n_orb, size_t n, double omega, const void* psi, const double* lam, void* u,
                               cudaStream_t st) {
        switch (n_orb) {
            case 1: return cudaSuccess;
            case 2: return wfield_n<2>(n, omega, psi, lam, u, st);
            case 3: return wfield_n<3>(n, omega, psi, lam, u, st);
            case 4: return wfield_n<4>(n, omega, psi, lam, u, st);
            case 5: return wfield_n<5>(n, omega, psi, lam, u, st);
            case 6: return wfield_n<6>(n, omega, psi, lam, u, st);
            case 7: return wfield_n<7>(n, omega, psi, lam, u, st);
            case 8: return wfield_n<8>(n, omega, psi, lam, u, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t orth_apply(int n_orb, size_t n, const double* Linv, void* f, void* psi, cudaStream_t st) {
        switch (n_orb) {
            case 1: return orth_n<1>(n, Linv, f, psi, st);
            case 2: return orth_n<2>(n, Linv, f, psi, st);
            case 3: return orth_n<3>(n, Linv, f, psi, st);
            case 4: return orth_n<4>(n, Linv, f, psi, st);
            case 5: return orth_n<5>(n, Linv, f, psi, st);
            case 6: return orth_n<6>(n, Linv, f, psi, st);
            case 7: return orth_n<7>(n, Linv, f, psi, st);
            case 8: return orth_n<8>(n, Linv, f, psi, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t gram(int n_orb, const Grid& g, double h, const void* psi, double* S, const Scratch& sc,
                            cudaStream_t st) {
        switch (n_orb) {
            case 1: return gram_n<1>(g, h, psi, S, sc, st);
            case 2: return gram_n<2>(g, h, psi, S, sc, st);
            case 3: return gram_n<3>(g, h, psi, S, sc, st);
            case 4: return gram_n<4>(g, h, psi, S, sc, st);
            case 5: return gram_n<5>(g, h, psi, S, sc, st);
            case 6: return gram_n<6>(g, h, psi, S, sc, st);
            case 7: return gram_n<7>(g, h, psi, S, sc, st);
            case 8: return gram_n<8>(g, h, psi, S, sc, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t init_orbitals(int n_orb, const Grid& g, double h, const OrbitalStart* o, void* psi,
                                     cudaStream_t st) {
        switch (n_orb) {
            case 1: return init_n<1>(g, h, o, psi, st);
            case 2: return init_n<2>(g, h, o, psi, st);
            case 3: return init_n<3>(g, h, o, psi, st);
            case 4: return init_n<4>(g, h, o, psi, st);
            case 5: return init_n<5>(g, h, o, psi, st);
            case 6: return init_n<6>(g, h, o, psi, st);
            case 7: return init_n<7>(g, h, o, psi, st);
            case 8: return init_n<8>(g, h, o, psi, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t equilibrium(int n_orb, size_t n, const Coef& c, const void* psi, void* f, cudaStream_t st) {
        switch (n_orb) {
            case 1: return eq_n<1>(n, c, psi, f, st);
            case 2: return eq_n<2>(n, c, psi, f, st);
            case 3: return eq_n<3>(n, c, psi, f, st);
            case 4: return eq_n<4>(n, c, psi, f, st);
            case 5: return eq_n<5>(n, c, psi, f, st);
            case 6: return eq_n<6>(n, c, psi, f, st);
            case 7: return eq_n<7>(n, c, psi, f, st);
            case 8: return eq_n<8>(n, c, psi, f, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t density(int n_orb, const Grid& g, double h, const void* psi, double* rho, double* mp,
                               const Scratch& sc, cudaStream_t st) {
        switch (n_orb) {
            case 1: return density_n<1>(g, h, psi, rho, mp, sc, st);
            case 2: return density_n<2>(g, h, psi, rho, mp, sc, st);
            case 3: return density_n<3>(g, h, psi, rho, mp, sc, st);
            case 4: return density_n<4>(g, h, psi, rho, mp, sc, st);
            case 5: return density_n<5>(g, h, psi, rho, mp, sc, st);
            case 6: return density_n<6>(g, h, psi, rho, mp, sc, st);
            case 7: return density_n<7>(g, h, psi, rho, mp, sc, st);
            case 8: return density_n<8>(g, h, psi, rho, mp, sc, st);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t energy_matrix(int n_orb, const Grid& g, const Coef& c, const void* psi, const double* V,
                                     double* out, const Scratch& sc, cudaStream_t st) {
        switch (n_orb) {
            case 1: return energy_n<1>(g, c, psi, V, out, sc, st);
            case 2: return energy_n<2>(g, c, psi, V, out, sc, st);
            case 3: return energy_n<3>(g, c, psi, V, out, sc, st);
            case 4: return energy_n<4>(g, c, psi, V, out, sc, st);
            case 5: return energy_n<5>(g, c, psi, V, out, sc, st);
            case 6: return energy_n<6>(g, c, psi, V, out, sc, st);
            case 7: return energy_n<7>(g, c, psi, V, out, sc, st);
            case 8: return energy_n<8>(g, c, psi, V, out, sc, st);
            default: return cudaErrorInvalidValue;
        }
    }

    static const PrecisionOps& table() {
        static const PrecisionOps t = {&relax, &w_field, &orth_apply, &gram, &init_orbitals,
                                       &equilibrium, &density, &energy_matrix, sizeof(T)};
        return t;
    }
};

}  // namespace lbks
