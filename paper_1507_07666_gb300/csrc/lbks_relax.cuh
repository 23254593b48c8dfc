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

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

// Resident 256-thread blocks per SM that the register allocator must leave
// room for in the stream-collide kernel (tuning knobs, set by measurement):
// the general FP64 collision keeps 19 doubles per thread and gets fewer; the
// batched build (per-system bases in registers) and more than five orbitals
// get one more than that.
#ifndef LBKS_RELAX_MIN_BLOCKS
#define LBKS_RELAX_MIN_BLOCKS 4
#endif
#ifndef LBKS_RELAX_MIN_BLOCKS_WIDE
#define LBKS_RELAX_MIN_BLOCKS_WIDE 2
#endif

namespace lbks {

template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) { return __ldg(p); }

template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// Populations are stored as TS and computed in T (TS = T, or bfloat16
// storage with float arithmetic).
template <typename T, typename TS>
__device__ __forceinline__ T to_compute(TS v) { return (T)v; }
template <>
__device__ __forceinline__ float to_compute<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename TS, typename T>
__device__ __forceinline__ TS to_store(T v) { return (TS)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }


// Neighbour bookkeeping of one site for pull streaming.
struct Site {
    uint32_t s;
    int x;
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
    t.x = x;
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
// turns S into Lambda and the next step's scale sigma.  One thread per site,
// orbitals in sequence (the W source of orbital j reaches it through u_j, so
// the orbitals of a site share nothing but the overlap products).
// OM1: omega = 1, where the collision forgets the arriving populations and
// only their sum psi enters (no (1 - omega) f term).
// PF: the populations of orbital j + 1 are loaded before orbital j is
// collided (twice the loads in flight per thread, one block fewer per SM).
template <typename T, int NO, bool OM1, bool BATCHED, bool PF = false>
constexpr int relax_min_blocks() {
    return PF                       ? LBKS_RELAX_MIN_BLOCKS_WIDE + (sizeof(T) == 8 ? 0 : 1)
           : (sizeof(T) == 8 && !OM1) ? LBKS_RELAX_MIN_BLOCKS_WIDE
           : (BATCHED || NO > 5)    ? LBKS_RELAX_MIN_BLOCKS_WIDE + 1
                                    : LBKS_RELAX_MIN_BLOCKS;
}

template <typename TS>
__device__ __forceinline__ TS zero_store() { return TS(0); }
template <>
__device__ __forceinline__ __nv_bfloat16 zero_store<__nv_bfloat16>() { return __float2bfloat16_rn(0.f); }

// BATCHED: the launch covers several systems (system = blockIdx.y); the
// single-system build keeps its array bases in the parameter bank instead of
// registers, which the register-bound kernel needs.
template <typename TS, typename T, int NO, bool OM1, bool BATCHED, bool PF>
__global__ void __launch_bounds__(kThreads, (relax_min_blocks<T, NO, OM1, BATCHED, PF>()))
    k_stream_collide(Grid g, Coef c, RelaxIO io, Scratch sc) {
    constexpr int NP = NO * (NO + 1) / 2;
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = BATCHED ? sys_id() : 0;
    // per-system bases are formed where they are used, from the parameter
    // bank and y, so that they need not stay live in registers
    const TS* __restrict__ fin = static_cast<const TS*>(io.f_in);
    const T* __restrict__ uin = static_cast<const T*>(io.u_in);
    TS* __restrict__ fout = static_cast<TS*>(io.f_out);
    T* __restrict__ psio = static_cast<T*>(io.psi_out);

    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};

    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        const T vr = (T)__ldg(io.V + y * N + s);
        T psi[NO];
        TS raw[19];  // PF: the next orbital's populations, in flight
        if (PF) {
#pragma unroll
            for (int p = 0; p < 19; ++p)
                raw[p] = has_source(t, p) ? ld_ro(fin + y * NO * 19 * N + (size_t)p * N + source_index(g, s, p))
                                          : zero_store<TS>();
        }
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const TS* fj = fin + (y * NO + j) * 19 * N;
            const T* uj = (j > 0 && uin != nullptr) ? uin + (y * (NO > 1 ? NO - 1 : 1) + j - 1) * N : nullptr;
            TS* oj = fout + (y * NO + j) * 19 * N;
            // all 19 loads are issued before any use (memory-level parallelism)
            T gp[19];
            if (PF) {
#pragma unroll
                for (int p = 0; p < 19; ++p) gp[p] = to_compute<T>(raw[p]);
                if (j + 1 < NO) {
#pragma unroll
                    for (int p = 0; p < 19; ++p)
                        raw[p] = has_source(t, p) ? ld_ro(fj + 19 * (size_t)N + (size_t)p * N + source_index(g, s, p))
                                                  : zero_store<TS>();
                }
            } else {
#pragma unroll
                for (int p = 0; p < 19; ++p)
                    gp[p] = has_source(t, p) ? to_compute<T>(ld_ro(fj + (size_t)p * N + source_index(g, s, p))) : T(0);
            }
            if (uj) {
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
#pragma unroll
            for (int p = 0; p < 19; ++p)
                st_stream(oj + (size_t)p * N + s, to_store<TS>(OM1 ? e[vclass(p)] : c1 * gp[p] + e[vclass(p)]));
            psio[(y * NO + j) * N + s] = ps;
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
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0) {
        double* S_out = io.S_out + y * NO * NO;
        double* lambda_out = io.lambda_out + y * NO * NO;
        double* sigma_out = io.sigma_out + y * NO;
        const double h3 = c.h * c.h * c.h;
        for (int j = 0; j < NO; ++j)
            for (int i = 0; i <= j; ++i) {
                const double sji = h3 * tot[tri(j, i)];
                S_out[j * NO + i] = sji;
                S_out[i * NO + j] = sji;
            }
        for (int j = 0; j < NO; ++j) {
            for (int k = 0; k < NO; ++k)
                lambda_out[j * NO + k] = (k < j) ? S_out[j * NO + k] / S_out[k * NO + k] : 0.0;
            sigma_out[j] = 1.0 / sqrt(S_out[j * NO + j]);
        }
    }
}

// u_(j-1)(r) = -omega sum_{k<j} Lambda_jk psi_k(r)
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_w_field(const Grid g, double omega, const T* __restrict__ psi,
                                                      const double* __restrict__ lam, T* __restrict__ u) {
    if (inactive(g)) return;
    const size_t n = g.N, y = sys_id();
    psi += y * NO * n;
    lam += y * NO * NO;
    u += y * (NO - 1) * n;
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

// The same for FP32, four consecutive sites per thread with 16-byte loads and
// stores (n a multiple of 4, 16-byte aligned arrays): four times the bytes in
// flight per load instruction.
template <int NO>
__global__ void __launch_bounds__(kThreads) k_w_field4(const Grid g, double omega, const float* __restrict__ psi,
                                                       const double* __restrict__ lam, float* __restrict__ u) {
    if (inactive(g)) return;
    const size_t n = g.N, y = sys_id(), n4 = n / 4;
    const float4* __restrict__ p4 = reinterpret_cast<const float4*>(psi + y * NO * n);
    float4* __restrict__ u4 = reinterpret_cast<float4*>(u + y * (NO - 1) * n);
    lam += y * NO * NO;
    float l[NO][NO];
#pragma unroll
    for (int j = 0; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < NO; ++k) l[j][k] = (float)(-omega * lam[j * NO + k]);
    for (size_t q = blockIdx.x * (size_t)kThreads + threadIdx.x; q < n4; q += (size_t)gridDim.x * kThreads) {
        float4 ps[NO];
#pragma unroll
        for (int k = 0; k < NO - 1; ++k) ps[k] = __ldg(p4 + k * n4 + q);
#pragma unroll
        for (int j = 1; j < NO; ++j) {
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < j; ++k) {
                w.x += l[j][k] * ps[k].x;
                w.y += l[j][k] * ps[k].y;
                w.z += l[j][k] * ps[k].z;
                w.w += l[j][k] * ps[k].w;
            }
            u4[(j - 1) * n4 + q] = w;
        }
    }
}

// f_jp <- sum_k Linv_jk f_kp, psi_j <- sum_k Linv_jk psi_k, in place per site.
template <typename TS, typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_orth_apply(const Grid g, const double* __restrict__ Linv,
                                                         TS* __restrict__ f, T* __restrict__ psi) {
    if (inactive(g)) return;
    const size_t n = g.N, y = sys_id();
    Linv += y * NO * NO;
    if (f) f += y * NO * 19 * n;
    if (psi) psi += y * NO * n;
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
                for (int k = 0; k < NO; ++k) a[k] = to_compute<T>(f[((size_t)k * 19 + p) * n + s]);
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    T o = T(0);
#pragma unroll
                    for (int k = 0; k <= j; ++k) o += L[j][k] * a[k];
                    f[((size_t)j * 19 + p) * n + s] = to_store<TS>(o);
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
    if (inactive(g)) return;
    psi += (size_t)sys_id() * NO * g.N;
    S += (size_t)sys_id() * NO * NO;
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
    double* partial = sys_partial(sc);
    block_sum_store<NP>(acc, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        for (int j = 0; j < NO; ++j)
            for (int i = 0; i <= j; ++i) {
                S[j * NO + i] = h3 * tot[tri(j, i)];
                S[i * NO + j] = h3 * tot[tri(j, i)];
            }
    }
}

// psi0_j(r) = exp(-|r - c_j|^2 / (2 w_j^2)); starts[system][j]
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_init_orbitals(Grid g, double h, const OrbitalStart* __restrict__ starts,
                                                            T* __restrict__ psi) {
    if (inactive(g)) return;
    const uint32_t N = g.N;
    const OrbitalStart* st = starts + (size_t)sys_id() * NO;
    psi += (size_t)sys_id() * NO * N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const uint32_t q = g.divx.div(s);
        const int x = (int)(s - q * (uint32_t)g.nx);
        const uint32_t z = g.divy.div(q);
        const int y = (int)(q - z * (uint32_t)g.ny);
        const double rx = (x - 0.5 * (g.nx - 1)) * h, ry = (y - 0.5 * (g.ny - 1)) * h,
                     rz = ((int)z - 0.5 * (g.nz - 1)) * h;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const double dx = rx - st[j].cx, dy = ry - st[j].cy, dz = rz - st[j].cz;
            const double w = st[j].width;
            psi[(size_t)j * N + s] = (T)exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * w * w));
        }
    }
}

// f_jp = xi_p psi_j
template <typename TS, typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_equilibrium(const Grid g, Coef c, const T* __restrict__ psi,
                                                          TS* __restrict__ f) {
    if (inactive(g)) return;
    const size_t n = g.N;
    psi += (size_t)sys_id() * NO * n;
    f += (size_t)sys_id() * NO * 19 * n;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const T a = psi[(size_t)j * n + s];
#pragma unroll
            for (int p = 0; p < 19; ++p) f[((size_t)j * 19 + p) * n + s] = to_store<TS>(xi[vclass(p)] * a);
        }
    }
}

// rho = 2 sum_j psi_j^2 and its moments about the box centre; mp[10], mp[11] =
// h^3 sum (rho - rho_ref)^2, h^3 sum rho^2 (rho_ref may alias rho: each
// site reads its reference before writing).
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_density(Grid g, double h, const T* __restrict__ psi,
                                                      double* __restrict__ rho, const double* rho_ref, double* mp,
                                                      Scratch sc) {
    if (inactive(g)) return;
    psi += (size_t)sys_id() * NO * g.N;
    rho += (size_t)sys_id() * g.N;
    rho_ref += (size_t)sys_id() * g.N;
    mp += (size_t)sys_id() * kMpStride;
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    const uint32_t N = g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        double r = 0.0;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const double a = (double)psi[(size_t)j * N + s];
            r += a * a;
        }
        r *= 2.0;
        const double dr = r - rho_ref[s];  // change from the reference density (stop rule)
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
        acc[10] += dr * dr; acc[11] += r * r;
    }
    double* partial = sys_partial(sc);
    block_sum_store<12>(acc, partial + (size_t)blockIdx.x * 12);
    __shared__ double tot[12];
    if (grid_total<12>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        const double h3 = h * h * h;
        const double tr = tot[4] + tot[5] + tot[6];
        mp[0] = h3 * tot[0];
        mp[1] = h3 * tot[1]; mp[2] = h3 * tot[2]; mp[3] = h3 * tot[3];
        mp[4] = h3 * (3.0 * tot[4] - tr); mp[5] = h3 * (3.0 * tot[5] - tr); mp[6] = h3 * (3.0 * tot[6] - tr);
        mp[7] = h3 * 3.0 * tot[7]; mp[8] = h3 * 3.0 * tot[8]; mp[9] = h3 * 3.0 * tot[9];
        mp[10] = h3 * tot[10]; mp[11] = h3 * tot[11];
    }
}

// H_jk = h^3 sum psi_j (T_h + V) psi_k, kin_j = h^3 sum psi_j T_h psi_j,
// T_h = (1 - K_xi) / (theta h^2), K_xi psi(r) = sum_p xi_p psi(r - v_p).
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_energy_matrix(Grid g, Coef c, const T* __restrict__ psi,
                                                            const double* __restrict__ V, double* out,
                                                            Scratch sc) {
    constexpr int K = NO * NO + NO;
    if (inactive(g)) return;
    psi += (size_t)sys_id() * NO * g.N;
    V += (size_t)sys_id() * g.N;
    out += (size_t)sys_id() * kEmatStride;
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const uint32_t N = g.N;
    const double inv = 1.0 / (c.theta * c.h * c.h);
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        const double vr = V[s];
        if constexpr (sizeof(T) == 4) {
            // FP32 orbitals: (1 - K_xi) psi = sum_p xi_p (psi(r) - psi(r - v_p)) (sum_p xi_p = 1).
            // A neighbour outside the box is psi = 0, so its term is xi_p psi(r).  A difference
            // is exact in FP32 when the two values are within a factor of two of each other
            // (Sterbenz's lemma), else it carries one rounding of the larger value (near nodes
            // and sign changes).  The weighted sums and products in FP32, the sums over sites
            // in FP64.
            float af[NO], hf[NO];
            const float xf[3] = {(float)c.xi[0], (float)c.xi[1], (float)c.xi[2]};
            const float invf = (float)inv, vf = (float)vr;
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const T* pj = psi + (size_t)j * N;
                const float aj = (float)pj[s];
                float d = 0.f;
#pragma unroll
                for (int p = 1; p < 19; ++p)
                    d += xf[vclass(p)] * (has_source(t, p) ? aj - (float)pj[source_index(g, s, p)] : aj);
                const float tp = d * invf;
                af[j] = aj;
                hf[j] = tp + vf * aj;
                acc[NO * NO + j] += (double)(aj * tp);
            }
#pragma unroll
            for (int j = 0; j < NO; ++j)
#pragma unroll
                for (int k = 0; k < NO; ++k) acc[j * NO + k] += (double)(af[j] * hf[k]);
        } else {
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
    }
    double* partial = sys_partial(sc);
    block_sum_store<K>(acc, partial + (size_t)blockIdx.x * K);
    __shared__ double tot[K];
    if (grid_total<K>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        const double h3 = c.h * c.h * c.h;
        for (int k = 0; k < K; ++k) out[k] = h3 * tot[k];
    }
}

}  // namespace lbks

#include "lbks_wide.cuh"
#include "lbks_pair.cuh"

namespace lbks {

// ----------------------------------------------------------------- launchers
// Every launcher covers B systems of one shape: grid (blocks per system, B).
template <typename Kern>
int blocks_per_sm(Kern kern) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

// Blocks per system: enough for the sites, at most `cap` resident blocks
// shared by the B systems (at least one each) and the scratch's capacity.
inline dim3 batch_grid(size_t n, int cap, int B, int scratch_blocks = 1 << 30) {
    const size_t need = (n + kThreads - 1) / kThreads;
    const int per = std::max(1, std::min(cap / std::max(B, 1), scratch_blocks));
    return dim3((unsigned)std::max<size_t>(1, std::min<size_t>(need, (size_t)per)), (unsigned)B);
}
inline dim3 elementwise_grid(size_t n, int B) { return batch_grid(n, num_sms() * 8, B); }

// The two-site kernel needs an even row length (pairs never straddle rows)
// and arrays aligned for two-element loads of every type it reads.
inline bool pairs_apply(const Grid& g, const RelaxIO& io) {
    auto al = [](const void* p, uintptr_t a) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % a == 0; };
    return g.nx % 2 == 0 && al(io.f_in, 16) && al(io.f_out, 16) && al(io.u_in, 16) && al(io.psi_out, 16) &&
           al(io.V, 16);
}

// One launch of the one-site kernel (PF: next orbital prefetched) / of the
// two-site kernel for NO orbitals of B systems.
template <typename TS, typename T, int NO, bool OM1, bool BATCHED, bool PF>
cudaError_t launch_stream_collide(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                  cudaStream_t st) {
    auto kern = k_stream_collide<TS, T, NO, OM1, BATCHED, PF>;
    static const int nb = blocks_per_sm(kern);
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    kern<<<batch_grid(g.N, nb * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(g, c, io, sc);
    count_launches(1);
    return cudaGetLastError();
}
template <typename TS, typename T, int NO, bool OM1, bool BATCHED, int W>
cudaError_t launch_stream_collide_row(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                      cudaStream_t st) {
    auto kern = k_stream_collide_pair<TS, T, NO, OM1, BATCHED, W>;
    static const int nb = blocks_per_sm(kern);
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    kern<<<batch_grid(g.N / W, nb * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(g, c, io, sc);
    count_launches(1);
    return cudaGetLastError();
}
// W sites per thread: four where the populations are bfloat16 and the rows
// take whole groups of four (the arrays are 16-byte aligned, pairs_apply),
// else two.
template <typename TS, typename T, int NO, bool OM1, bool BATCHED>
cudaError_t launch_stream_collide_pair(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                       cudaStream_t st) {
    constexpr int W4 = row_width_max<TS>();
    if (W4 == 4 && g.nx % 4 == 0)
        return launch_stream_collide_row<TS, T, NO, OM1, BATCHED, W4>(g, c, io, sc, B, st);
    return launch_stream_collide_row<TS, T, NO, OM1, BATCHED, 2>(g, c, io, sc, B, st);
}

// The two-site and the prefetching variants for NO <= kMaxOrb orbitals, each
// compiled in a translation unit of its own (lbks_relax_<precision>_<variant>.cu)
// so that the per-precision units stay small enough to build in parallel.
// The row (two- or four-site) kernels are compiled in five translation units
// per precision -- orbital counts 1-4, and 5, 6, 7, 8 one each -- so that no
// unit holds more than a few of them.
template <typename TS, typename T, int LO, int HI>
cudaError_t launch_relax_pairs_range(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io,
                                     const Scratch& sc, int B, cudaStream_t st);
template <typename TS, typename T>
inline cudaError_t launch_relax_pairs(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io,
                                      const Scratch& sc, int B, cudaStream_t st) {
    switch (NO) {
        case 5: return launch_relax_pairs_range<TS, T, 5, 5>(NO, om1, g, c, io, sc, B, st);
        case 6: return launch_relax_pairs_range<TS, T, 6, 6>(NO, om1, g, c, io, sc, B, st);
        case 7: return launch_relax_pairs_range<TS, T, 7, 7>(NO, om1, g, c, io, sc, B, st);
        case 8: return launch_relax_pairs_range<TS, T, 8, 8>(NO, om1, g, c, io, sc, B, st);
        default: return launch_relax_pairs_range<TS, T, 1, 4>(NO, om1, g, c, io, sc, B, st);
    }
}
template <typename TS, typename T>
cudaError_t launch_relax_prefetch(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io,
                                  const Scratch& sc, int B, cudaStream_t st);
// The bulk-copy stream-collide (lbks_bulk.cuh) for any orbital count, its
// overlap fused (exact: FP64 products); FP32 and bfloat16 populations.
template <typename TS, typename T>
cudaError_t launch_relax_bulk(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                              bool exact, cudaStream_t st);
// Orbital-storage relaxation at omega = 1 (lbks_psi.cuh; io.f_in / f_out hold
// psi, io.V the potential of the collision that produced psi), compiled in
// lbks_relax_<precision>_psi.cu.
// kernel: kPsiKernelTiled, kPsiKernelDirect or kPsiKernelTma (the last needs
// psi_tma_applies and forms the W source from io.lambda_in at any orbital count).
template <typename T>
cudaError_t launch_relax_psi(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                             int kernel, cudaStream_t st);

// The bulk copies need 16-byte pieces of whole index ranges: N a multiple of
// the elements per 16 bytes of the populations and of the W field, 16-byte
// aligned arrays, and omega = 1 (three distinct post-collision values).
inline bool bulk_applies(const Grid& g, const Coef& c, const RelaxIO& io, size_t elem) {
    auto al = [](const void* p) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    return c.omega == 1.0 && g.N % (16 / elem) == 0 && g.N % 4 == 0 && al(io.f_in) && al(io.f_out) &&
           al(io.u_in) && al(io.psi_out) && al(io.V);
}

template <typename TS, typename T>
struct Ops {
    template <int NO, bool OM1>
    static cudaError_t relax_nm(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                int variant, cudaStream_t st) {
        const int v = variant & kRelaxVariantMask;
        if (v == kRelaxPairs && pairs_apply(g, io)) return launch_relax_pairs<TS, T>(NO, OM1, g, c, io, sc, B, st);
        if (v == kRelaxPrefetch && NO > 1) return launch_relax_prefetch<TS, T>(NO, OM1, g, c, io, sc, B, st);
        if constexpr (sizeof(T) == 4)
            if (v == kRelaxBulk && bulk_applies(g, c, io, sizeof(TS)))
                return launch_relax_bulk<TS, T>(NO, g, c, io, sc, B, (variant & kRelaxExactOverlap) != 0, st);
        return B > 1 ? launch_stream_collide<TS, T, NO, OM1, true, false>(g, c, io, sc, B, st)
                     : launch_stream_collide<TS, T, NO, OM1, false, false>(g, c, io, sc, B, st);
    }
    template <int NO>
    static cudaError_t relax_n(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                               int variant, cudaStream_t st) {
        return c.omega == 1.0 ? relax_nm<NO, true>(g, c, io, sc, B, variant, st)
                              : relax_nm<NO, false>(g, c, io, sc, B, variant, st);
    }
    template <int NO>
    static cudaError_t wfield_n(const Grid& g, double omega, const void* psi, const double* lam, void* u, int B,
                                cudaStream_t st) {
        if (NO < 2) return cudaSuccess;
        auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
        if (sizeof(T) == 4 && g.N % 4 == 0 && al(psi) && al(u))
            k_w_field4<NO><<<elementwise_grid(g.N / 4, B), kThreads, 0, st>>>(g, omega, (const float*)psi, lam,
                                                                              (float*)u);
        else
            k_w_field<T, NO><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, omega, (const T*)psi, lam, (T*)u);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t orth_n(const Grid& g, const double* Linv, void* f, void* psi, int B, cudaStream_t st) {
        k_orth_apply<TS, T, NO><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, Linv, (TS*)f, (T*)psi);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t gram_n(const Grid& g, double h, const void* psi, double* S, const Scratch& sc, int B,
                              cudaStream_t st) {
        auto kern = k_gram<T, NO>;
        if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
        kern<<<batch_grid(g.N, blocks_per_sm(kern) * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(
            g, h, (const T*)psi, S, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t init_n(const Grid& g, double h, const OrbitalStart* starts, void* psi, int B,
                              cudaStream_t st) {
        k_init_orbitals<T, NO><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, h, starts, (T*)psi);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t eq_n(const Grid& g, const Coef& c, const void* psi, void* f, int B, cudaStream_t st) {
        k_equilibrium<TS, T, NO><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, c, (const T*)psi, (TS*)f);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t density_n(const Grid& g, double h, const void* psi, double* rho, const double* rho_ref,
                                 double* mp, const Scratch& sc, int B, cudaStream_t st) {
        auto kern = k_density<T, NO>;
        if (sc.max_vals < 12 || sc.systems < B) return cudaErrorInvalidValue;
        kern<<<batch_grid(g.N, blocks_per_sm(kern) * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(
            g, h, (const T*)psi, rho, rho_ref, mp, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    template <int NO>
    static cudaError_t energy_n(const Grid& g, const Coef& c, const void* psi, const double* V, double* out,
                                const Scratch& sc, int B, cudaStream_t st) {
        auto kern = k_energy_matrix<T, NO>;
        if (sc.max_vals < NO * NO + NO || sc.systems < B) return cudaErrorInvalidValue;
        kern<<<batch_grid(g.N, blocks_per_sm(kern) * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(
            g, c, (const T*)psi, V, out, sc);
        count_launches(1);
        return cudaGetLastError();
    }

    // ---- more than kMaxOrb orbitals (runtime orbital count)
    template <typename Kern>
    static cudaError_t with_smem(Kern kern, size_t bytes) {
        return bytes > 48 * 1024 ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                                 : cudaSuccess;
    }
    static dim3 tile_grid(const Grid& g, int B, const Scratch& sc) {
        const size_t tiles = (g.N + kWideTile - 1) / kWideTile;
        const int per = std::max(1, std::min(sc.max_blocks, num_sms() * 2 / std::max(B, 1)));
        return dim3((unsigned)std::max<size_t>(1, std::min<size_t>(tiles, (size_t)per)), (unsigned)B);
    }
    // FP32 orbitals, per-step overlap (sigma and Lambda, which every step
    // measures again): tensor cores.  exact: FP64 sums of SIMT products (the
    // orthonormalising overlaps, where the tensor cores' truncating FP32
    // accumulation would leave a ~1e-6 relative bias on the norms).
    template <bool LAM>
    static cudaError_t gram_wide(int NO, const Grid& g, double h, const void* psi, double* S, double* lam,
                                 double* sigma, const Scratch& sc, int B, cudaStream_t st, bool exact = !LAM) {
        const int NP = NO * (NO + 1) / 2;
        if (sc.max_vals < NP || sc.systems < B) return cudaErrorInvalidValue;
        if constexpr (std::is_same<T, float>::value)
            if (!exact) return launch_gram_tc(NO, g, h, (const float*)psi, S, lam, sigma, sc, B, st);
        auto kern = k_gram_wide<T, LAM>;
        const size_t smem = (size_t)NO * kWideTile * sizeof(T) + sizeof(double) * NP;
        cudaError_t e = with_smem(kern, smem);
        if (e != cudaSuccess) return e;
        kern<<<tile_grid(g, B, sc), kThreads, smem, st>>>(g, h, (const T*)psi, NO, S, lam, sigma, sc);
        count_launches(1);
        return cudaGetLastError();
    }
    static cudaError_t relax_wide(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                  int variant, cudaStream_t st) {
        if constexpr (sizeof(T) == 4)
            if ((variant & kRelaxVariantMask) == kRelaxBulk && bulk_applies(g, c, io, sizeof(TS)))
                return launch_relax_bulk<TS, T>(NO, g, c, io, sc, B, (variant & kRelaxExactOverlap) != 0, st);
        if ((size_t)NO * B > 65535) return cudaErrorInvalidConfiguration;
        if ((variant & kRelaxVariantMask) == kRelaxPairs && pairs_apply(g, io)) {
            auto kern =
                c.omega == 1.0 ? k_stream_collide_wide_pair<TS, T, true> : k_stream_collide_wide_pair<TS, T, false>;
            kern<<<dim3((g.N / 2 + kThreads - 1) / kThreads, (unsigned)(NO * B)), kThreads, 0, st>>>(g, c, io, NO);
        } else {
            auto kern = c.omega == 1.0 ? k_stream_collide_wide<TS, T, true> : k_stream_collide_wide<TS, T, false>;
            kern<<<dim3((g.N + kThreads - 1) / kThreads, (unsigned)(NO * B)), kThreads, 0, st>>>(g, c, io, NO);
        }
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return gram_wide<true>(NO, g, c.h, io.psi_out, io.S_out, io.lambda_out, io.sigma_out, sc, B, st,
                               (variant & kRelaxExactOverlap) != 0);
    }
    template <int MAXO>
    static cudaError_t wfield_wide_m(int NO, const Grid& g, double omega, const void* psi, const double* lam,
                                     void* u, int B, cudaStream_t st) {
        if constexpr (sizeof(T) == 4 && MAXO >= 32 && MAXO <= 48) {  // FP32: two sites per thread, packed FMAs (spill-free here)
            auto kern = k_w_field_wide2<MAXO>;
            static const int nb = blocks_per_sm(kern);
            kern<<<batch_grid((g.N + 1) / 2, nb * num_sms(), B), kThreads, 0, st>>>(g, omega, (const float*)psi, lam,
                                                                                    (float*)u, NO);
        } else {
            auto kern = k_w_field_wide<T, MAXO>;
            static const int nb = blocks_per_sm(kern);
            kern<<<batch_grid(g.N, nb * num_sms(), B), kThreads, 0, st>>>(g, omega, (const T*)psi, lam, (T*)u, NO);
        }
        count_launches(1);
        return cudaGetLastError();
    }
    static cudaError_t wfield_wide(int NO, const Grid& g, double omega, const void* psi, const double* lam, void* u,
                                   int B, cudaStream_t st) {
        if (NO <= 16) return wfield_wide_m<16>(NO, g, omega, psi, lam, u, B, st);
        if (NO <= 24) return wfield_wide_m<24>(NO, g, omega, psi, lam, u, B, st);
        if (NO <= 32) return wfield_wide_m<32>(NO, g, omega, psi, lam, u, B, st);
        if (NO <= 40) return wfield_wide_m<40>(NO, g, omega, psi, lam, u, B, st);
        if (NO <= 48) return wfield_wide_m<48>(NO, g, omega, psi, lam, u, B, st);
        return wfield_wide_m<kMaxOrbWide>(NO, g, omega, psi, lam, u, B, st);
    }
    template <int MAXO>
    static cudaError_t orth_wide_m(int NO, const Grid& g, const double* Linv, void* f, void* psi, int B,
                                   cudaStream_t st) {
        auto kern = k_orth_apply_wide_reg<TS, T, MAXO>;
        static const int nb = blocks_per_sm(kern);
        kern<<<batch_grid(g.N, nb * num_sms(), B), kThreads, 0, st>>>(g, Linv, (TS*)f, (T*)psi, NO);
        count_launches(1);
        return cudaGetLastError();
    }
    static cudaError_t orth_wide(int NO, const Grid& g, const double* Linv, void* f, void* psi, int B,
                                 cudaStream_t st) {
        if (NO <= 16) return orth_wide_m<16>(NO, g, Linv, f, psi, B, st);
        if (NO <= 24) return orth_wide_m<24>(NO, g, Linv, f, psi, B, st);
        if (NO <= 32) return orth_wide_m<32>(NO, g, Linv, f, psi, B, st);
        if (NO <= 40) return orth_wide_m<40>(NO, g, Linv, f, psi, B, st);
        if (NO <= 48) return orth_wide_m<48>(NO, g, Linv, f, psi, B, st);
        const size_t smem = ((size_t)NO * kThreads + (size_t)NO * NO) * sizeof(T);
        cudaError_t e = with_smem(k_orth_apply_wide<TS, T>, smem);
        if (e != cudaSuccess) return e;
        k_orth_apply_wide<TS, T><<<batch_grid(g.N, num_sms() * 2, B), kThreads, smem, st>>>(g, Linv, (TS*)f, (T*)psi,
                                                                                             NO);
        count_launches(1);
        return cudaGetLastError();
    }
    static cudaError_t energy_wide(int NO, const Grid& g, const Coef& c, const void* psi, const double* V, double* out,
                                   const Scratch& sc, int B, cudaStream_t st) {
        const int K = NO * (NO + 1) / 2 + NO;
        if (sc.max_vals < K || sc.systems < B) return cudaErrorInvalidValue;
        const size_t smem = 3 * (size_t)NO * kWideTile * sizeof(T) + sizeof(double) * K;
        cudaError_t e = with_smem(k_energy_matrix_wide<T>, smem);
        if (e != cudaSuccess) return e;
        k_energy_matrix_wide<T><<<tile_grid(g, B, sc), kThreads, smem, st>>>(g, c, (const T*)psi, V, out, sc, NO);
        count_launches(1);
        return cudaGetLastError();
    }

#define LBKS_SWITCH_NO(CALL)                  \
    switch (n_orb) {                          \
        case 1: return CALL(1);               \
        case 2: return CALL(2);               \
        case 3: return CALL(3);               \
        case 4: return CALL(4);               \
        case 5: return CALL(5);               \
        case 6: return CALL(6);               \
        case 7: return CALL(7);               \
        case 8: return CALL(8);               \
        default: return n_orb <= kMaxOrbWide ? WIDE : cudaErrorInvalidValue; \
    }
    static cudaError_t relax(int n_orb, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                             int variant, cudaStream_t st) {
#define CALL(NO) relax_n<NO>(g, c, io, sc, B, variant, st)
#define WIDE relax_wide(n_orb, g, c, io, sc, B, variant, st)
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t w_field(int n_orb, const Grid& g, double omega, const void* psi, const double* lam, void* u,
                               int B, cudaStream_t st) {
#define CALL(NO) wfield_n<NO>(g, omega, psi, lam, u, B, st)
#define WIDE wfield_wide(n_orb, g, omega, psi, lam, u, B, st)
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t orth_apply(int n_orb, const Grid& g, const double* Linv, void* f, void* psi, int B,
                                  cudaStream_t st) {
#define CALL(NO) orth_n<NO>(g, Linv, f, psi, B, st)
#define WIDE orth_wide(n_orb, g, Linv, f, psi, B, st)
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t gram(int n_orb, const Grid& g, double h, const void* psi, double* S, const Scratch& sc, int B,
                            cudaStream_t st) {
#define CALL(NO) gram_n<NO>(g, h, psi, S, sc, B, st)
#define WIDE gram_wide<false>(n_orb, g, h, psi, S, nullptr, nullptr, sc, B, st)
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t init_orbitals(int n_orb, const Grid& g, double h, const OrbitalStart* o, void* psi, int B,
                                     cudaStream_t st) {
#define CALL(NO) init_n<NO>(g, h, o, psi, B, st)
#define WIDE (k_init_orbitals_wide<T><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, h, o, (T*)psi, n_orb), \
              count_launches(1), cudaGetLastError())
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t equilibrium(int n_orb, const Grid& g, const Coef& c, const void* psi, void* f, int B,
                                   cudaStream_t st) {
#define CALL(NO) eq_n<NO>(g, c, psi, f, B, st)
#define WIDE (k_equilibrium_wide<TS, T><<<elementwise_grid(g.N, B), kThreads, 0, st>>>(g, c, (const T*)psi, (TS*)f, \
                                                                                         n_orb),                   \
              count_launches(1), cudaGetLastError())
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t density(int n_orb, const Grid& g, double h, const void* psi, double* rho,
                               const double* rho_ref, double* mp, const Scratch& sc, int B, cudaStream_t st) {
#define CALL(NO) density_n<NO>(g, h, psi, rho, rho_ref, mp, sc, B, st)
#define WIDE (k_density_wide<T><<<batch_grid(g.N, num_sms() * 4, B, sc.max_blocks), kThreads, 0, st>>>(    \
                  g, h, (const T*)psi, rho, rho_ref, mp, sc, n_orb),                                     \
              count_launches(1), cudaGetLastError())
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
    static cudaError_t energy_matrix(int n_orb, const Grid& g, const Coef& c, const void* psi, const double* V,
                                     double* out, const Scratch& sc, int B, cudaStream_t st) {
#define CALL(NO) energy_n<NO>(g, c, psi, V, out, sc, B, st)
#define WIDE energy_wide(n_orb, g, c, psi, V, out, sc, B, st)
        LBKS_SWITCH_NO(CALL)
#undef WIDE
#undef CALL
    }
#undef LBKS_SWITCH_NO

    static cudaError_t relax_psi(int n_orb, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc,
                                 int B, int variant, cudaStream_t st) {
        // variant kPsiKernelTiled: the shared-memory tiled stencil; kPsiKernelDirect: one site per thread
        // from L1; kPsiKernelTma: boxes copied by the tensor memory accelerator (anything else: tiled)
        // (the tiled kernel's tile shape rides in the bits from kPsiShapeShift on)
        const int v = variant & kRelaxVariantMask;
        const int shape = variant & (0xff << kPsiShapeShift);
        cudaError_t e = launch_relax_psi<T>(
            n_orb, g, c, io, sc, B,
            v == kPsiKernelDirect || v == kPsiKernelTma || v == kPsiKernelZ ? v : (kPsiKernelTiled | shape), st);
        if (e != cudaSuccess || n_orb <= kMaxOrb) return e;  // up to kMaxOrb: overlap fused
        return gram_wide<true>(n_orb, g, c.h, io.f_out, io.S_out, io.lambda_out, io.sigma_out, sc, B, st,
                               (variant & kRelaxExactOverlap) != 0);
    }
    static const PrecisionOps& table() {
        static const PrecisionOps t = {&relax,   &relax_psi, &w_field, &orth_apply,    &gram,      &init_orbitals,
                                       &equilibrium, &density, &energy_matrix, sizeof(TS), sizeof(T)};
        return t;
    }
};

}  // namespace lbks
