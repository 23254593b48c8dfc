// Relaxation kernels for more orbitals than the fused kernel handles
// (kMaxOrb < N_O <= kMaxOrbWide): the orbital count is a runtime value, the
// overlap products leave the stream-collide kernel for a tiled Gram kernel
// (the N_O x N_O x N contraction S = h^3 Psi Psi^T), and the W field, the
// orthonormalisation and the energy matrix stage orbital tiles in shared
// memory.  Included by lbks_relax.cuh; same conventions (system = blockIdx.y,
// arrays of consecutive systems, TS storage / T arithmetic).
#pragma once

namespace lbks {

constexpr int kWideTile = 64;  // sites per shared-memory tile

// Fused pull-stream + normalisation + collision + potential source, one
// (site, orbital) per thread: blockIdx.y = system * N_O + orbital, so the
// blocks of one orbital stream through its 19 population arrays together.
// psi is written for the Gram kernel.  Every orbital also rereads V (8 B per
// orbital-site, mostly from L2).
template <typename TS, typename T, bool OM1>
__global__ void __launch_bounds__(kThreads, 4) k_stream_collide_wide(Grid g, Coef c, RelaxIO io, int NO) {
    const int y = (int)blockIdx.y / NO, j = (int)blockIdx.y - y * NO;
    if (g.active && !g.active[y]) return;
    const uint32_t N = g.N;
    const uint32_t s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= N) return;
    const size_t oj = (size_t)y * NO + j;  // orbital index over all systems
    const TS* __restrict__ fj = static_cast<const TS*>(io.f_in) + oj * 19 * N;
    const T* __restrict__ uj =
        (j > 0 && io.u_in != nullptr) ? static_cast<const T*>(io.u_in) + ((size_t)y * (NO - 1) + j - 1) * N : nullptr;
    TS* __restrict__ out = static_cast<TS*>(io.f_out) + oj * 19 * N;
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const Site t = decode(g, s);
    T gp[19];
#pragma unroll
    for (int p = 0; p < 19; ++p)
        gp[p] = has_source(t, p) ? to_compute<T>(ld_ro(fj + (size_t)p * N + source_index(g, s, p))) : T(0);
    if (uj) {
#pragma unroll
        for (int p = 0; p < 19; ++p)
            if (has_source(t, p)) gp[p] += xi[vclass(p)] * ld_ro(uj + source_index(g, s, p));
    }
    const T vr = (T)__ldg(io.V + (size_t)y * N + s);
    T ps = T(0);
#pragma unroll
    for (int p = 0; p < 19; ++p) ps += gp[p];
    const T sig = (T)io.sigma_in[oj];
    ps *= sig;
    const T A = om * ps, B = dt * vr * ps;
    const T e[3] = {xi[0] * A - chi[0] * B, xi[1] * A - chi[1] * B, xi[2] * A - chi[2] * B};
    const T c1 = om1 * sig;
#pragma unroll
    for (int p = 0; p < 19; ++p)
        st_stream(out + (size_t)p * N + s, to_store<TS>(OM1 ? e[vclass(p)] : c1 * gp[p] + e[vclass(p)]));
    static_cast<T*>(io.psi_out)[oj * N + s] = ps;
}

// S = h^3 Psi Psi^T over the packed lower triangle (NP pairs): tiles of
// kWideTile sites in shared memory, per-thread pair sums in T over a tile,
// FP64 across tiles and blocks.  With LAM: Lambda and sigma as in the fused
// kernel.  Dynamic shared memory: NO * kWideTile * sizeof(T) + NP doubles.
template <typename T, bool LAM>
__global__ void __launch_bounds__(kThreads) k_gram_wide(Grid g, double h, const T* __restrict__ psi, int NO,
                                                        double* S, double* lam, double* sigma, Scratch sc) {
    if (inactive(g)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);  // [NO][kWideTile]
    double* tot = reinterpret_cast<double*>(smem + (size_t)NO * kWideTile * sizeof(T));
    const int NP = NO * (NO + 1) / 2;
    const uint32_t N = g.N;
    const size_t y = sys_id();
    psi += y * NO * N;
    constexpr int kMaxPairsPerThread = (kMaxOrbWide * (kMaxOrbWide + 1) / 2 + kThreads - 1) / kThreads;
    double acc[kMaxPairsPerThread];
    int pa[kMaxPairsPerThread], pb[kMaxPairsPerThread];
#pragma unroll
    for (int q = 0; q < kMaxPairsPerThread; ++q) {
        acc[q] = 0.0;
        const int k = threadIdx.x + q * kThreads;
        if (k < NP) tri_pair(k, pa[q], pb[q]);
        else pa[q] = pb[q] = -1;
    }
    const uint32_t tiles = (N + kWideTile - 1) / kWideTile;
    for (uint32_t ti = blockIdx.x; ti < tiles; ti += gridDim.x) {
        const uint32_t base = ti * kWideTile;
        for (int i = threadIdx.x; i < NO * kWideTile; i += kThreads) {
            const int j = i / kWideTile, s = i % kWideTile;
            tile[i] = (base + s < N) ? psi[(size_t)j * N + base + s] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxPairsPerThread; ++q) {
            if (pa[q] < 0) continue;
            const T* ra = tile + pa[q] * kWideTile;
            const T* rb = tile + pb[q] * kWideTile;
            T part = T(0);
#pragma unroll 8
            for (int s = 0; s < kWideTile; ++s) part += ra[s] * rb[s];
            acc[q] += (double)part;
        }
        __syncthreads();
    }
    double* partial = sys_partial(sc);
#pragma unroll
    for (int q = 0; q < kMaxPairsPerThread; ++q) {
        const int k = threadIdx.x + q * kThreads;
        if (k < NP) partial[(size_t)blockIdx.x * NP + k] = acc[q];
    }
    if (grid_total_rt(partial, sys_counter(sc), tot, NP))
        store_overlap_block(tot, NO, h, S + y * NO * NO, LAM ? lam + y * NO * NO : nullptr,
                            LAM ? sigma + y * NO : nullptr);
}

// 16-byte shared-memory loads that the compiler may not hoist out of the
// site loop (it would otherwise keep the whole coefficient matrix live in
// registers and spill).
__device__ __forceinline__ void lds16(const float* p, float (&v)[4]) {
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void lds16(const double* p, double (&v)[2]) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "r"((uint32_t)__cvta_generic_to_shared(p)));
}

// u_(j-1) = -omega sum_{k<j} Lambda_jk psi_k, one site per thread: the
// site's N_O orbital values stay in registers (MAXO >= N_O, a compile-time
// bound; loops unrolled and cut at the runtime N_O) and -omega Lambda sits in
// shared memory (row pitch MAXO, zero beyond N_O and on and above the
// diagonal), read 16 bytes at a time by broadcast.  Streams psi in and u out
// once: HBM-bound.
template <typename T, int MAXO>
__global__ void __launch_bounds__(kThreads) k_w_field_wide(const Grid g, double omega, const T* __restrict__ psi,
                                                           const double* __restrict__ lam, T* __restrict__ u, int NO) {
    constexpr int V = 16 / sizeof(T);  // coefficients per shared-memory load
    static_assert(MAXO % V == 0, "row pitch must keep 16-byte alignment");
    if (inactive(g)) return;
    __shared__ __align__(16) T L[MAXO * MAXO];
    const size_t n = g.N, y = sys_id();
    psi += y * NO * n;
    lam += y * NO * NO;
    u += y * (NO - 1) * n;
    for (int i = threadIdx.x; i < MAXO * MAXO; i += kThreads) {
        const int j = i / MAXO, k = i % MAXO;
        L[i] = (j < NO && k < j) ? (T)(-omega * lam[j * NO + k]) : T(0);
    }
    __syncthreads();
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        T ps[MAXO];
        const T* pp = psi + s;
#pragma unroll
        for (int k = 0; k < MAXO; ++k) {
            ps[k] = k < NO ? __ldcs(pp) : T(0);
            pp += n;
        }
        T* up = u + s;
#pragma unroll
        for (int j = 1; j < MAXO; ++j) {
            if (j >= NO) break;
            T w = T(0);
#pragma unroll
            for (int kb = 0; kb < j; kb += V) {
                T l[V];
                lds16(&L[j * MAXO + kb], l);
#pragma unroll
                for (int e = 0; e < V; ++e) w += l[e] * ps[kb + e];
            }
            __stcs(up, w);
            up += n;
        }
    }
}

// FP32 form of k_w_field_wide with two sites per thread (s and s + kThreads
// of a 2 kThreads-site chunk): the two sites' values of an orbital form one
// float2, so each 16-byte broadcast load of -omega Lambda serves both sites
// and each packed FMA (fma.rn.f32x2, __ffma2_rn) does both: half the shared
// loads and half the FMA instructions per site.
template <int MAXO>
__global__ void __launch_bounds__(kThreads, 2) k_w_field_wide2(const Grid g, double omega,
                                                              const float* __restrict__ psi,
                                                              const double* __restrict__ lam, float* __restrict__ u,
                                                              int NO) {
    static_assert(MAXO % 4 == 0, "row pitch must keep 16-byte alignment");
    if (inactive(g)) return;
    __shared__ __align__(16) float L[MAXO * MAXO];
    const size_t n = g.N, y = sys_id();
    psi += y * NO * n;
    lam += y * NO * NO;
    u += y * (NO - 1) * n;
    for (int i = threadIdx.x; i < MAXO * MAXO; i += kThreads) {
        const int j = i / MAXO, k = i % MAXO;
        L[i] = (j < NO && k < j) ? (float)(-omega * lam[j * NO + k]) : 0.f;
    }
    __syncthreads();
    const size_t chunk = 2 * (size_t)kThreads;
    for (size_t base = blockIdx.x * chunk; base < n; base += (size_t)gridDim.x * chunk) {
        const size_t s0 = base + threadIdx.x, s1 = s0 + kThreads;
        const bool h0 = s0 < n, h1 = s1 < n;
        float2 ps[MAXO];
#pragma unroll
        for (int k = 0; k < MAXO; ++k) {
            ps[k].x = (k < NO && h0) ? __ldcs(psi + (size_t)k * n + s0) : 0.f;
            ps[k].y = (k < NO && h1) ? __ldcs(psi + (size_t)k * n + s1) : 0.f;
        }
#pragma unroll
        for (int j = 1; j < MAXO; ++j) {
            if (j >= NO) break;
            float2 w = make_float2(0.f, 0.f);
#pragma unroll
            for (int kb = 0; kb < j; kb += 4) {
                float l[4];
                lds16(&L[j * MAXO + kb], l);
#pragma unroll
                for (int e = 0; e < 4; ++e) w = __ffma2_rn(make_float2(l[e], l[e]), ps[kb + e], w);
            }
            if (h0) __stcs(u + (size_t)(j - 1) * n + s0, w.x);
            if (h1) __stcs(u + (size_t)(j - 1) * n + s1, w.y);
        }
    }
}

// In-place orthonormalisation f_jp <- sum_k Linv_jk f_kp, psi likewise:
// per site, one velocity at a time, the NO values staged per thread in
// shared memory.  Dynamic shared memory: (NO * kThreads + NO * NO) * sizeof(T).
// The same with each site's NO values of one population in registers (MAXO
// a compile-time bound on NO) and L^-1 in shared memory read 16 bytes at a
// time by every thread of the warp at once (broadcast): the triangular
// product costs one shared-memory load per four (FP32) or two (FP64)
// multiply-adds instead of two loads per multiply-add.  Rows are formed from
// the top, so row j reads the original values k <= j, not yet overwritten.
template <typename TS, typename T, int MAXO>
__global__ void __launch_bounds__(kThreads) k_orth_apply_wide_reg(const Grid g, const double* __restrict__ Linv,
                                                                  TS* __restrict__ f, T* __restrict__ psi, int NO) {
    constexpr int V = 16 / sizeof(T);  // coefficients per shared-memory load
    static_assert(MAXO % V == 0, "row pitch must keep 16-byte alignment");
    if (inactive(g)) return;
    __shared__ __align__(16) T L[MAXO * MAXO];
    const size_t n = g.N, y = sys_id();
    Linv += y * NO * NO;
    if (f) f += y * NO * 19 * n;
    if (psi) psi += y * NO * n;
    for (int i = threadIdx.x; i < MAXO * MAXO; i += kThreads) {
        const int j = i / MAXO, k = i % MAXO;
        L[i] = (j < NO && k <= j) ? (T)Linv[j * NO + k] : T(0);
    }
    __syncthreads();
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        for (int p = (f ? 0 : 19); p <= 19; ++p) {
            if (p == 19 && !psi) break;
            T x[MAXO];
#pragma unroll
            for (int k = 0; k < MAXO; ++k)
                x[k] = k >= NO ? T(0)
                       : (p < 19) ? to_compute<T>(f[((size_t)k * 19 + p) * n + s])
                                  : psi[(size_t)k * n + s];
#pragma unroll
            for (int j = MAXO - 1; j >= 0; --j) {
                if (j >= NO) continue;
                T w = T(0);
#pragma unroll
                for (int kb = 0; kb <= j; kb += V) {
                    T l[V];
                    lds16(&L[j * MAXO + kb], l);
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (kb + e <= j) w += l[e] * x[kb + e];
                }
                x[j] = w;
            }
#pragma unroll
            for (int j = 0; j < MAXO; ++j) {
                if (j >= NO) break;
                if (p < 19) f[((size_t)j * 19 + p) * n + s] = to_store<TS>(x[j]);
                else psi[(size_t)j * n + s] = x[j];
            }
        }
    }
}

template <typename TS, typename T>
__global__ void __launch_bounds__(kThreads) k_orth_apply_wide(const Grid g, const double* __restrict__ Linv,
                                                              TS* __restrict__ f, T* __restrict__ psi, int NO) {
    if (inactive(g)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    T* col = reinterpret_cast<T*>(smem);  // [NO][kThreads]
    T* L = col + (size_t)NO * kThreads;   // [NO][NO]
    const size_t n = g.N, y = sys_id();
    Linv += y * NO * NO;
    if (f) f += y * NO * 19 * n;
    if (psi) psi += y * NO * n;
    for (int i = threadIdx.x; i < NO * NO; i += kThreads) L[i] = (T)Linv[i];
    __syncthreads();
    T* mine = col + threadIdx.x;
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads) {
        for (int p = (f ? 0 : 19); p <= 19; ++p) {
            if (p == 19 && !psi) break;
            for (int k = 0; k < NO; ++k)
                mine[k * kThreads] = (p < 19) ? to_compute<T>(f[((size_t)k * 19 + p) * n + s]) : psi[(size_t)k * n + s];
            for (int j = NO - 1; j >= 0; --j) {  // from the top: row j reads rows k <= j, not yet overwritten
                T o = T(0);
                for (int k = 0; k <= j; ++k) o += L[j * NO + k] * mine[k * kThreads];
                mine[j * kThreads] = o;
            }
            for (int j = 0; j < NO; ++j) {
                if (p < 19) f[((size_t)j * 19 + p) * n + s] = to_store<TS>(mine[j * kThreads]);
                else psi[(size_t)j * n + s] = mine[j * kThreads];
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_init_orbitals_wide(Grid g, double h, const OrbitalStart* __restrict__ starts,
                                                                 T* __restrict__ psi, int NO) {
    if (inactive(g)) return;
    const uint32_t N = g.N;
    const OrbitalStart* st = starts + (size_t)sys_id() * NO;
    psi += (size_t)sys_id() * NO * N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const uint32_t q = g.divx.div(s);
        const int x = (int)(s - q * (uint32_t)g.nx);
        const uint32_t z = g.divy.div(q);
        const int yy = (int)(q - z * (uint32_t)g.ny);
        const double rx = (x - 0.5 * (g.nx - 1)) * h, ry = (yy - 0.5 * (g.ny - 1)) * h,
                     rz = ((int)z - 0.5 * (g.nz - 1)) * h;
        for (int j = 0; j < NO; ++j) {
            const double dx = rx - st[j].cx, dy = ry - st[j].cy, dz = rz - st[j].cz;
            const double w = st[j].width;
            psi[(size_t)j * N + s] = (T)exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * w * w));
        }
    }
}

template <typename TS, typename T>
__global__ void __launch_bounds__(kThreads) k_equilibrium_wide(const Grid g, Coef c, const T* __restrict__ psi,
                                                               TS* __restrict__ f, int NO) {
    if (inactive(g)) return;
    const size_t n = g.N;
    psi += (size_t)sys_id() * NO * n;
    f += (size_t)sys_id() * NO * 19 * n;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    for (size_t s = blockIdx.x * (size_t)kThreads + threadIdx.x; s < n; s += (size_t)gridDim.x * kThreads)
        for (int j = 0; j < NO; ++j) {
            const T a = psi[(size_t)j * n + s];
#pragma unroll
            for (int p = 0; p < 19; ++p) f[((size_t)j * 19 + p) * n + s] = to_store<TS>(xi[vclass(p)] * a);
        }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_density_wide(Grid g, double h, const T* __restrict__ psi,
                                                           double* __restrict__ rho, const double* rho_ref,
                                                           double* mp, Scratch sc, int NO) {
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
        const int yy = (int)(q - z * (uint32_t)g.ny);
        const double rx = (x - 0.5 * (g.nx - 1)) * h, ry = (yy - 0.5 * (g.ny - 1)) * h,
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

// Energy matrix for many orbitals: per tile, psi, (T_h + V) psi and T_h psi in
// shared memory; H over the packed lower triangle (symmetrised by the host)
// and kin on the diagonal, FP64 across tiles and blocks.  Output per system
// (kEmatWideStride doubles): H[NO][NO] then kin[NO].
// Dynamic shared memory: 3 * NO * kWideTile * sizeof(T) + (NP + NO) doubles.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_energy_matrix_wide(Grid g, Coef c, const T* __restrict__ psi,
                                                                 const double* __restrict__ V, double* out, Scratch sc,
                                                                 int NO) {
    if (inactive(g)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    T* A = reinterpret_cast<T*>(smem);      // psi [NO][tile]
    T* Hp = A + (size_t)NO * kWideTile;     // (T_h + V) psi
    T* Tp = Hp + (size_t)NO * kWideTile;    // T_h psi
    double* tot = reinterpret_cast<double*>(Tp + (size_t)NO * kWideTile);
    const int NP = NO * (NO + 1) / 2, K = NP + NO;
    const uint32_t N = g.N;
    const size_t y = sys_id();
    psi += y * NO * N;
    V += y * N;
    out += y * kEmatWideStride;
    const T inv = (T)(1.0 / (c.theta * c.h * c.h));
    constexpr int kMaxPerThread = (kMaxOrbWide * (kMaxOrbWide + 1) / 2 + kMaxOrbWide + kThreads - 1) / kThreads;
    double acc[kMaxPerThread];
    int pa[kMaxPerThread], pb[kMaxPerThread];
#pragma unroll
    for (int q = 0; q < kMaxPerThread; ++q) {
        acc[q] = 0.0;
        const int k = threadIdx.x + q * kThreads;
        if (k < NP) tri_pair(k, pa[q], pb[q]);
        else if (k < K) pa[q] = pb[q] = -2 - (k - NP);  // kinetic term of orbital k - NP
        else pa[q] = pb[q] = -1;
    }
    const uint32_t tiles = (N + kWideTile - 1) / kWideTile;
    for (uint32_t ti = blockIdx.x; ti < tiles; ti += gridDim.x) {
        const uint32_t base = ti * kWideTile;
        for (int i = threadIdx.x; i < NO * kWideTile; i += kThreads) {
            const int j = i / kWideTile, sl = i % kWideTile;
            const uint32_t s = base + sl;
            T a = T(0), tp = T(0), hp = T(0);
            if (s < N) {
                const Site t = decode(g, s);
                const T* pj = psi + (size_t)j * N;
                a = pj[s];
                // (1 - K_xi) psi = sum_p xi_p (psi(r) - psi(r - v_p)) (sum_p xi_p = 1); a neighbour
                // outside the box is psi = 0, so its term is xi_p psi(r).  A difference is exact
                // in T when the two values are within a factor of two of each other (Sterbenz's
                // lemma), else it carries one rounding of the larger value.
                T d = T(0);
#pragma unroll
                for (int p = 1; p < 19; ++p)
                    d += (T)c.xi[vclass(p)] * (has_source(t, p) ? a - pj[source_index(g, s, p)] : a);
                tp = d * inv;
                hp = tp + (T)V[s] * a;
            }
            A[i] = a;
            Tp[i] = tp;
            Hp[i] = hp;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kMaxPerThread; ++q) {
            if (pa[q] == -1) continue;
            const T* ra;
            const T* rb;
            if (pa[q] >= 0) {
                ra = A + pa[q] * kWideTile;
                rb = Hp + pb[q] * kWideTile;
            } else {
                const int j = -2 - pa[q];
                ra = A + j * kWideTile;
                rb = Tp + j * kWideTile;
            }
            T part = T(0);
#pragma unroll 8
            for (int s = 0; s < kWideTile; ++s) part += ra[s] * rb[s];
            acc[q] += (double)part;
        }
        __syncthreads();
    }
    double* partial = sys_partial(sc);
#pragma unroll
    for (int q = 0; q < kMaxPerThread; ++q) {
        const int k = threadIdx.x + q * kThreads;
        if (k < K) partial[(size_t)blockIdx.x * K + k] = acc[q];
    }
    if (grid_total_rt(partial, sys_counter(sc), tot, K) && threadIdx.x == 0) {
        const double h3 = c.h * c.h * c.h;
        for (int a = 0; a < NO; ++a)
            for (int b = 0; b <= a; ++b) {
                out[a * NO + b] = h3 * tot[tri(a, b)];
                out[b * NO + a] = h3 * tot[tri(a, b)];
            }
        for (int j = 0; j < NO; ++j) out[NO * NO + j] = h3 * tot[NP + j];
    }
}

}  // namespace lbks
