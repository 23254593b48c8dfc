// Stream-collide over pairs of x-neighbouring sites (nx even): the same
// update as k_stream_collide, but every population of both sites arrives in
// one aligned two-element load (bfloat16 x 2 = 4 bytes, float x 2 = 8 bytes),
// which halves the load and store instructions per byte -- the limit of the
// one-site kernel with 2-byte bfloat16 populations.
//
// Pull streaming with a velocity of x-component +1 needs, for the pair's
// first site, the element left of the pair's source pair: the lane to the
// left loaded it (its pair lies two sites to the left in the same source
// row), so it arrives by warp shuffle; lane 0 loads it itself.  x-component
// -1 mirrors this with the lane to the right and lane 31.  Where the
// neighbouring lane sits in another row the element is not needed: the site
// is on the box face and has no source there.  Every lane of a warp runs the
// shuffles (lanes past the last pair load nothing).
// Included by lbks_relax.cuh.
#pragma once

namespace lbks {

template <typename TS>
struct Pack2;
template <>
struct Pack2<float> {
    using type = float2;
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ static float lo(float2 v) { return v.x; }
    __device__ static float hi(float2 v) { return v.y; }
    __device__ static float2 make(float a, float b) { return make_float2(a, b); }
};
template <>
struct Pack2<__nv_bfloat16> {
    using type = __nv_bfloat162;
    __device__ static __nv_bfloat162 zero() { return __floats2bfloat162_rn(0.f, 0.f); }
    __device__ static float lo(__nv_bfloat162 v) { return __low2float(v); }
    __device__ static float hi(__nv_bfloat162 v) { return __high2float(v); }
    __device__ static __nv_bfloat162 make(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <>
struct Pack2<double> {
    using type = double2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double lo(double2 v) { return v.x; }
    __device__ static double hi(double2 v) { return v.y; }
    __device__ static double2 make(double a, double b) { return make_double2(a, b); }
};

// Values of population array `src` (element type E) arriving along velocity
// p at the two sites of the pair: x-shift by shuffle as described above.
// row: index of the pair's source pair (s0 - offset of v_p without its x part).
// ok: the source row exists and the lane is live; v0 / v1: the x-source of
// site 0 / site 1 exists.
template <typename E, typename T, int VX>
__device__ __forceinline__ void pull_pair(const E* __restrict__ src, uint32_t row, bool ok, bool v0, bool v1,
                                          int lane, T& g0, T& g1) {
    using P = Pack2<E>;
    const typename P::type q = ok ? __ldg(reinterpret_cast<const typename P::type*>(src + row)) : P::zero();
    const T a = (T)P::lo(q), b = (T)P::hi(q);
    if (VX == 0) {
        g0 = a;
        g1 = b;
    } else if (VX > 0) {  // source x - 1
        T left = __shfl_up_sync(0xffffffffu, b, 1);
        if (lane == 0) left = (ok && v0) ? to_compute<T>(__ldg(src + row - 1)) : T(0);
        g0 = v0 ? left : T(0);
        g1 = a;
    } else {  // source x + 1
        T right = __shfl_down_sync(0xffffffffu, a, 1);
        if (lane == 31) right = (ok && v1) ? to_compute<T>(__ldg(src + row + 2)) : T(0);
        g0 = b;
        g1 = v1 ? right : T(0);
    }
}

// Velocities with x-component of the sign of sx (9, 5 and 5 for 0, +1, -1).
__host__ __device__ constexpr int vx_count(int sx) {
    int n = 0;
    for (int p = 0; p < 19; ++p) n += (vel(p, 0) > 0 ? 1 : vel(p, 0) < 0 ? -1 : 0) == sx ? 1 : 0;
    return n;
}

// pull_pair in two phases, so that all loads of a site pair are in flight
// before the first shuffle waits on one: load_pair issues the aligned pair
// load and, on the lanes at the warp's edges, the element beyond it;
// shift_pair then forms the two arriving values.
static_assert(vx_count(0) == 9 && vx_count(1) == 5 && vx_count(-1) == 5, "D3Q19 x-components");

template <typename E, int VX>
struct PairLoad {
    typename Pack2<E>::type q;
    E edge;
};
template <typename E, int VX>
__device__ __forceinline__ PairLoad<E, VX> load_pair(const E* __restrict__ src, uint32_t row, bool ok, bool v0,
                                                     bool v1, int lane) {
    using P = Pack2<E>;
    PairLoad<E, VX> r;
    r.q = ok ? __ldg(reinterpret_cast<const typename P::type*>(src + row)) : P::zero();
    r.edge = E(0);
    if (VX > 0 && lane == 0 && ok && v0) r.edge = __ldg(src + row - 1);
    if (VX < 0 && lane == 31 && ok && v1) r.edge = __ldg(src + row + 2);
    return r;
}
template <typename E, typename T, int VX>
__device__ __forceinline__ void shift_pair(const PairLoad<E, VX>& r, bool v0, bool v1, int lane, T& g0, T& g1) {
    using P = Pack2<E>;
    const T a = (T)P::lo(r.q), b = (T)P::hi(r.q);
    if (VX == 0) {
        g0 = a;
        g1 = b;
    } else if (VX > 0) {
        T left = __shfl_up_sync(0xffffffffu, b, 1);
        if (lane == 0) left = to_compute<T>(r.edge);
        g0 = v0 ? left : T(0);
        g1 = a;
    } else {
        T right = __shfl_down_sync(0xffffffffu, a, 1);
        if (lane == 31) right = to_compute<T>(r.edge);
        g0 = b;
        g1 = v1 ? right : T(0);
    }
}

// Sums of the populations of array base f (element E, one array of N per
// velocity; stride N between velocities, or 0 for the W field, whose single
// array is pulled along every velocity with weight xi_p) arriving at the two
// sites of the pair, every load issued before the first shuffle.  W
// (with the W field): adds xi_p w_p; KEEP: also stores each velocity's pair in
// g0/g1 (for the (1 - omega) term).
template <typename E, typename T, bool KEEP, int NG>
__device__ __forceinline__ void gather_pair(const E* __restrict__ f, size_t stride, const T (&wt)[3], bool weighted,
                                            const Grid& g, const Site& t, uint32_t s0, bool live, bool x0l, bool x1r,
                                            int lane, T& ps0, T& ps1, T (&g0)[NG], T (&g1)[NG]) {
    const int nxy = g.nx * g.ny;
    PairLoad<E, 0> l0[vx_count(0)];
    PairLoad<E, 1> lp[vx_count(1)];
    PairLoad<E, -1> lm[vx_count(-1)];
    int a = 0, b = 0, c = 0;
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        const int vy = vel(p, 1), vz = vel(p, 2);
        const bool ok = live && (vy == 0 || (vy > 0 ? t.ym : t.yp)) && (vz == 0 || (vz > 0 ? t.zm : t.zp));
        const uint32_t row = (uint32_t)((int)s0 - vy * g.nx - vz * nxy);
        const E* src = f + (size_t)p * stride;
        if (vel(p, 0) == 0) l0[a++] = load_pair<E, 0>(src, row, ok, true, true, lane);
        else if (vel(p, 0) > 0) lp[b++] = load_pair<E, 1>(src, row, ok, x0l, true, lane);
        else lm[c++] = load_pair<E, -1>(src, row, ok, true, x1r, lane);
    }
    a = b = c = 0;
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        T a0, a1;
        if (vel(p, 0) == 0) shift_pair<E, T, 0>(l0[a++], true, true, lane, a0, a1);
        else if (vel(p, 0) > 0) shift_pair<E, T, 1>(lp[b++], x0l, true, lane, a0, a1);
        else shift_pair<E, T, -1>(lm[c++], true, x1r, lane, a0, a1);
        if (weighted) {
            a0 *= wt[vclass(p)];
            a1 *= wt[vclass(p)];
        }
        ps0 += a0;
        ps1 += a1;
        if constexpr (KEEP) {
            g0[p] += a0;
            g1[p] += a1;
        }
    }
}

// W consecutive elements of one array in one aligned load (W = 2, or 4 for
// float and bfloat16), unpacked to the compute type T and packed from it.
template <typename E, int W>
struct VecW;
template <>
struct VecW<float, 2> {
    using type = float2;
    template <typename T>
    __device__ static void get(float2 v, T (&a)[2]) { a[0] = (T)v.x; a[1] = (T)v.y; }
    __device__ static float2 put(const float (&a)[2]) { return make_float2(a[0], a[1]); }
    __device__ static float2 zero() { return make_float2(0.f, 0.f); }
};
template <>
struct VecW<float, 4> {
    using type = float4;
    template <typename T>
    __device__ static void get(float4 v, T (&a)[4]) { a[0] = (T)v.x; a[1] = (T)v.y; a[2] = (T)v.z; a[3] = (T)v.w; }
    __device__ static float4 put(const float (&a)[4]) { return make_float4(a[0], a[1], a[2], a[3]); }
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <>
struct VecW<double, 2> {
    using type = double2;
    template <typename T>
    __device__ static void get(double2 v, T (&a)[2]) { a[0] = (T)v.x; a[1] = (T)v.y; }
    __device__ static double2 put(const double (&a)[2]) { return make_double2(a[0], a[1]); }
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
};
template <>
struct VecW<__nv_bfloat16, 2> {
    using type = __nv_bfloat162;
    template <typename T>
    __device__ static void get(__nv_bfloat162 v, T (&a)[2]) { a[0] = __low2float(v); a[1] = __high2float(v); }
    __device__ static __nv_bfloat162 put(const float (&a)[2]) { return __floats2bfloat162_rn(a[0], a[1]); }
    __device__ static __nv_bfloat162 zero() { return __floats2bfloat162_rn(0.f, 0.f); }
};
template <>
struct VecW<__nv_bfloat16, 4> {  // four bfloat16 in 8 bytes
    using type = uint2;
    template <typename T>
    __device__ static void get(uint2 v, T (&a)[4]) {
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
        a[0] = __low2float(lo);
        a[1] = __high2float(lo);
        a[2] = __low2float(hi);
        a[3] = __high2float(hi);
    }
    __device__ static uint2 put(const float (&a)[4]) {
        const __nv_bfloat162 lo = __floats2bfloat162_rn(a[0], a[1]), hi = __floats2bfloat162_rn(a[2], a[3]);
        return make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
    __device__ static uint2 zero() { return make_uint2(0u, 0u); }
};

// One velocity's aligned W-element load and, on the warp's edge lanes, the
// element beyond it that an x-shift needs (see pull_pair).
template <typename E, int W, int VX>
struct RowLoad {
    typename VecW<E, W>::type q;
    E edge;
};
template <typename E, int W, int VX>
__device__ __forceinline__ RowLoad<E, W, VX> load_row(const E* __restrict__ src, uint32_t row, bool ok, bool v0,
                                                      bool vlast, int lane) {
    using P = VecW<E, W>;
    RowLoad<E, W, VX> r;
    r.q = ok ? __ldg(reinterpret_cast<const typename P::type*>(src + row)) : P::zero();
    r.edge = E(0);
    if (VX > 0 && lane == 0 && ok && v0) r.edge = __ldg(src + row - 1);
    if (VX < 0 && lane == 31 && ok && vlast) r.edge = __ldg(src + row + W);
    return r;
}
// The W values arriving along the velocity: x-component +1 takes the element
// left of the group from the lane to the left, -1 the element right of it
// from the lane to the right; v0 / vlast: the first / last site has that source.
template <typename E, typename T, int W, int VX>
__device__ __forceinline__ void shift_row(const RowLoad<E, W, VX>& r, bool v0, bool vlast, int lane, T (&gs)[W]) {
    T a[W];
    VecW<E, W>::get(r.q, a);
    if (VX == 0) {
#pragma unroll
        for (int k = 0; k < W; ++k) gs[k] = a[k];
    } else if (VX > 0) {
        T left = __shfl_up_sync(0xffffffffu, a[W - 1], 1);
        if (lane == 0) left = to_compute<T>(r.edge);
        gs[0] = v0 ? left : T(0);
#pragma unroll
        for (int k = 1; k < W; ++k) gs[k] = a[k - 1];
    } else {
        T right = __shfl_down_sync(0xffffffffu, a[0], 1);
        if (lane == 31) right = to_compute<T>(r.edge);
#pragma unroll
        for (int k = 0; k < W - 1; ++k) gs[k] = a[k + 1];
        gs[W - 1] = vlast ? right : T(0);
    }
}

// Sums of the populations arriving at the W sites of a group: f holds one
// array of N per velocity (stride N), or, for the W field, one array pulled
// along every velocity (stride 0) with weight xi_p (weighted).  Every load is
// issued before the first shuffle.  KEEP: also adds each velocity's values to
// gk[p][k] (for the (1 - omega) term).
template <typename E, typename T, int W, bool KEEP, int NG>
__device__ __forceinline__ void gather_row(const E* __restrict__ f, size_t stride, const T (&wt)[3], bool weighted,
                                           const Grid& g, const Site& t, uint32_t s0, bool live, bool v0, bool vlast,
                                           int lane, T (&ps)[W], T (&gk)[NG][W]) {
    const int nxy = g.nx * g.ny;
    RowLoad<E, W, 0> l0[vx_count(0)];
    RowLoad<E, W, 1> lp[vx_count(1)];
    RowLoad<E, W, -1> lm[vx_count(-1)];
    int a = 0, b = 0, c = 0;
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        const int vy = vel(p, 1), vz = vel(p, 2);
        const bool ok = live && (vy == 0 || (vy > 0 ? t.ym : t.yp)) && (vz == 0 || (vz > 0 ? t.zm : t.zp));
        const uint32_t row = (uint32_t)((int)s0 - vy * g.nx - vz * nxy);
        const E* src = f + (size_t)p * stride;
        if (vel(p, 0) == 0) l0[a++] = load_row<E, W, 0>(src, row, ok, true, true, lane);
        else if (vel(p, 0) > 0) lp[b++] = load_row<E, W, 1>(src, row, ok, v0, true, lane);
        else lm[c++] = load_row<E, W, -1>(src, row, ok, true, vlast, lane);
    }
    a = b = c = 0;
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        T v[W];
        if (vel(p, 0) == 0) shift_row<E, T, W, 0>(l0[a++], true, true, lane, v);
        else if (vel(p, 0) > 0) shift_row<E, T, W, 1>(lp[b++], v0, true, lane, v);
        else shift_row<E, T, W, -1>(lm[c++], true, vlast, lane, v);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const T x = weighted ? wt[vclass(p)] * v[k] : v[k];
            ps[k] += x;
            if constexpr (KEEP) gk[p][k] += x;
        }
    }
}

// Sites per thread of the row kernel: four for bfloat16 populations (8-byte
// loads) where the rows take whole groups of four, else two (a tuning knob
// for float populations, set by measurement).
#ifndef LBKS_ROW_WIDTH_F32
#define LBKS_ROW_WIDTH_F32 2
#endif
template <typename TS>
constexpr int row_width_max() {
    return sizeof(TS) == 2 ? 4 : sizeof(TS) == 4 ? LBKS_ROW_WIDTH_F32 : 2;
}

// Resident 256-thread blocks per SM the register allocator must allow: two
// sites per thread hold twice the populations of the one-site kernel, so two
// blocks (1024 sites per SM in flight, as the one-site kernel's four).
#ifndef LBKS_PAIR_MIN_BLOCKS
#define LBKS_PAIR_MIN_BLOCKS 2
#endif
template <typename TS, int NO, bool BATCHED>
constexpr int pair_min_blocks() {
    return LBKS_PAIR_MIN_BLOCKS;
}

// Stream-collide of W x-neighbouring sites per thread (the update of
// k_stream_collide): every population of the group in one aligned load.
template <typename TS, typename T, int NO, bool OM1, bool BATCHED, int W>
__global__ void __launch_bounds__(kThreads, (pair_min_blocks<TS, NO, BATCHED>()))
    k_stream_collide_pair(Grid g, Coef c, RelaxIO io, Scratch sc) {
    constexpr int NP = NO * (NO + 1) / 2;
    using PS = VecW<TS, W>;
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N, NG_ = N / W;
    const size_t y = BATCHED ? sys_id() : 0;
    const TS* __restrict__ fin = static_cast<const TS*>(io.f_in);
    const T* __restrict__ uin = static_cast<const T*>(io.u_in);
    TS* __restrict__ fout = static_cast<TS*>(io.f_out);
    T* __restrict__ psio = static_cast<T*>(io.psi_out);
    const int lane = threadIdx.x & 31;

    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};

    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    // block-uniform trip count: every lane of a warp takes part in the shuffles
    for (uint32_t i0 = blockIdx.x * kThreads; i0 < NG_; i0 += gridDim.x * kThreads) {
        const uint32_t i = i0 + threadIdx.x;
        const bool live = i < NG_;
        const uint32_t s0 = live ? W * i : 0;
        const Site t = decode(g, s0);
        const bool v0 = t.xm;                  // the first site pulls from x - 1
        const bool vlast = t.x + W < g.nx;     // the last site pulls from x + 1
        T vr[W];
#pragma unroll
        for (int k = 0; k < W; ++k) vr[k] = T(0);
        if (live) {
#pragma unroll
            for (int k = 0; k < W; k += 2) {
                const double2 v = __ldg(reinterpret_cast<const double2*>(io.V + y * N + s0 + k));
                vr[k] = (T)v.x;
                vr[k + 1] = (T)v.y;
            }
        }
        T pso[NO][W];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const TS* fj = fin + (y * NO + j) * 19 * N;
            const T* uj = (j > 0 && uin != nullptr) ? uin + (y * (NO > 1 ? NO - 1 : 1) + j - 1) * N : nullptr;
            TS* oj = fout + (y * NO + j) * 19 * N;
            constexpr int NG = OM1 ? 1 : 19;  // omega = 1: only the sums enter the collision
            T gk[NG][W];
#pragma unroll
            for (int p = 0; p < NG; ++p)
#pragma unroll
                for (int k = 0; k < W; ++k) gk[p][k] = T(0);
            T ps[W];
#pragma unroll
            for (int k = 0; k < W; ++k) ps[k] = T(0);
            gather_row<TS, T, W, !OM1, NG>(fj, N, xi, false, g, t, s0, live, v0, vlast, lane, ps, gk);
            if (uj)  // warp-uniform: the W field, weight xi_p
                gather_row<T, T, W, !OM1, NG>(uj, 0, xi, true, g, t, s0, live, v0, vlast, lane, ps, gk);
            T A[W], Bv[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                ps[k] *= sig[j];
                A[k] = om * ps[k];
                Bv[k] = dt * vr[k] * ps[k];
            }
            const T c1 = om1 * sig[j];
            if (live) {
#pragma unroll
                for (int p = 0; p < 19; ++p) {
                    const int q = vclass(p);
                    T e[W];  // T is double for double populations, float for float and bfloat16 ones
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        e[k] = xi[q] * A[k] - chi[q] * Bv[k];
                        if constexpr (!OM1) e[k] += c1 * gk[p][k];
                    }
                    __stcs(reinterpret_cast<typename PS::type*>(oj + (size_t)p * N + s0), PS::put(e));
                }
                *reinterpret_cast<typename VecW<T, W>::type*>(psio + (y * NO + j) * N + s0) = VecW<T, W>::put(ps);
            }
#pragma unroll
            for (int k = 0; k < W; ++k) pso[j][k] = live ? ps[k] : T(0);
        }
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int m = 0; m <= j; ++m) {
                T sum = T(0);
#pragma unroll
                for (int k = 0; k < W; ++k) sum += pso[j][k] * pso[m][k];
                acc[tri(j, m)] += sum;
            }
    }

    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
        store_overlap(tot, NO, c.h, io.S_out + y * NO * NO, io.lambda_out + y * NO * NO, io.sigma_out + y * NO);
}

// More than kMaxOrb orbitals: the same two-site update with one orbital per
// thread (blockIdx.y = system * NO + orbital), the psi epilogue only (the
// overlap runs as its own kernel, as after k_stream_collide_wide).  Every
// population of both sites arrives in one two-element load; the stores are
// two-element streaming stores.
template <typename TS, typename T, bool OM1>
__global__ void __launch_bounds__(kThreads, OM1 ? 4 : 3) k_stream_collide_wide_pair(Grid g, Coef c, RelaxIO io, int NO) {
    using PS = Pack2<TS>;
    using PT = Pack2<T>;
    const int y = (int)blockIdx.y / NO, j = (int)blockIdx.y - y * NO;
    if (g.active && !g.active[y]) return;  // block-uniform
    const uint32_t N = g.N, NH = N >> 1;
    const uint32_t i = blockIdx.x * kThreads + threadIdx.x;
    const bool live = i < NH;
    const uint32_t s0 = live ? 2 * i : 0;
    const int lane = threadIdx.x & 31;
    const size_t oj = (size_t)y * NO + j;
    const TS* __restrict__ fj = static_cast<const TS*>(io.f_in) + oj * 19 * N;
    const T* __restrict__ uj =
        (j > 0 && io.u_in != nullptr) ? static_cast<const T*>(io.u_in) + ((size_t)y * (NO - 1) + j - 1) * N : nullptr;
    TS* __restrict__ out = static_cast<TS*>(io.f_out) + oj * 19 * N;
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const Site t = decode(g, s0);
    const bool x0_has_left = t.xm, x1_has_right = t.x + 2 < g.nx;
    // at omega = 1 only the sums of the arriving populations enter the
    // collision; otherwise every population is kept for the (1 - omega) term
    constexpr int NG = OM1 ? 1 : 19;
    T g0[NG], g1[NG];
#pragma unroll
    for (int p = 0; p < NG; ++p) g0[p] = g1[p] = T(0);
    T ps0 = T(0), ps1 = T(0);
    gather_pair<TS, T, !OM1, NG>(fj, N, xi, false, g, t, s0, live, x0_has_left, x1_has_right, lane, ps0, ps1, g0, g1);
    if (uj)  // block-uniform: the W field, weight xi_p
        gather_pair<T, T, !OM1, NG>(uj, 0, xi, true, g, t, s0, live, x0_has_left, x1_has_right, lane, ps0, ps1, g0,
                                    g1);
    if (!live) return;  // no shuffles below
    T vr0, vr1;
    {
        const double2 v = __ldg(reinterpret_cast<const double2*>(io.V + (size_t)y * N + s0));
        vr0 = (T)v.x;
        vr1 = (T)v.y;
    }
    const T sig = (T)io.sigma_in[oj];
    ps0 *= sig;
    ps1 *= sig;
    const T A0 = om * ps0, B0 = dt * vr0 * ps0, A1 = om * ps1, B1 = dt * vr1 * ps1;
    const T c1 = om1 * sig;
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        const int k = vclass(p);
        const T e0 = xi[k] * A0 - chi[k] * B0, e1 = xi[k] * A1 - chi[k] * B1;
        T o0 = e0, o1 = e1;
        if constexpr (!OM1) {
            o0 += c1 * g0[p];
            o1 += c1 * g1[p];
        }
        __stcs(reinterpret_cast<typename PS::type*>(out + (size_t)p * N + s0), PS::make(o0, o1));
    }
    *reinterpret_cast<typename PT::type*>(static_cast<T*>(io.psi_out) + oj * N + s0) = PT::make(ps0, ps1);
}

}  // namespace lbks
