// Deterministic block and grid reductions (warp shuffles, FP64 partials, the
// last arriving block finishes the grid sum in a fixed order).
#pragma once

#include "lbks_internal.cuh"

namespace lbks {

template <int K>
__device__ __forceinline__ void warp_sum(double (&v)[K]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
}

__device__ __forceinline__ double warp_sum1(double t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    return t;
}

// Sums v over the first NW warps of the block and stores the K totals at dst
// (block-contiguous).  Every thread of the block must call it; warps from NW
// on (a producer warp) contribute nothing.  blockDim.x >= 32 NW.
template <int K, int NW = kThreads / 32>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double* dst) {
    __shared__ double sh[NW][K];
    warp_sum<K>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0 && w < NW) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[w][k] = v[k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < NW; ++i) t += sh[i][k];
        dst[k] = t;
    }
}

// The last block's sum of the K values stored by each of the gridDim.x blocks
// (partial[b*K + k]) into tot[k], in a fixed order.
__device__ __forceinline__ void sum_over_blocks(const double* partial, double* tot, int K) {
    const int nb = (int)gridDim.x;
    if (K >= 64) {
        // many values (overlaps of many orbitals): one value per thread, eight
        // independent partial sums over the blocks in flight at a time, loads
        // coalesced across threads (values are contiguous per block)
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            int b = 0;
            for (; b + 8 <= nb; b += 8) {
#pragma unroll
                for (int i = 0; i < 8; ++i) t[i] += __ldcg(partial + (size_t)(b + i) * K + k);
            }
            for (int i = 0; b < nb; ++b, ++i) t[i] += __ldcg(partial + (size_t)b * K + k);
            tot[k] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
        }
    } else {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int k = w; k < K; k += nw) {
            double t = 0.0;
            for (int b = lane; b < nb; b += 32) t += __ldcg(partial + (size_t)b * K + k);
            t = warp_sum1(t);
            if (lane == 0) tot[k] = t;
        }
    }
}

// After every block stored its K partials at partial[blockIdx.x*K ...], the
// block that arrives last sums them over the grid in a fixed order into the
// shared array `tot` and returns true (in all of its threads); the others
// return false.  The counter is left at zero for the next launch.
template <int K>
__device__ __forceinline__ bool grid_total(const double* partial, unsigned* counter, double* tot) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    sum_over_blocks(partial, tot, K);
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// This block's system in a batched launch, and the system's scratch region.
__device__ __forceinline__ int sys_id() { return (int)blockIdx.y; }
__device__ __forceinline__ bool inactive(const Grid& g) { return g.active && !g.active[blockIdx.y]; }
__device__ __forceinline__ double* sys_partial(const Scratch& sc) {
    return sc.partial + (size_t)blockIdx.y * sc.max_blocks * sc.max_vals;
}
__device__ __forceinline__ unsigned* sys_counter(const Scratch& sc) { return sc.counter + blockIdx.y; }

// Index of pair (j, i), i <= j, in the packed lower triangle.
__host__ __device__ constexpr int tri(int j, int i) { return j * (j + 1) / 2 + i; }

// Grid total of K runtime values (per-system scratch region), fixed order.
__device__ __forceinline__ bool grid_total_rt(const double* partial, unsigned* counter, double* tot, int K) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    sum_over_blocks(partial, tot, K);
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

// Pair index -> (a, b), b <= a, in the packed lower triangle.
__device__ __forceinline__ void tri_pair(int k, int& a, int& b) {
    a = (int)((sqrtf(8.0f * k + 1.0f) - 1.0f) * 0.5f);
    while (tri(a + 1, 0) <= k) ++a;
    while (tri(a, 0) > k) --a;
    b = k - tri(a, 0);
}

// Overlap S = h^3 * (packed pair totals), both triangles; with lam != nullptr
// also Lambda_ab = S_ab / S_bb (a > b, else 0) and sigma_a = 1 / sqrt(S_aa),
// the coupling and normalisation factors of the next relaxation step.
// One thread.
__device__ inline void store_overlap(const double* tot, int NO, double h, double* S, double* lam, double* sigma) {
    const double h3 = h * h * h;
    for (int a = 0; a < NO; ++a)
        for (int b = 0; b <= a; ++b) {
            const double v = h3 * tot[tri(a, b)];
            S[a * NO + b] = v;
            S[b * NO + a] = v;
        }
    if (lam) {
        for (int a = 0; a < NO; ++a) {
            for (int b = 0; b < NO; ++b) lam[a * NO + b] = (b < a) ? S[a * NO + b] / S[b * NO + b] : 0.0;
            sigma[a] = 1.0 / sqrt(S[a * NO + a]);
        }
    }
}

// store_overlap by all threads of the (last) block, with the same arithmetic
// (Lambda_ab = S_ab / S_bb, sigma_a = 1 / sqrt(S_aa)).  Every thread of the
// block must call it.
__device__ inline void store_overlap_block(const double* tot, int NO, double h, double* S, double* lam,
                                           double* sigma) {
    const double h3 = h * h * h;
    for (int i = threadIdx.x; i < NO * NO; i += blockDim.x) {
        const int a = i / NO, b = i - a * NO;
        S[i] = h3 * tot[a >= b ? tri(a, b) : tri(b, a)];
        if (lam) lam[i] = (b < a) ? (h3 * tot[tri(a, b)]) / (h3 * tot[tri(b, b)]) : 0.0;
    }
    if (lam)
        for (int a = threadIdx.x; a < NO; a += blockDim.x) sigma[a] = 1.0 / sqrt(h3 * tot[tri(a, a)]);
}

}  // namespace lbks
