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

// Sums v over the block and stores the K totals at dst (block-contiguous).
// Every thread of the block must call it.  blockDim.x == kThreads.
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double* dst) {
    __shared__ double sh[kThreads / 32][K];
    warp_sum<K>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[w][k] = v[k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) t += sh[i][k];
        dst[k] = t;
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
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = w; k < K; k += nw) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(partial + (size_t)b * K + k);
        t = warp_sum1(t);
        if (lane == 0) tot[k] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
    return true;
}

}  // namespace lbks
