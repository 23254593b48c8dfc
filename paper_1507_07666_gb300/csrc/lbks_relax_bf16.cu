// BF16-storage instantiation of the relaxation kernels: populations stored as
// bfloat16 (half the bytes of FP32), collision arithmetic, orbitals and the
// W field in float, overlaps, density moments and energies in FP64 partials.
#include "lbks_relax.cuh"

namespace lbks {

const PrecisionOps& ops_bf16() { return Ops<__nv_bfloat16, float>::table(); }

namespace {
__global__ void __launch_bounds__(kThreads) k_bf16_to_f32(size_t n, const __nv_bfloat16* __restrict__ src,
                                                          float* __restrict__ dst) {
    for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kThreads)
        dst[i] = __bfloat162float(src[i]);
}
}  // namespace

cudaError_t launch_bf16_to_f32(const void* src, void* dst, size_t n, cudaStream_t st) {
    const size_t need = (n + kThreads - 1) / kThreads;
    const int grid = (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)num_sms() * 8));
    k_bf16_to_f32<<<grid, kThreads, 0, st>>>(n, static_cast<const __nv_bfloat16*>(src), static_cast<float*>(dst));
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lbks
