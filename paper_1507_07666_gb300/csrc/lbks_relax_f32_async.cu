// FP32 instantiation of the staged (cp.async) stream-collide kernels.
#include "lbks_relax_variants.cuh"

namespace lbks {
template cudaError_t launch_relax_async<float, float>(int, bool, const Grid&, const Coef&, const RelaxIO&,
                                                   const Scratch&, int, cudaStream_t);
}  // namespace lbks
