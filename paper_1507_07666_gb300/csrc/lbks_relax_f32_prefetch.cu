// FP32 instantiation of the prefetching one-site stream-collide kernels.
#include "lbks_relax_variants.cuh"

namespace lbks {
template cudaError_t launch_relax_prefetch<float, float>(int, bool, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int,
                                     cudaStream_t);
}  // namespace lbks
