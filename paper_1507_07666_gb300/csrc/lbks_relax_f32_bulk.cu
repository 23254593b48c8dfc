// FP32 instantiation of the bulk-copy stream-collide kernel.
#include "lbks_relax_variants.cuh"

namespace lbks {
template cudaError_t launch_relax_bulk<float, float>(int, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int,
                                                     bool, cudaStream_t);
}  // namespace lbks
