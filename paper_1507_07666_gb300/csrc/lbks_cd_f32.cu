// FP32 instantiation of the concurrent-dynamics step (FP64 overlap sums).
#include "lbks_cd.cuh"

namespace lbks {
template cudaError_t launch_cd_step<float>(int, const Grid&, const CdCoef&, const CdIO&, const Scratch&, int,
                                           cudaStream_t);
template cudaError_t launch_cd_overlap<float>(int, const Grid&, const void*, double, double*, double*,
                                              const Scratch&, int, cudaStream_t);
}  // namespace lbks
