// FP32 instantiation of the relaxation kernels: float populations and
// collide, FP64 block partials for overlaps, density moments and energies.
#include "lbks_relax.cuh"

namespace lbks {
const PrecisionOps& ops_f32() { return Ops<float, float>::table(); }
}  // namespace lbks
