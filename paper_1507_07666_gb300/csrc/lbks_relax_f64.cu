// FP64 instantiation of the relaxation kernels (the plain path).
#include "lbks_relax.cuh"

namespace lbks {
const PrecisionOps& ops_f64() { return Ops<double, double>::table(); }
}  // namespace lbks
