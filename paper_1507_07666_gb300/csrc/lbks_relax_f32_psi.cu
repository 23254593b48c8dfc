// F32 instantiation of the orbital-storage relaxation (omega = 1).
#include "lbks_psi.cuh"

namespace lbks {
template cudaError_t launch_relax_psi<float>(int, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int, int,
                                          cudaStream_t);
}  // namespace lbks
