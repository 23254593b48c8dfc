// FP64 instantiation of the row (two- or four-site) stream-collide kernels, 8 orbitals.
#include "lbks_relax_variants.cuh"

namespace lbks {
template cudaError_t launch_relax_pairs_range<double, double, 8, 8>(int, bool, const Grid&, const Coef&,
                                                                     const RelaxIO&, const Scratch&, int, cudaStream_t);
}  // namespace lbks
