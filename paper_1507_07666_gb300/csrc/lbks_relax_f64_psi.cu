// F64 instantiation of the orbital-storage relaxation (omega = 1); the
// staged stencil's launchers are compiled in lbks_relax_f64_psi_tile.cu.
#include "lbks_psi.cuh"

namespace lbks {
LBKS_PSI_TILE_INST(extern, double)
template cudaError_t launch_relax_psi<double>(int, const Grid&, const Coef&, const RelaxIO&, const Scratch&, int, int,
                                          cudaStream_t);
}  // namespace lbks
