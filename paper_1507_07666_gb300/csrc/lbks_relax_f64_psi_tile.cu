// F64 instantiation of the staged orbital-storage stencil (every tile shape).
#include "lbks_psi.cuh"

namespace lbks {
LBKS_PSI_TILE_INST(, double)
}  // namespace lbks
