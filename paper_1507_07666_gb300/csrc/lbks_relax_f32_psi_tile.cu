// F32 instantiation of the staged orbital-storage stencil (every tile shape).
#include "lbks_psi.cuh"

namespace lbks {
LBKS_PSI_TILE_INST(, float)
}  // namespace lbks
