// Render kernels of degree 5 (all storage types, shading on and off,
// uniform and general knots): instantiated here so that the degrees compile
// in parallel.
#include "render_kernels.cuh"

namespace mfadvr {
MFADVR_RENDER_DEGREE(5)
}  // namespace mfadvr
