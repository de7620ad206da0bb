// Point-query kernels of degree 2 (all storage types, query kinds and knot
// kinds): instantiated here so that the degrees compile in parallel.
#include "eval_kernels.cuh"

namespace mfadvr {
MFADVR_EVAL_DEGREE(2)
}  // namespace mfadvr
