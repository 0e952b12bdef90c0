// Blocked-sweep kernels and launchers: 25-point variable-coefficient (Listing 3), FP32 field, BF16 coefficients.
#include "blocked_impl.cuh"

namespace stg {
STG_BLOCKED_LAUNCHERS(, K25V, float, __nv_bfloat16)
}  // namespace stg
