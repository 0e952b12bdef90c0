// Blocked-sweep kernels and launchers: 7-point variable-coefficient (Listing 2), FP32.
#include "blocked_impl.cuh"

namespace stg {
STG_BLOCKED_LAUNCHERS(, K7V, float, float)
}  // namespace stg
