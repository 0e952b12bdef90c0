// Blocked-sweep kernels and launchers: 25-point variable-coefficient (Listing 3), FP64.
#include "blocked_impl.cuh"

namespace stg {
STG_BLOCKED_LAUNCHERS(, K25V, double, double)
}  // namespace stg
