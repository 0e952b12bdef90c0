// Blocked-sweep kernels and launchers: 7-point constant-coefficient (Listing 1), FP64.
#include "blocked_impl.cuh"

namespace stg {
STG_BLOCKED_LAUNCHERS(, K7C, double, double)
}  // namespace stg
