// Temporally blocked sweep: the non-template entry points (dispatch on stencil
// kind and element types). The kernels and launchers are in blocked_impl.cuh;
// their instantiations are compiled in blocked_<stencil>_<type>.cu, one file per
// supported combination.
#include "blocked_launchers.h"

namespace stg {
STG_BLOCKED_FOR_EACH_7C(STG_BLOCKED_LAUNCHERS, extern)
STG_BLOCKED_FOR_EACH_7V(STG_BLOCKED_LAUNCHERS, extern)
STG_BLOCKED_FOR_EACH_25V(STG_BLOCKED_LAUNCHERS, extern)
}  // namespace stg

#define STG_BLOCKED_MAIN
#include "blocked_impl.cuh"
