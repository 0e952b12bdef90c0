// Launchers of the temporally blocked sweep, one per (stencil kind, field type,
// coefficient type); defined in blocked_impl.cuh and instantiated in
// blocked_<stencil>_<type>.cu.
#pragma once
#include "internal.h"

namespace stg {

template <int KIND, typename TF, typename TC>
cudaError_t launch_blocked(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                           cudaStream_t st, long long* launches);
template <int KIND, typename TF, typename TC>
cudaError_t batch_launch_t(const BatchLaunch& bl, cudaStream_t s);
template <int KIND, typename TF, typename TC>
cudaError_t persist_t(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn, void* ws,
                      size_t ws_bytes, const PersistCtl& ctl, cudaStream_t st, long long* launches);

}  // namespace stg

// Explicit instantiation (PREFIX empty) or instantiation declaration (PREFIX extern)
// of the launchers of one (stencil kind, field type, coefficient type); use inside
// namespace stg.
#define STG_BLOCKED_LAUNCHERS(PREFIX, KIND, TF, TC)                                                           \
    PREFIX template cudaError_t launch_blocked<KIND, TF, TC>(const SweepArgs&, void* const[2], int, int,     \
                                                            const BlockedTune&, cudaStream_t, long long*);  \
    PREFIX template cudaError_t batch_launch_t<KIND, TF, TC>(const BatchLaunch&, cudaStream_t);              \
    PREFIX template cudaError_t persist_t<KIND, TF, TC>(const SweepArgs&, void* const[2], int, int,          \
                                                       const BlockedTune&, void*, size_t, const PersistCtl&, \
                                                       cudaStream_t, long long*);

// The (kind, field, coefficient) combinations the library supports.
#define STG_BLOCKED_FOR_EACH_7C(M, P) M(P, K7C, float, float) M(P, K7C, double, double)
#define STG_BLOCKED_FOR_EACH_7V(M, P) \
    M(P, K7V, float, float) M(P, K7V, float, __nv_bfloat16) M(P, K7V, double, double)
#define STG_BLOCKED_FOR_EACH_25V(M, P) \
    M(P, K25V, float, float) M(P, K25V, float, __nv_bfloat16) M(P, K25V, double, double)
