// Tensor-memory-accelerator copies and mbarriers (inline PTX, sm_90 and later).
//
// A copy `cp.async.bulk.tensor` moves one box of a tensor map (a 3D view of a
// padded array) into shared memory and completes its bytes on an mbarrier; the
// innermost coordinate of a box times the element size must be a multiple of 16
// bytes, which the callers check on the host. Every wait here is bounded: one
// that runs out sets *status (when given) and returns false.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace stg {

constexpr unsigned TMA_WAIT_POLLS = 1u << 22;  // with the back-off below: > 0.25 s

__device__ __forceinline__ uint32_t tma_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
// Makes the initialisations above visible to the other threads and to the copy engine.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival that also announces `bytes` of copies completing on this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
// Waits until the phase of parity `parity` has completed (bounded).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int* status) {
    if (mbar_test(a, parity)) return true;
    for (unsigned n = 0; n < TMA_WAIT_POLLS; ++n) {
        if (n >= 64) __nanosleep(64);
        if (mbar_test(a, parity)) return true;
    }
    if (status) atomicCAS(status, 0, 1);
    return false;
}

// Orders this thread's earlier generic-proxy view of global memory (values other
// CTAs published and this thread acquired) before its later tensor copies.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

// One box of a 3D tensor map at element coordinates (x, y, z) into shared memory.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

}  // namespace stg
