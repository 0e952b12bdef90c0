// An allocation-free way to run a batch of grids (stencil_batch_run_noalloc).
//
// Some callers cannot allocate device memory for the batch's workspace: code
// whose device memory is owned by another allocator (a framework's caching
// allocator, a pre-sized arena) and that has no handle on it, or code that must
// not call cudaMalloc in a latency-critical loop because cudaMalloc can
// synchronise the device. For them this file keeps the batch's scratch (grid
// descriptors, the tile list, the dependency flags and the status word) in one
// fixed array in device memory that belongs to the library and lives as long as
// the library is loaded. The grids' own arrays are still the caller's.
#include <vector>

#include "../../include/stencil_gb300.h"
#include "internal.h"

namespace stg {

// Largest batch scratch this entry point can hold. Every GPU that loads the
// library reserves this much device memory until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(4) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up on every
// call, with the caller's device current (cheap; a cached address would outlive a
// reset of the device's context).
static cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// true if p is device memory (or device-mapped host memory) of device dev.
static bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type != cudaMemoryTypeUnregistered && at.device == dev;
}

}  // namespace stg

extern "C" int stencil_batch_run_noalloc(const stencil_t* grids, const int* T, int n, const stencil_tuning* tuning,
                                         void* cuda_stream, int* status_out) {
    using namespace stg;
    if (!grids || !T || n < 1 || !tuning) return STENCIL_EINVAL;
    std::vector<BatchGrid> g(n);
    for (int q = 0; q < n; ++q) {
        if (!grids[q] || T[q] < 0) return STENCIL_EINVAL;
        int rc = grid_batch_view(grids[q], &g[q].a, &g[q].field[0], &g[q].field[1], &g[q].parity);
        if (rc != STENCIL_OK) return rc;
        g[q].T = T[q];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the plan upload waits for the stream, which a capturing stream cannot do
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return STENCIL_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return STENCIL_EINVAL;
    // the scratch is the current device's: the grids' arrays and the stream must be on it too
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STENCIL_ECUDA;
    if (s != nullptr && (cudaStreamGetDevice(s, &sdev) != cudaSuccess || sdev != dev)) return STENCIL_EINVAL;
    for (int q = 0; q < n; ++q)
        if (!on_device(g[q].field[0], dev) || !on_device(g[q].field[1], dev)) return STENCIL_EINVAL;
    BlockedTune tn{tuning->dw, tuning->nf, tuning->warps, 0};
    BatchLaunch bl;
    if (batch_plan(g.data(), n, tn, &bl) != cudaSuccess) return STENCIL_EINVAL;
    if (bl.bytes > NOALLOC_SCRATCH_BYTES) return STENCIL_EINVAL;  // plan larger than the static scratch
    void* ws = nullptr;
    if (scratch_address(&ws) != cudaSuccess) return STENCIL_ECUDA;
    if (batch_upload(g.data(), n, tn, &bl, ws, s) != cudaSuccess) return STENCIL_ECUDA;
    if (batch_launch(bl, s) != cudaSuccess) return STENCIL_ECUDA;
    for (int q = 0; q < n; ++q) grid_set_parity(grids[q], (g[q].parity + T[q]) & 1);
    if (status_out) {
        int v = 0;
        if (cudaStreamSynchronize(s) != cudaSuccess) return STENCIL_ECUDA;
        if (cudaMemcpy(&v, bl.ws + bl.off_counters + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return STENCIL_ECUDA;
        *status_out = v == 0 ? STENCIL_OK : STENCIL_ETIMEOUT;
    }
    return STENCIL_OK;
}
