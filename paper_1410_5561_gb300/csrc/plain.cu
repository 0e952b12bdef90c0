// Plain one-step-per-pass streaming sweep (the analog of the paper's spatially
// blocked baseline, Section IV, "Spt. Blk."): every launch reads u_t once and
// writes u_{t+1} once, so it moves 2*s_f + n_c*s_c bytes per LUP at best.
//
// Thread mapping: a warp covers 32 vectors of V = 16/sizeof(field) consecutive
// x values (128-bit accesses); a CTA stacks BY warps along y; each thread walks
// a chunk of z planes (sweep_column.cuh: register ring of the column's planes,
// neighbours through L1/L2, coefficients with evict-first loads). The number
// of z chunks is chosen from the kernel's occupancy so that the CTAs fill
// whole waves of the GPU.
#include <mutex>

#include "internal.h"
#include "sweep_column.cuh"

namespace stg {

// Per stencil and element types: planes loaded ahead (PF) and the CTAs per SM the register
// allocation must allow (MINB), chosen by measurement on GB300. The constant-coefficient
// sweep has a single HBM stream per thread and wants loads in flight; the variable ones
// issue n_c + 1 streaming loads per plane already and are limited by the registers their
// coefficient vectors take (the 25-point BF16 / FP64 sweeps double their speed at 2 CTAs).
template <int KIND, typename TF, typename TC> struct PlainCfg { static constexpr int PF = 1, MINB = 1; };
template <typename TF> struct PlainCfg<K7C, TF, TF> { static constexpr int PF = 3, MINB = 5; };
template <> struct PlainCfg<K7V, float, float> { static constexpr int PF = 0, MINB = 3; };
template <> struct PlainCfg<K7V, double, double> { static constexpr int PF = 0, MINB = 3; };
template <> struct PlainCfg<K25V, float, float> { static constexpr int PF = 0, MINB = 1; };
template <> struct PlainCfg<K25V, float, __nv_bfloat16> { static constexpr int PF = 1, MINB = 2; };
template <> struct PlainCfg<K25V, double, double> { static constexpr int PF = 1, MINB = 2; };

template <int KIND, typename TF, typename TC, int BY, int PF>
__global__ void __launch_bounds__(32 * BY, (PlainCfg<KIND, TF, TC>::MINB))
plain_sweep_kernel(Layout L, const TF* __restrict__ src, TF* __restrict__ dst, CoefPtrs<TC> C,
                   TF c0, TF c1, int zchunk) {
    constexpr int V = 16 / sizeof(TF);
    const int i0 = (blockIdx.x * 32 + threadIdx.x) * V;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zchunk;
    const int k1 = min(L.nz, k0 + zchunk);
    if (k0 >= k1) return;
    sweep_column<KIND, TF, TC, PF, true>(L, src, dst, C, c0, c1, i0, j, k0, k1);
}

// The plain sweep with every load of a plane copied D planes ahead into per-thread shared-memory
// slots (ColumnAsync): the copies in flight hold shared memory, not registers.
template <int KIND, typename TF, typename TC, int BY, int D>
__global__ void __launch_bounds__(32 * BY) plain_async_kernel(Layout L, const TF* __restrict__ src, TF* __restrict__ dst,
                                                              CoefPtrs<TC> C, TF c0, TF c1, int zchunk) {
    constexpr int V = 16 / sizeof(TF);
    using Col = ColumnAsync<KIND, TF, TC, true, D>;
    extern __shared__ __align__(16) unsigned char plain_smem[];
    const int i0 = (blockIdx.x * 32 + threadIdx.x) * V;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zchunk;
    const int k1 = min(L.nz, k0 + zchunk);
    if (k0 >= k1) return;
    constexpr int NT = 32 * BY;
    const int tid = (int)(threadIdx.y * 32 + threadIdx.x);
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(plain_smem);
    Col col;
    col.begin(L, src, C, i0, j, k0, k1, s0 + (uint32_t)(tid * 16), (uint32_t)(NT * 16),
              s0 + (uint32_t)(D * Col::SF * NT * 16 + tid * Col::CB), (uint32_t)(NT * Col::CB));
    for (int k = k0; k < k1; ++k) col.plane(L, src, dst, C, c0, c1, i0, k);
}

// Resident CTAs per SM of one kernel instantiation times the SM count, per device
// (one cache per instantiation: the template arguments name the kernel).
template <int KIND, typename TF, typename TC, typename KernelT>
static int plain_slots(KernelT kernel, int threads, size_t smem = 0) {
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (cached[dev] == 0) {
        int sms = 0, per = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) return 0;
        cached[dev] = sms * (per > 0 ? per : 1);
    }
    return cached[dev];
}

// z chunks per column: minimise (waves of CTAs) x (planes per chunk + ring warm-up),
// with chunks of at least 16 planes.
static int plain_chunks(long long xy, int nz, int R, int slots) {
    if (slots <= 0) slots = 8 * 152;
    int best = 1;
    long long best_cost = -1;
    const int maxchunks = (nz + 15) / 16 > 0 ? (nz + 15) / 16 : 1;
    for (int n = 1; n <= maxchunks; ++n) {
        const int zc = (nz + n - 1) / n;
        const int nn = (nz + zc - 1) / zc;
        const long long waves = (xy * nn + slots - 1) / slots;
        const long long cost = waves * (zc + 2 * R);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = nn;
        }
    }
    return best;
}

template <int KIND, typename TF, typename TC>
static cudaError_t launch_plain(const SweepArgs& a, const void* src, void* dst, cudaStream_t s) {
    constexpr int BY = 8;
    constexpr int PF = PlainCfg<KIND, TF, TC>::PF;
    constexpr int V = 16 / sizeof(TF);
    const Layout& L = a.L;
    if (L.nx == 0 || L.ny == 0 || L.nz == 0) return cudaSuccess;
    CoefPtrs<TC> C{};
    for (int m = 0; m < KindTraits<KIND>::NC; ++m) C.c[m] = static_cast<const TC*>(a.coef[m]);
    dim3 block(32, BY);
    unsigned gx = (unsigned)((L.nx + 32 * V - 1) / (32 * V));
    unsigned gy = (unsigned)((L.ny + BY - 1) / BY);
    if (a.plain_prefetch == 2) {
        constexpr int D = 2;
        using Col = ColumnAsync<KIND, TF, TC, true, D>;
        auto kernel = plain_async_kernel<KIND, TF, TC, BY, D>;
        const size_t smem = (size_t)D * 32 * BY * (Col::SF * 16 + KindTraits<KIND>::NC * Col::CB);
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int nchunks = plain_chunks((long long)gx * gy, L.nz, KindTraits<KIND>::R,
                                         plain_slots<KIND, TF, TC>(kernel, 32 * BY, smem));
        const int zchunk = (L.nz + nchunks - 1) / nchunks;
        kernel<<<dim3(gx, gy, (unsigned)nchunks), block, smem, s>>>(L, static_cast<const TF*>(src), static_cast<TF*>(dst),
                                                                     C, (TF)a.c0, (TF)a.c1, zchunk);
        return cudaGetLastError();
    }
    auto kernel = plain_sweep_kernel<KIND, TF, TC, BY, PF>;
    const int nchunks = plain_chunks((long long)gx * gy, L.nz, KindTraits<KIND>::R, plain_slots<KIND, TF, TC>(kernel, 32 * BY));
    const int zchunk = (L.nz + nchunks - 1) / nchunks;
    dim3 grid(gx, gy, (unsigned)nchunks);
    kernel<<<grid, block, 0, s>>>(L, static_cast<const TF*>(src), static_cast<TF*>(dst), C, (TF)a.c0, (TF)a.c1,
                                  zchunk);
    return cudaGetLastError();
}

cudaError_t plain_step(const SweepArgs& a, const void* src, void* dst, cudaStream_t s) {
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) return launch_plain<K7C, float, float>(a, src, dst, s);
            if (a.fdt == DT_F64) return launch_plain<K7C, double, double>(a, src, dst, s);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) return launch_plain<K7V, float, float>(a, src, dst, s);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_plain<K7V, float, __nv_bfloat16>(a, src, dst, s);
            if (a.fdt == DT_F64 && a.cdt == DT_F64) return launch_plain<K7V, double, double>(a, src, dst, s);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) return launch_plain<K25V, float, float>(a, src, dst, s);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_plain<K25V, float, __nv_bfloat16>(a, src, dst, s);
            if (a.fdt == DT_F64 && a.cdt == DT_F64) return launch_plain<K25V, double, double>(a, src, dst, s);
            break;
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ fill
template <typename T>
__global__ void fill_kernel(T* __restrict__ p, size_t n, T v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ------------------------------------------------------------------ interior copy
// Dense (nz, ny, nx) rows <-> the padded layout's interior rows. Either side may be device
// memory or page-locked host memory mapped into the device's address space (read and written
// over the host link by the kernel's own loads and stores, which keeps many 16-byte accesses
// in flight: faster than a pitched DMA of short rows). One CTA per row, 16-byte accesses when
// both row starts and the row length allow, else elementwise.
__global__ void copy_rows_kernel(const char* __restrict__ src, char* __restrict__ dst, Layout L, int eb,
                                 int to_padded) {
    const size_t rows = (size_t)L.ny * L.nz;
    const size_t rb = (size_t)L.nx * eb;
    for (size_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const int y = (int)(r % (size_t)L.ny), z = (int)(r / (size_t)L.ny);
        const size_t pad = L.at(0, y, z) * (size_t)eb;
        const char* a = src + (to_padded ? r * rb : pad);
        char* b = dst + (to_padded ? pad : r * rb);
        if ((((uintptr_t)a | (uintptr_t)b | rb) & 15u) == 0) {
            for (size_t i = threadIdx.x; i < rb / 16; i += blockDim.x)
                reinterpret_cast<uint4*>(b)[i] = reinterpret_cast<const uint4*>(a)[i];
        } else {
            for (size_t i = threadIdx.x; i < rb; i += blockDim.x) b[i] = a[i];
        }
    }
}

cudaError_t copy_rows(const Layout& L, int eb, const void* src, void* dst, bool to_padded, cudaStream_t s) {
    const size_t rows = (size_t)L.ny * L.nz;
    if (rows == 0 || L.nx == 0) return cudaSuccess;
    unsigned blocks = rows < (size_t)152 * 16 ? (unsigned)rows : 152u * 16u;
    copy_rows_kernel<<<blocks, 256, 0, s>>>(static_cast<const char*>(src), static_cast<char*>(dst), L, eb,
                                            to_padded ? 1 : 0);
    return cudaGetLastError();
}

// Dense copy by the SMs' own loads and stores, with few CTAs: each thread keeps DC_U
// independent 16-byte loads in flight, so a handful of SMs can stream host memory over the
// link while the other SMs run a sweep.
constexpr int DC_U = 8;
__global__ void __launch_bounds__(1024) dense_copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                          size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (DC_U - 1) * stride < n; i += DC_U * stride) {
        uint4 v[DC_U];
#pragma unroll
        for (int u = 0; u < DC_U; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < DC_U; ++u) dst[i + u * stride] = v[u];
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

cudaError_t dense_copy(void* dst, const void* src, size_t bytes, int ctas, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    dense_copy_kernel<<<(unsigned)ctas, 1024, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst),
                                                      bytes / 16);
    return cudaGetLastError();
}

cudaError_t fill_value(void* p, size_t n, int dt, double v, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (blocks > 152u * 16u) blocks = 152u * 16u;
    if (dt == DT_F32) fill_kernel<float><<<blocks, 256, 0, s>>>((float*)p, n, (float)v);
    else if (dt == DT_F64) fill_kernel<double><<<blocks, 256, 0, s>>>((double*)p, n, v);
    else fill_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((__nv_bfloat16*)p, n, __double2bfloat16(v));
    return cudaGetLastError();
}

}  // namespace stg
