// Wavefront temporal blocking through L2: the thread group of Section II-A
// (several threads sharing one cache block, the paper's nWD variants) spread
// over the whole GPU, with the 129 MB L2 as the shared cache block.
//
// One launch advances the grid by h time steps (a pass). The grid is cut into
// xy tiles (32 vectors of x by BY rows, one CTA's worth) and z chunks of ZC
// planes. Unit (l, c, q) computes time level l of the pass (u_{t+l+1} from
// u_{t+l}) on chunk c of tile q with the plain sweep's column update
// (sweep_column.cuh), so every value is bit-identical to the plain sweep. Level
// l trails level l-1 by LAG chunks: the units are listed in wave order
// w = c + LAG * l (higher levels first within a wave), and a CTA pops the next
// unit from an atomic counter. Unit (l, c, q) waits (bounded) for the units
// (l-1, c', q') with c' in c-1..c+1 and q' in the 3 x 3 tiles around q, which
// wrote every value it reads (R <= ZC and R <= BY) and which have finished
// reading every cell it overwrites (level l writes the array that holds
// u_{t+l-1}). Those units have smaller indices, so the smallest unfinished unit
// can always run: no launch can deadlock, whatever the number of resident CTAs.
//
// HBM traffic per pass: u_t and the coefficients read once, u_{t+h} written
// once; the intermediate levels' values and the coefficient planes are read
// again from L2 by the next level a few chunks later (written-back
// intermediates add s_f per level). The L2 holds about (LAG + 1) ZC planes of
// every array while a pass runs.
#include <type_traits>

#include "adjoint_column.cuh"
#include "internal.h"
#include "sweep_column.cuh"

namespace stg {

constexpr int WAVE_MAXW = 1024;  // waves per pass
constexpr int WAVE_MAXLV = 64;   // time levels per pass

template <typename TF, typename TC>
struct WaveArgs {
    Layout L;
    TF* lv[WAVE_MAXLV + 1];  // level l reads lv[l] and writes lv[l + 1]
    CoefPtrs<TC> C;
    TF c0, c1;
    int h, lag;     // levels in this pass; chunks between consecutive levels
    int zc, nch;    // planes per chunk; chunks
    int ntx, nty;   // xy tiles
    int nitems;
    int* status;    // sticky: 1 once a dependency wait gave up
    int* never;     // a flag no unit sets (the stall hook waits on it)
    int* head;      // next unit to pop
    int* flags;     // [h][nch][nty][ntx]: 1 when the unit has finished
    unsigned spin_limit;
    int stall_item;
    int nwaves;
    int wbase[WAVE_MAXW + 1];  // first unit of each wave
};

__device__ __forceinline__ void wv_st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// Levels active in wave w: c = w - lag * l in [0, nch).
__host__ __device__ inline void wave_levels(int w, int h, int lag, int nch, int& lmin, int& lmax) {
    lmax = w / lag;
    if (lmax > h - 1) lmax = h - 1;
    const int d = w - nch + 1;
    lmin = d <= 0 ? 0 : (d + lag - 1) / lag;
}

// OP = 0: the forward step (sweep_column); OP = 1: the adjoint's transposed step (lambda_column).
template <int KIND, typename TF, typename TC, int BY, int PF, int OP>
__global__ void __launch_bounds__(32 * BY, 1) wave_kernel(const __grid_constant__ WaveArgs<TF, TC> A) {
    constexpr int V = 16 / sizeof(TF);
    __shared__ int s_item[2];
    const int ntiles = A.ntx * A.nty;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_item[0] = atomicAdd(A.head, 1);
    __syncthreads();
    for (int buf = 0;; buf ^= 1) {
        const int i = s_item[buf];
        if (i >= A.nitems) break;
        // unit i: wave, level, chunk, tile
        int lo = 0, hi = A.nwaves - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.wbase[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int w = lo, o = i - A.wbase[lo];
        int lmin, lmax;
        wave_levels(w, A.h, A.lag, A.nch, lmin, lmax);
        const int l = lmax - o / ntiles, q = o % ntiles;
        const int c = w - A.lag * l;
        const int qx = q % A.ntx, qy = q / A.ntx;
        if (threadIdx.y == 0) {
            // pop the next unit now, so its index is ready when this one ends
            if (threadIdx.x == 0) s_item[buf ^ 1] = atomicAdd(A.head, 1);
            // lane d < 27 waits for unit (l-1, c + dc, tile (qx + dx, qy + dy)); lane 27 for the stall hook
            const int lane = threadIdx.x;
            const int* flag = nullptr;
            if (l > 0 && lane < 27) {
                const int dc = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
                const int cc = c + dc, yy = qy + dy, xx = qx + dx;
                if (cc >= 0 && cc < A.nch && yy >= 0 && yy < A.nty && xx >= 0 && xx < A.ntx)
                    flag = A.flags + (((size_t)(l - 1) * A.nch + cc) * A.nty + yy) * A.ntx + xx;
            }
            if (lane == 27 && i == A.stall_item) flag = A.never;
            if (flag) {
                unsigned n = 0;
                while (*(volatile const int*)flag == 0) {
                    if (*(volatile const int*)A.status != 0) break;
                    if (++n > A.spin_limit) {
                        atomicCAS(A.status, 0, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncwarp();
            // one converged fence for the warp: each lane that saw a flag set orders the
            // values published before it ahead of this SM's loads below
            if (l > 0 || i == A.stall_item) __threadfence();
        }
        __syncthreads();
        const int i0 = (qx * 32 + (int)threadIdx.x) * V;
        const int j = qy * BY + (int)threadIdx.y;
        const int k0 = c * A.zc;
        const int k1 = min(A.L.nz, k0 + A.zc);
        if (i0 < A.L.nx && j < A.L.ny) {
            const TF* src = A.lv[l];
            TF* dst = A.lv[l + 1];
            if constexpr (OP == 1)
                lambda_column<KIND, TF, TC, true>(A.L, src, dst, A.C, i0, j, k0, k1);
            else if (l == A.h - 1)  // the last level's coefficients are not read again in this pass
                sweep_column<KIND, TF, TC, PF, true, true>(A.L, src, dst, A.C, A.c0, A.c1, i0, j, k0, k1);
            else
                sweep_column<KIND, TF, TC, PF, false, true>(A.L, src, dst, A.C, A.c0, A.c1, i0, j, k0, k1);
        }
        __syncthreads();  // every thread's stores of the unit precede thread 0's fence and flag
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            wv_st_release(A.flags + (((size_t)l * A.nch + c) * A.nty + qy) * A.ntx + qx, 1);
        }
    }
}

// Stream form, used when every (level, tile) pair can hold a resident CTA: CTA
// (l, q) walks all z chunks of level l on tile q in order, keeping its column's
// plane ring in registers across chunks (no per-chunk warm-up). Before chunk c
// it waits until the level-(l-1) CTAs of the 3 x 3 tiles around q have finished
// chunks <= c + 1 (the same dependencies as the unit form) and, to keep the L2
// band short, until the level-(l+1) CTA of its own tile has finished chunk
// c - LEAD. Progress counters are monotonic per (level, tile). No wait can
// deadlock while all CTAs are resident: a CTA at the lowest chunk among those
// not finished has its lower level at least two chunks ahead or can let it
// advance, since a lower level may lead by LEAD >= 2 chunks.
constexpr int WAVE_LEAD = 3;

// All chunks of one (level, tile) stream; COEF_STREAM for the last level, whose
// coefficient loads are evict-first (no later level of the pass reads them).
template <int KIND, typename TF, typename TC, int BY, bool COEF_STREAM, int CP, int OP>
__device__ __forceinline__ void wave_stream(const WaveArgs<TF, TC>& A, int l, int q) {
    constexpr int V = 16 / sizeof(TF);
    extern __shared__ __align__(16) unsigned char wave_smem[];
    const int ntiles = A.ntx * A.nty;
    const int qx = q % A.ntx, qy = q / A.ntx;
    const int i0 = (qx * 32 + (int)threadIdx.x) * V;
    const int j = qy * BY + (int)threadIdx.y;
    const bool act = i0 < A.L.nx && j < A.L.ny;
    const TF* src = A.lv[l];
    TF* dst = A.lv[l + 1];
    int* prog = A.flags;  // [h][ntiles]: chunks finished
    const bool last = l == A.h - 1;
    // CP = 0: loads issued per plane; CP > 0: every load of a plane copied CP planes ahead into this
    // thread's shared-memory slots (field vectors first, then the coefficient vectors)
    using Col = std::conditional_t<(CP > 0), ColumnAsync<KIND, TF, TC, COEF_STREAM, (CP > 0 ? CP : 1)>,
                                   Column<KIND, TF, TC, 0, COEF_STREAM, true, 0>>;
    Col col;
    constexpr int NT = 32 * BY;
    constexpr int CB = (int)sizeof(Vec<TC, V>);
    constexpr int SF = ColumnAsync<KIND, TF, TC, COEF_STREAM, 1>::SF;
    const int tid = (int)(threadIdx.y * 32 + threadIdx.x);
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(wave_smem);
    const uint32_t fslot = s0 + (uint32_t)(tid * 16), fstep = (uint32_t)(NT * 16);
    const uint32_t cslot = s0 + (uint32_t)((CP > 0 ? CP : 1) * SF * NT * 16 + tid * CB), cstep = (uint32_t)(NT * CB);
    for (int c = 0; c < A.nch; ++c) {
        if (threadIdx.y == 0) {
            const int lane = threadIdx.x;
            const int* flag = nullptr;
            int need = 0;
            if (l > 0 && lane < 9) {  // level l-1 of the 3 x 3 tiles: chunks <= c + 1 finished
                const int yy = qy + lane / 3 - 1, xx = qx + lane % 3 - 1;
                if (yy >= 0 && yy < A.nty && xx >= 0 && xx < A.ntx) {
                    flag = prog + (size_t)(l - 1) * ntiles + (size_t)yy * A.ntx + xx;
                    need = c + 2 < A.nch ? c + 2 : A.nch;
                }
            }
            if (lane == 9 && !last && c - WAVE_LEAD > 0) {  // level l+1 of this tile: chunk c - LEAD finished
                flag = prog + (size_t)(l + 1) * ntiles + q;
                need = c - WAVE_LEAD;
            }
            if (lane == 10 && c == 0 && (int)blockIdx.x == A.stall_item) {
                flag = A.never;
                need = 1;
            }
            if (flag) {
                unsigned n = 0;
                while (*(volatile const int*)flag < need) {
                    if (*(volatile const int*)A.status != 0) break;
                    if (++n > A.spin_limit) {
                        atomicCAS(A.status, 0, 1);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __syncwarp();
            __threadfence();  // values published before the counters precede this SM's loads
        }
        __syncthreads();
        const int k0 = c * A.zc;
        const int k1 = min(A.L.nz, k0 + A.zc);
        if (act) {
            if constexpr (OP == 1) {
                lambda_column<KIND, TF, TC, true>(A.L, src, dst, A.C, i0, j, k0, k1);
            } else {
                if (c == 0) {
                    if constexpr (CP > 0) col.begin(A.L, src, A.C, i0, j, 0, A.L.nz, fslot, fstep, cslot, cstep);
                    else col.begin(A.L, src, i0, j, 0, A.L.nz);
                }
                for (int k = k0; k < k1; ++k) col.plane(A.L, src, dst, A.C, A.c0, A.c1, i0, k);
            }
        }
        __syncthreads();  // every thread's stores of the chunk precede thread 0's fence and counter
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            wv_st_release(prog + (size_t)l * ntiles + q, c + 1);
        }
    }
}

template <int KIND, typename TF, typename TC, int BY, int CP, int OP>
__global__ void __launch_bounds__(32 * BY, 1) wave_stream_kernel(const __grid_constant__ WaveArgs<TF, TC> A) {
    const int ntiles = A.ntx * A.nty;
    const int l = (int)blockIdx.x / ntiles, q = (int)blockIdx.x % ntiles;
    if (l == A.h - 1) wave_stream<KIND, TF, TC, BY, true, CP, OP>(A, l, q);
    else wave_stream<KIND, TF, TC, BY, false, CP, OP>(A, l, q);
}

// ------------------------------------------------------------------- host side

template <int KIND, typename TF, typename TC> struct WaveCfg { static constexpr int PF = 1; };
template <typename TF> struct WaveCfg<K7C, TF, TF> { static constexpr int PF = 3; };
template <> struct WaveCfg<K25V, float, float> { static constexpr int PF = 0; };

// Geometry of one pass: chunks, tiles, waves and units; false if the tuning is
// malformed for this grid.
struct WaveShape {
    int h, lag, zc, nch, ntx, nty, nwaves, nitems, cp;
    size_t flag_words;
};

static bool wave_shape(const SweepArgs& a, int h, int zc, int by, int lag, WaveShape* s, int cp = 0) {
    const int R = kind_radius(a.kind);
    const int V = 16 / dtype_bytes(a.fdt);
    if (h < 1 || h > WAVE_MAXLV || zc < R || zc < 1 || by < R || lag < 2) return false;
    if (by != 4 && by != 8 && by != 16) return false;
    s->h = h;
    s->lag = lag;
    s->cp = cp;
    s->zc = zc;
    s->nch = (a.L.nz + zc - 1) / zc;
    s->ntx = (a.L.nx + 32 * V - 1) / (32 * V);
    s->nty = (a.L.ny + by - 1) / by;
    s->nwaves = s->nch + lag * (h - 1);
    if (s->nwaves > WAVE_MAXW) return false;
    long long units = (long long)h * s->nch * s->ntx * s->nty;
    if (units > (1LL << 30)) return false;
    s->nitems = (int)units;
    s->flag_words = (size_t)units;
    return true;
}

template <int KIND, typename TF, typename TC, int BY, int OP>
static cudaError_t wave_pass(const SweepArgs& a, void* const* lvl, const WaveShape& sh, int* ws,
                             const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    constexpr int PF = WaveCfg<KIND, TF, TC>::PF;
    auto kfn = wave_kernel<KIND, TF, TC, BY, PF, OP>;
    WaveArgs<TF, TC> A{};
    A.L = a.L;
    for (int l = 0; l <= sh.h; ++l) A.lv[l] = static_cast<TF*>(lvl[l]);
    for (int m = 0; m < kind_ncoef(a.kind); ++m) A.C.c[m] = static_cast<const TC*>(a.coef[m]);
    A.c0 = (TF)a.c0;
    A.c1 = (TF)a.c1;
    A.h = sh.h;
    A.lag = sh.lag;
    A.zc = sh.zc;
    A.nch = sh.nch;
    A.ntx = sh.ntx;
    A.nty = sh.nty;
    A.nitems = sh.nitems;
    A.status = ws + WAVE_WS_STATUS;
    A.never = ws + WAVE_WS_NEVER;
    A.head = ws + WAVE_WS_HEAD;
    A.flags = ws + WAVE_WS_FLAGS;
    A.spin_limit = ctl.spin_limit;
    A.stall_item = ctl.stall_item;
    A.nwaves = sh.nwaves;
    const int ntiles = sh.ntx * sh.nty;
    int n = 0;
    for (int w = 0; w < sh.nwaves; ++w) {
        A.wbase[w] = n;
        int lmin, lmax;
        wave_levels(w, sh.h, sh.lag, sh.nch, lmin, lmax);
        if (lmax >= lmin) n += (lmax - lmin + 1) * ntiles;
    }
    A.wbase[sh.nwaves] = n;
    if (n != sh.nitems) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, 32 * BY, 0))) return e;
    long long ctas = (long long)(per > 0 ? per : 1) * sms;
    if (ctas > sh.nitems) ctas = sh.nitems;
    // the never-set flag, the unit counter and the completion flags start at 0; the status is kept
    if ((e = cudaMemsetAsync(ws + WAVE_WS_NEVER, 0, sizeof(int) * (WAVE_WS_FLAGS - WAVE_WS_NEVER + sh.flag_words),
                             st)))
        return e;
    kfn<<<(unsigned)ctas, dim3(32, BY), 0, st>>>(A);
    if ((e = cudaGetLastError())) return e;
    if (launches) ++*launches;
    return cudaSuccess;
}

// Stream form of one pass (see wave_stream_kernel): cudaErrorNotReady if the
// (level, tile) pairs outnumber the CTAs that can be resident at once.
template <int KIND, typename TF, typename TC, int BY, int CP, int OP>
static cudaError_t wave_pass_stream(const SweepArgs& a, void* const* lvl, const WaveShape& sh, int* ws,
                                    const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    auto kfn = wave_stream_kernel<KIND, TF, TC, BY, CP, OP>;
    constexpr int V = 16 / sizeof(TF);
    constexpr int SF = ColumnAsync<KIND, TF, TC, false, 1>::SF;
    const size_t smem = (size_t)CP * 32 * BY * (SF * 16 + KindTraits<KIND>::NC * sizeof(Vec<TC, V>));
    if constexpr (CP > 0) {
        int dev0 = 0, optin = 0;
        cudaGetDevice(&dev0);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev0);
        if (smem > (size_t)optin || sh.zc < KindTraits<KIND>::R + CP) return cudaErrorNotReady;
    }
    const int ntiles = sh.ntx * sh.nty;
    const long long streams = (long long)sh.h * ntiles;
    int dev = 0, sms = 0, per = 0;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, 32 * BY, smem))) return e;
    if (streams > (long long)per * sms) return cudaErrorNotReady;
    WaveArgs<TF, TC> A{};
    A.L = a.L;
    for (int l = 0; l <= sh.h; ++l) A.lv[l] = static_cast<TF*>(lvl[l]);
    for (int m = 0; m < kind_ncoef(a.kind); ++m) A.C.c[m] = static_cast<const TC*>(a.coef[m]);
    A.c0 = (TF)a.c0;
    A.c1 = (TF)a.c1;
    A.h = sh.h;
    A.lag = sh.lag;
    A.zc = sh.zc;
    A.nch = sh.nch;
    A.ntx = sh.ntx;
    A.nty = sh.nty;
    A.nitems = (int)streams;
    A.status = ws + WAVE_WS_STATUS;
    A.never = ws + WAVE_WS_NEVER;
    A.head = ws + WAVE_WS_HEAD;
    A.flags = ws + WAVE_WS_FLAGS;
    A.spin_limit = ctl.spin_limit;
    A.stall_item = ctl.stall_item;
    if ((e = cudaMemsetAsync(ws + WAVE_WS_NEVER, 0, sizeof(int) * (WAVE_WS_FLAGS - WAVE_WS_NEVER + (size_t)streams),
                             st)))
        return e;
    kfn<<<(unsigned)streams, dim3(32, BY), smem, st>>>(A);
    if ((e = cudaGetLastError())) return e;
    if (launches) ++*launches;
    return cudaSuccess;
}

template <int KIND, typename TF, typename TC, int BY, int OP = 0>
static cudaError_t wave_pass_any(const SweepArgs& a, void* const* lvl, const WaveShape& sh, int* ws,
                                 const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    cudaError_t e = cudaErrorNotReady;
    if (OP == 0 && sh.cp == 2) e = wave_pass_stream<KIND, TF, TC, BY, (OP == 0 ? 2 : 0), OP>(a, lvl, sh, ws, ctl, st, launches);
    if (e == cudaErrorNotReady) e = wave_pass_stream<KIND, TF, TC, BY, 0, OP>(a, lvl, sh, ws, ctl, st, launches);
    if (e != cudaErrorNotReady) return e;
    return wave_pass<KIND, TF, TC, BY, OP>(a, lvl, sh, ws, ctl, st, launches);
}

template <int KIND, typename TF, typename TC>
static cudaError_t wave_run_t(const SweepArgs& a, void* const field[2], int p0, int T, const WaveTune& tn, void* ws,
                              size_t ws_bytes, const PersistCtl& ctl, cudaStream_t st, long long* launches,
                              long long* tile_passes) {
    int* w = static_cast<int*>(ws);
    for (int t = 0; t < T;) {
        const int h = T - t < tn.h ? T - t : tn.h;
        WaveShape sh{};
        if (!wave_shape(a, h, tn.zc, tn.by, tn.lag, &sh, tn.cp)) return cudaErrorInvalidValue;
        if (sizeof(int) * (WAVE_WS_FLAGS + sh.flag_words) > ws_bytes) return cudaErrorInvalidValue;
        cudaError_t e = cudaErrorInvalidValue;
        void* lvl[WAVE_MAXLV + 1];
        for (int l = 0; l <= h; ++l) lvl[l] = field[(p0 + t + l) & 1];
        if (tn.cp == 4) {  // tile copies into shared memory where the grid and device allow them
            e = wave_tma_pass(a, lvl, h, tn, w, ctl, st, launches);
            if (e == cudaSuccess) {
                if (tile_passes) ++*tile_passes;
                t += h;
                continue;
            }
            if (e != cudaErrorNotReady) return e;
        }
        if (tn.by == 4) e = wave_pass_any<KIND, TF, TC, 4>(a, lvl, sh, w, ctl, st, launches);
        else if (tn.by == 8) e = wave_pass_any<KIND, TF, TC, 8>(a, lvl, sh, w, ctl, st, launches);
        else if (tn.by == 16) e = wave_pass_any<KIND, TF, TC, 16>(a, lvl, sh, w, ctl, st, launches);
        if (e != cudaSuccess) return e;
        t += h;
    }
    return cudaSuccess;
}

size_t wave_workspace_bytes(const SweepArgs& a, const WaveTune& tn) {
    WaveShape sh{};
    if (!wave_shape(a, tn.h, tn.zc, tn.by, tn.lag, &sh)) return 0;
    return sizeof(int) * (WAVE_WS_FLAGS + sh.flag_words);
}

cudaError_t wave_run(const SweepArgs& a, void* const field[2], int p0, int T, const WaveTune& tn, void* ws,
                     size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s, long long* launches,
                     long long* tile_passes) {
    if (T <= 0 || a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    if (!ws) return cudaErrorInvalidValue;
#define STG_WR(KK, TTF, TTC) \
    return wave_run_t<KK, TTF, TTC>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches, tile_passes)
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) STG_WR(K7C, float, float);
            if (a.fdt == DT_F64) STG_WR(K7C, double, double);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WR(K7V, float, float);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WR(K7V, float, __nv_bfloat16);
            if (a.fdt == DT_F64) STG_WR(K7V, double, double);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WR(K25V, float, float);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WR(K25V, float, __nv_bfloat16);
            if (a.fdt == DT_F64) STG_WR(K25V, double, double);
            break;
    }
#undef STG_WR
    return cudaErrorInvalidValue;
}


// One pass whose levels read and write the given arrays (levels[l] -> levels[l + 1],
// l < nlev - 1): every intermediate time level is kept, e.g. the states a checkpointed
// adjoint recomputes.
template <int KIND, typename TF, typename TC, int OP>
static cudaError_t wave_levels_t(const SweepArgs& a, void* const* levels, int nlev, const WaveTune& tn, void* ws,
                                 size_t ws_bytes, const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    const int h = nlev - 1;
    WaveShape sh{};
    if (!wave_shape(a, h, tn.zc, tn.by, tn.lag, &sh, tn.cp)) return cudaErrorInvalidValue;
    if (sizeof(int) * (WAVE_WS_FLAGS + sh.flag_words) > ws_bytes) return cudaErrorInvalidValue;
    int* w = static_cast<int*>(ws);
    if (tn.by == 4) return wave_pass_any<KIND, TF, TC, 4, OP>(a, levels, sh, w, ctl, st, launches);
    if (tn.by == 8) return wave_pass_any<KIND, TF, TC, 8, OP>(a, levels, sh, w, ctl, st, launches);
    if (tn.by == 16) return wave_pass_any<KIND, TF, TC, 16, OP>(a, levels, sh, w, ctl, st, launches);
    return cudaErrorInvalidValue;
}

cudaError_t wave_run_levels(const SweepArgs& a, void* const* levels, int nlev, const WaveTune& tn, void* ws,
                            size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s, long long* launches, bool transposed) {
    if (nlev < 2 || a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    if (!ws) return cudaErrorInvalidValue;
#define STG_WL(KK, TTF, TTC, OP) return wave_levels_t<KK, TTF, TTC, OP>(a, levels, nlev, tn, ws, ws_bytes, ctl, s, launches)
    if (transposed) {  // the adjoint's cotangent recursion (variable-coefficient stencils)
        if (a.kind == K7V) {
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WL(K7V, float, float, 1);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WL(K7V, float, __nv_bfloat16, 1);
            if (a.fdt == DT_F64) STG_WL(K7V, double, double, 1);
        } else if (a.kind == K25V) {
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WL(K25V, float, float, 1);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WL(K25V, float, __nv_bfloat16, 1);
            if (a.fdt == DT_F64) STG_WL(K25V, double, double, 1);
        }
        return cudaErrorInvalidValue;
    }
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) STG_WL(K7C, float, float, 0);
            if (a.fdt == DT_F64) STG_WL(K7C, double, double, 0);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WL(K7V, float, float, 0);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WL(K7V, float, __nv_bfloat16, 0);
            if (a.fdt == DT_F64) STG_WL(K7V, double, double, 0);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) STG_WL(K25V, float, float, 0);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16) STG_WL(K25V, float, __nv_bfloat16, 0);
            if (a.fdt == DT_F64) STG_WL(K25V, double, double, 0);
            break;
    }
#undef STG_WL
    return cudaErrorInvalidValue;
}

}  // namespace stg
