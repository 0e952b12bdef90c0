// Wavefront pass of the 25-point stencil (Listing 3) with its operands staged in shared
// memory: the field by the tensor memory accelerator, the coefficients by per-thread copies.
//
// The schedule is the stream form of the L2 wavefront (wavefront.cu): CTA (l, q)
// computes time level l of the pass on xy tile q (128 columns by 8 rows) for all
// z, level l trailing level l-1 through the same per-(level, tile) progress
// counters, so the dependencies and the deadlock argument are unchanged. What
// differs is how the operands arrive. In the column walk every thread loads its
// own 24 vectors per plane (x, y and z neighbours, 13 coefficients) and waits a
// full memory latency for them, and the 180 registers it needs leave room for 8
// warps per SM. Here one producer warp copies, per plane, the tile's field plane
// with its 4-cell x and y halos (one tensor box) into a shared-memory ring several
// planes ahead, so the 11 neighbour vectors of a point group are read from shared
// memory and each field value crosses L2 once per CTA. Each consumer thread copies
// its own 13 coefficient vectors NCS - 1 planes ahead into slots of its own with
// cp.async (no value is shared, so per-thread copies duplicate nothing; 13 tensor
// boxes per plane proved slower: the copy engine takes about 100 ns per box).
//
//   field ring:        NFS slots of (136 x 16) FP32, plane p in slot (p + R) mod NFS
//   mbarriers:         full (the copy's bytes landed) and empty (all 8 consumer warps
//                      are done with the slot) per field slot
//   coefficient slots: NCS planes x 13 arrays x 256 threads x one vector
//
// Each update is evaluated by upd25v in Listing 3's order with the same operand
// values as the plain sweep, so results are bit-identical to it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.h"
#include "tma.cuh"

namespace stg {

namespace {

constexpr int TW_R = 4;                    // radius of the 25-point stencil
constexpr int TW_BY = 8;                   // tile rows (one consumer warp each)
constexpr int TW_XW = 32 * 4 + 2 * TW_R;   // box width: 128 interior columns and the x halos
constexpr int TW_MAXLV = 64;               // time levels per pass
constexpr int TW_LEAD = 3;                 // chunks a level may lead the next one (as in the stream form)

template <typename TC>
struct TwCfg {
    static constexpr int YH = TW_BY + 2 * TW_R;                   // field box rows
    static constexpr int FSB = TW_XW * YH * 4;                    // field slot bytes (8704)
    static constexpr int CVB = 4 * (int)sizeof(TC);               // one thread's coefficient vector
    static constexpr int CSB = 13 * 32 * TW_BY * CVB;             // one plane's per-thread slots
    static constexpr int NCS = sizeof(TC) == 4 ? 2 : 4;           // coefficient planes in flight + 1
    static constexpr int NFS = 2 * TW_R + 1 + NCS;                // the z window and the planes ahead
    static constexpr int BAR = 2 * NFS * 8;
    static constexpr size_t SMEM = (size_t)NFS * FSB + (size_t)NCS * CSB + BAR;
    static_assert(FSB % 128 == 0, "box destinations stay 128-byte aligned");
};

struct TwArgs {
    CUtensorMap fmap[2];     // the two field arrays, box (136, 16, 1)
    const void* cf[13];      // coefficient arrays
    Layout L;
    float* lv[TW_MAXLV + 1];  // level l writes lv[l + 1]
    int lvmap[TW_MAXLV];      // level l reads the array of fmap[lvmap[l]]
    int h, zc, nch, ntx, nty;
    int* status;  // sticky: 1 once a wait gave up
    int* never;   // a flag nothing sets (the stall hook waits on it)
    int* flags;   // [h][ntiles]: chunks finished
    unsigned spin_limit;
    int stall_item;
};

__device__ __forceinline__ int tw_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void tw_st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// Bounded wait until *flag >= need.
__device__ __forceinline__ void tw_spin_ge(const TwArgs& A, const int* flag, int need) {
    unsigned n = 0;
    while (tw_ld_acquire(flag) < need) {
        if (*(volatile const int*)A.status != 0) return;
        if (++n > A.spin_limit) {
            atomicCAS(A.status, 0, 1);
            return;
        }
        __nanosleep(32);
    }
}

template <typename TC> struct CoefVec;
template <> struct CoefVec<float> {
    static __device__ __forceinline__ void ld(uint32_t a, float* c) {
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]) : "r"(a));
    }
};
template <> struct CoefVec<__nv_bfloat16> {
    static __device__ __forceinline__ void ld(uint32_t a, float* c) {
        uint32_t u0, u1;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(u0), "=r"(u1) : "r"(a));
        c[0] = __uint_as_float(u0 << 16);  // BF16 widens exactly: its bits above 16 zero bits
        c[1] = __uint_as_float(u0 & 0xffff0000u);
        c[2] = __uint_as_float(u1 << 16);
        c[3] = __uint_as_float(u1 & 0xffff0000u);
    }
};
__device__ __forceinline__ Vec<float, 4> tw_ld4(uint32_t a) {
    Vec<float, 4> r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "r"(a));
    return r;
}

template <typename TC>
__global__ void __launch_bounds__(32 * (TW_BY + 1), 1) wave_tma_kernel(const __grid_constant__ TwArgs A) {
    using Cfg = TwCfg<TC>;
    constexpr int R = TW_R, BY = TW_BY, NFS = Cfg::NFS, NCS = Cfg::NCS;
    extern __shared__ __align__(1024) unsigned char tw_smem[];
    const uint32_t fring = tma_smem(tw_smem);
    const uint32_t cring = fring + NFS * Cfg::FSB;
    const uint32_t bars = cring + NCS * Cfg::CSB;
    const uint32_t ffull = bars, fempty = bars + 8 * NFS;
    const int ntiles = A.ntx * A.nty;
    const int l = (int)blockIdx.x / ntiles, q = (int)blockIdx.x % ntiles;
    const int qx = q % A.ntx, qy = q / A.ntx;
    const int x0 = qx * 128, y0 = qy * BY;
    const int nz = A.L.nz;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    int* const prog = A.flags;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NFS; ++s) {
            mbar_init(ffull + 8 * s, 1);
            mbar_init(fempty + 8 * s, BY);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (warp == BY) {
        // ---- producer warp: dependency waits on all lanes, copies issued by lane 0
        const CUtensorMap* fm = &A.fmap[A.lvmap[l]];
        const int xs = A.L.xo + x0 - R;  // box origin in x (multiple of 8 elements, checked on the host)
        const bool last = l == A.h - 1;
        int prev_have = 0;               // chunks of level l-1 known finished on the 3 x 3 tiles
        auto issue_field = [&](int p) {  // field plane p (-R <= p < nz + R) of level l's input
            bool waited = p == -R;       // the first copy orders the launch's start, later ones their waits
            if (p >= 0 && p < nz) {
                const int c = p / A.zc;
                int need = c + 1 < A.nch ? c + 1 : A.nch;
                if (l > 0 && need > prev_have) {  // level l-1 wrote plane p of the 3 x 3 tiles
                    if (lane < 9) {
                        const int yy = qy + lane / 3 - 1, xx = qx + lane % 3 - 1;
                        if (yy >= 0 && yy < A.nty && xx >= 0 && xx < A.ntx)
                            tw_spin_ge(A, prog + (size_t)(l - 1) * ntiles + (size_t)yy * A.ntx + xx, need);
                    }
                    prev_have = need;
                    waited = true;
                }
                // keep the L2 band short: level l+1 of this tile has finished chunk c - LEAD
                if (!last && p % A.zc == 0 && c - TW_LEAD > 0) {
                    if (lane == 9) tw_spin_ge(A, prog + (size_t)(l + 1) * ntiles + q, c - TW_LEAD);
                    waited = true;
                }
                if (lane == 10 && p == 0 && (int)blockIdx.x == A.stall_item) tw_spin_ge(A, A.never, 1);
            }
            __syncwarp();
            if (lane == 0) {
                const int it = p + R, s = it % NFS, u = it / NFS;
                if (u > 0) mbar_wait(fempty + 8 * s, (uint32_t)((u - 1) & 1), A.status);
                if (waited) {  // values other CTAs published (acquired by the polling lanes) before the copy
                    __threadfence();
                    fence_proxy_async_global();
                }
                mbar_arrive_expect_tx(ffull + 8 * s, (uint32_t)Cfg::FSB);
                // rows y0 - R .. y0 + BY + R - 1 are padded rows y0 .. ; planes p + R likewise
                tma_load_3d(fring + (uint32_t)(s * Cfg::FSB), fm, xs, y0, p + R, ffull + 8 * s);
            }
            __syncwarp();
        };
        for (int p = -R; p < R; ++p) issue_field(p);
        for (int z = 0; z < nz; ++z) issue_field(z + R);
        // no copy may be in flight when the CTA exits: wait (bounded) for each slot's last phase
        if (lane == 0) {
            const int nf = nz + 2 * R;
            for (int s = 0; s < NFS && s < nf; ++s) {
                const int u = (nf - 1 - s) / NFS;  // last use of slot s
                mbar_wait(ffull + 8 * s, (uint32_t)(u & 1), A.status);
            }
        }
        return;
    }

    // ---- consumer warps: warp w updates row y0 + w, lane the vector at x0 + 4 lane
    const int j = y0 + warp;
    const int i0 = x0 + lane * 4;
    const bool act = j < A.L.ny && i0 < A.L.nx;
    float* const dst = A.lv[l + 1];
    constexpr uint32_t RB = TW_XW * 4;  // field box row bytes
    const uint32_t frow = (uint32_t)(((warp + R) * TW_XW + R + lane * 4) * 4);   // the vector in a field slot
    const uint32_t cslot = cring + (uint32_t)(threadIdx.x * Cfg::CVB);  // + (plane slot * 13 + m) * 256 CVB
    auto coef_copy = [&](int p) {  // this thread's 13 coefficient vectors of plane p into its slots
        if (act && p < nz) {
            const size_t g = A.L.at(i0, j, p);
            const uint32_t d = cslot + (uint32_t)((p % NCS) * Cfg::CSB);
#pragma unroll
            for (int m = 0; m < 13; ++m) {
                const char* src = static_cast<const char*>(A.cf[m]) + g * sizeof(TC);
                const uint32_t dst = d + (uint32_t)(m * 32 * BY * Cfg::CVB);
                if constexpr (sizeof(TC) == 4)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
                else
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int p = 0; p < NCS - 1; ++p) coef_copy(p);
    for (int it = 0; it < 2 * R; ++it) mbar_wait(ffull + 8 * (it % NFS), (uint32_t)((it / NFS) & 1), A.status);
    size_t gidx = A.L.at(i0, j, 0);
    const size_t sz = A.L.plane();
    for (int z = 0; z < nz; ++z) {
        {
            const int it = z + 2 * R;  // field plane z + R
            mbar_wait(ffull + 8 * (it % NFS), (uint32_t)((it / NFS) & 1), A.status);
            coef_copy(z + NCS - 1);  // into the slot of plane z - 1, whose values are consumed
            if constexpr (NCS == 2) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            else asm volatile("cp.async.wait_group 3;\n" ::: "memory");
        }
        auto fslot = [&](int p) { return fring + (uint32_t)(((p + R) % NFS) * Cfg::FSB) + frow; };
        const uint32_t fc = fslot(z);
        float xl[12];  // x line [i0 - 4, i0 + 8)
        {
            const Vec<float, 4> a = tw_ld4(fc - 16), b = tw_ld4(fc), c = tw_ld4(fc + 16);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                xl[e] = a.v[e];
                xl[4 + e] = b.v[e];
                xl[8 + e] = c.v[e];
            }
        }
        Vec<float, 4> yp[4], ym[4], zp[4], zm[4];
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            yp[d - 1] = tw_ld4(fc + (uint32_t)d * RB);
            ym[d - 1] = tw_ld4(fc - (uint32_t)d * RB);
            zp[d - 1] = tw_ld4(fslot(z + d));
            zm[d - 1] = tw_ld4(fslot(z - d));
        }
        float cv[13][4];
        const uint32_t cb = cslot + (uint32_t)((z % NCS) * Cfg::CSB);
#pragma unroll
        for (int m = 0; m < 13; ++m) CoefVec<TC>::ld(cb + (uint32_t)(m * 32 * BY * Cfg::CVB), cv[m]);
        Vec<float, 4> out;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float c[13], xp[4], xm[4], ypp[4], ymm[4], zpp[4], zmm[4];
#pragma unroll
            for (int m = 0; m < 13; ++m) c[m] = cv[m][e];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                xp[d] = xl[4 + e + d + 1];
                xm[d] = xl[4 + e - d - 1];
                ypp[d] = yp[d].v[e];
                ymm[d] = ym[d].v[e];
                zpp[d] = zp[d].v[e];
                zmm[d] = zm[d].v[e];
            }
            out.v[e] = upd25v<float>(c, xl[4 + e], xp, xm, ypp, ymm, zpp, zmm);
        }
        if (act) {
            if (i0 + 4 <= A.L.nx) {
                stv<float, 4>(dst + gidx, out);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < A.L.nx) dst[gidx + e] = out.v[e];
            }
        }
        gidx += sz;
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(fempty + 8 * (z % NFS));  // plane z - R: slot (z - R + R) mod NFS
        }
        if (z % A.zc == A.zc - 1 || z == nz - 1) {  // chunk z / zc finished by every consumer warp
            asm volatile("bar.sync 1, %0;\n" ::"r"(32 * BY) : "memory");
            if (threadIdx.x == 0) {
                __threadfence();
                tw_st_release(prog + (size_t)l * ntiles + q, z / A.zc + 1);
            }
        }
    }
}

// The driver's tensor-map encoder, looked up through the runtime (the library does not link
// the driver library, so that it loads on machines without a GPU); null if unavailable.
PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

bool encode_3d(CUtensorMap* m, CUtensorMapDataType dt, int eb, const void* base, const Layout& L, int bx, int by) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)L.px, (cuuint64_t)L.py, (cuuint64_t)L.pz};
    const cuuint64_t strides[2] = {(cuuint64_t)L.px * eb, (cuuint64_t)L.px * L.py * eb};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, es,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename TC>
cudaError_t wave_tma_t(const SweepArgs& a, void* const* lvl, int h, const WaveTune& tn, int* ws, const PersistCtl& ctl,
                       cudaStream_t st, long long* launches) {
    using Cfg = TwCfg<TC>;
    const Layout& L = a.L;
    if (tn.by != TW_BY || h < 1 || h > TW_MAXLV || tn.zc < TW_R) return cudaErrorNotReady;
    // box origins in x are L.xo - R + 128 q: 16-byte aligned for FP32 and BF16 when L.xo - R is a multiple of 8
    if ((L.xo - TW_R) % 8 != 0 || L.xo < TW_R) return cudaErrorNotReady;
    for (int lv = 2; lv < h; ++lv)
        if (lvl[lv] != lvl[lv & 1]) return cudaErrorNotReady;  // the levels alternate between two arrays
    const int ntx = (L.nx + 127) / 128, nty = (L.ny + TW_BY - 1) / TW_BY, ntiles = ntx * nty;
    const long long ctas = (long long)h * ntiles;
    auto kfn = wave_tma_kernel<TC>;
    int dev = 0, sms = 0, per = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    if (Cfg::SMEM > (size_t)optin) return cudaErrorNotReady;
    if ((e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, 32 * (TW_BY + 1), Cfg::SMEM))) return e;
    if (ctas > (long long)per * sms) return cudaErrorNotReady;  // every (level, tile) CTA must be resident
    TwArgs A{};
    if (!encode_3d(&A.fmap[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, lvl[0], L, TW_XW, TW_BY + 2 * TW_R))
        return cudaErrorNotReady;
    if (!encode_3d(&A.fmap[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, h > 1 ? lvl[1] : lvl[0], L, TW_XW,
                   TW_BY + 2 * TW_R))
        return cudaErrorNotReady;
    for (int m = 0; m < 13; ++m) A.cf[m] = a.coef[m];
    A.L = L;
    for (int lv = 0; lv <= h; ++lv) A.lv[lv] = static_cast<float*>(lvl[lv]);
    for (int lv = 0; lv < h; ++lv) A.lvmap[lv] = lv & 1;
    A.h = h;
    A.zc = tn.zc;
    A.nch = (L.nz + tn.zc - 1) / tn.zc;
    A.ntx = ntx;
    A.nty = nty;
    A.status = ws + WAVE_WS_STATUS;
    A.never = ws + WAVE_WS_NEVER;
    A.flags = ws + WAVE_WS_FLAGS;
    A.spin_limit = ctl.spin_limit;
    A.stall_item = ctl.stall_item;
    if ((e = cudaMemsetAsync(ws + WAVE_WS_NEVER, 0, sizeof(int) * (WAVE_WS_FLAGS - WAVE_WS_NEVER + (size_t)ctas), st)))
        return e;
    kfn<<<(unsigned)ctas, 32 * (TW_BY + 1), Cfg::SMEM, st>>>(A);
    if ((e = cudaGetLastError())) return e;
    if (launches) ++*launches;
    return cudaSuccess;
}

}  // namespace

cudaError_t wave_tma_pass(const SweepArgs& a, void* const* lvl, int h, const WaveTune& tn, int* ws,
                          const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    if (a.kind != K25V || a.fdt != DT_F32) return cudaErrorNotReady;
    if (a.cdt == DT_F32) return wave_tma_t<float>(a, lvl, h, tn, ws, ctl, st, launches);
    if (a.cdt == DT_BF16) return wave_tma_t<__nv_bfloat16>(a, lvl, h, tn, ws, ctl, st, launches);
    return cudaErrorNotReady;
}

}  // namespace stg
