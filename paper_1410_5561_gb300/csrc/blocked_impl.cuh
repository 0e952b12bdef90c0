// Temporally blocked sweep: diamond tiling in (y, t), wavefront along z,
// overlapped (trapezoidal) tiles along x.
//
// Paper: Section II-A (multicore wavefront diamond blocking, MWD): extruded
// diamonds in the (y, t) plane, traversed as a wavefront along z, with a group
// of threads sharing one cache block; "frontlines" N_F planes per level per
// wavefront step; Section III-A (tiling of the leading dimension). The GPU
// version:
//
// * Tile geometry. With slope R per step and width D (a multiple of 2R),
//   update (y, t) (producing u_{t+1}(y)) belongs to tile (a, b) with
//   a = floor((y + R t) / D), b = floor((y - R t) / D). Row k = a - b holds
//   tiles that are mutually independent; tile (k, b) depends on (k-1, b) and
//   (k-1, b+1). Each row advances D/(2R) steps on average (the diamond volume
//   N_z D^2 / (2R) of Section III-C). Rows run as successive launches on one
//   stream: the GPU counterpart of the paper's FIFO queue of ready diamonds.
// * One CTA (the thread group) processes one tile for one x-tile and all z.
//   Along x the CTA computes a trapezoid: level l covers R*(Lt-1-l) extra
//   columns on each side, so x-tiles exchange no data. The x-tiles of one
//   diamond run as one thread-block cluster that advances in lockstep (an
//   execution-only barrier per step), which orders a neighbour's HBM store
//   after the loads of the same (parity-array) cells in its overlap.
// * Each time level l keeps a ring of Q = 3 N_F + R (R = 4: 3 N_F + 2R) planes in shared memory
//   holding u_{t_l} on rows N_l = Yc(t_l) +- R. Level l computes planes
//   [s N_F - l d, s N_F - l d + N_F) at step s with d = N_F + R, so the levels
//   of one step are independent and one __syncthreads per step suffices.
//   Boundary rows are prefetched one step ahead with cp.async.
// * Every warp owns a fixed set of (level, row) items for the whole sweep; for
//   the radius-1 stencils it keeps the item's z-window in registers across
//   steps, so each plane costs one shared-memory load of the new plane, the
//   y-neighbour loads and a few shuffles for the x-neighbours.
// * HBM traffic is only the diamond boundary (Section III-C): rows of N_l not
//   computed by level l-1 are loaded from array (p0 + t_l) & 1; an update is
//   stored to array (p0 + t + 1) & 1 only if a point of another tile reads it
//   (or t = T-1). Coefficients are read through L2.
// * The per-point arithmetic is the shared update of common.cuh, so results
//   are bit-identical to the plain sweep.
//
// This file holds the kernels and their host-side launchers as templates. It is
// compiled in several translation units: blocked_<stencil>_<type>.cu instantiate
// the launchers of one combination each (so the library builds in parallel), and
// blocked.cu (with STG_BLOCKED_MAIN) holds the non-template entry points that
// dispatch on kind and element types.
#pragma once
#include <type_traits>
#include <vector>

#include "blocked_launchers.h"
#include "internal.h"

namespace stg {

constexpr int MAXLV = 64;        // levels per tile (D/R - 1 <= 64)
constexpr int MAXTASK = 256;     // HBM-load / fill row tasks per tile
constexpr int MAXITEM = 256;     // computed rows per tile (one warp-wide chunk each)
constexpr int BLK_MAXT = 512;    // threads per CTA
constexpr int MAXCLUSTER = 16;   // x-tiles of one diamond run as one cluster

struct TileMeta {
    int Lt, t0, ntask, nitem, nring;
    int clo[MAXLV], chi[MAXLV];        // computed rows (interior), empty: clo == chi
    int nlo[MAXLV], nhi[MAXLV];        // ring rows [nlo, nhi) in [-R, Ny + R)
    int wlo[MAXLV], whi[MAXLV];        // computed rows NOT stored to HBM
    int roff[MAXLV];                   // ring element offset in shared memory
    int vlo[MAXLV];                    // first computed ring vector
    int xlo[MAXLV], xhi[MAXLV];        // computed x range (interior coordinates)
    int ldlo[MAXLV], ldhi[MAXLV];      // ring vectors loaded for this level's input
    short tl[MAXTASK], ty[MAXTASK];    // load / fill tasks for interior planes
    unsigned char tfill[MAXTASK];
    int tpre[MAXTASK + 1];             // vectors of tasks [0, i): a task moves one ring row
    short il[MAXITEM], iy[MAXITEM];    // compute items (level, first row, 32-vector chunk, rows)
    unsigned char ich[MAXITEM], inr[MAXITEM];
};

// Per-grid constants of a blocked sweep.
template <typename TF, typename TC>
struct GridArgs {
    Layout L;
    TF* f[2];
    const TC* C[13];
    TF c0, c1, halo;
    int p0, T, D, Xt, EH, Xs, CX;
    int Xe;  // width of the first and last x tiles (Xt, or Xt plus the one-sided overlap)
};

// Row launch: every tile (row, bmin + blockIdx.y) of one diamond row, x tile blockIdx.x.
template <typename TF, typename TC>
struct BlkParams {
    GridArgs<TF, TC> G;
    int row, bmin;
};

__host__ __device__ inline void level_rows(int D, int R, int Ny, int a, int b, int t, int& lo, int& hi) {
    int l1 = a * D - R * t, l2 = b * D + R * t;
    int h1 = a * D + D - R * t, h2 = b * D + D + R * t;
    lo = l1 > l2 ? l1 : l2;
    hi = h1 < h2 ? h1 : h2;
    if (lo < 0) lo = 0;
    if (hi > Ny) hi = Ny;
    if (lo >= hi) lo = hi = 0;
}

__host__ __device__ inline void row_trange(int D, int R, int T, int k, int& tlo, int& thi) {
    int m = D / (2 * R);
    tlo = (k - 1) * m + 1;
    if (tlo < 0) tlo = 0;
    thi = (k + 1) * m;
    if (thi > T) thi = T;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_u32(uint32_t s, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Predicated copy: no branch (so no divergent region) for lanes without a pair.
__device__ __forceinline__ void cp_async16_if(bool p, uint32_t s, const void* gmem) {
    asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q cp.async.cg.shared.global [%1], [%2], 16;\n}\n"
                 ::"r"((unsigned)p), "r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Predicated 128-bit global store (no branch).
template <typename TF, int V> struct Stg;
template <> struct Stg<float, 4> {
    static __device__ __forceinline__ void st_if(bool p, float* a, const Vec<float, 4>& x) {
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.global.v4.f32 [%1], {%2, %3, %4, %5};\n}\n"
                     ::"r"((unsigned)p), "l"(a), "f"(x.v[0]), "f"(x.v[1]), "f"(x.v[2]), "f"(x.v[3]));
    }
};
template <> struct Stg<double, 2> {
    static __device__ __forceinline__ void st_if(bool p, double* a, const Vec<double, 2>& x) {
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.global.v2.f64 [%1], {%2, %3};\n}\n"
                     ::"r"((unsigned)p), "l"(a), "d"(x.v[0]), "d"(x.v[1]));
    }
};

// Execution-only barrier across the cluster (the x-tiles of one diamond). It
// carries no memory ordering: it only keeps the x-tiles in lockstep so that a
// neighbour's HBM store of step s lands after this CTA's cp.async loads issued
// at step s-2 or earlier have completed (their wait_group precedes the arrive).
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }

// CTA barrier (__syncthreads) that returns a token: shared-memory loads that take
// the token as an operand (Lds::ldt) cannot be moved above the barrier, while the
// compiler stays free to schedule them within the step.
__device__ __forceinline__ uint32_t bar_sync_token(uint32_t x) {
    uint32_t t;
    asm volatile("bar.sync 0;\n\tmov.u32 %0, %1;\n" : "=r"(t) : "r"(x) : "memory");
    return t;
}

// Shared-memory vector access through 32-bit shared-window addresses.
template <typename TF, int V> struct Lds;
template <> struct Lds<float, 4> {
    // Loads ordered only by the barrier token tok (data written before that barrier
    // and not rewritten until the next one): free to be scheduled within a step.
    static __device__ __forceinline__ Vec<float, 4> ldt(uint32_t a, uint32_t tok) {
        Vec<float, 4> r;
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
            : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "r"(a), "r"(tok));
        return r;
    }
    static __device__ __forceinline__ float ld1t(uint32_t a, uint32_t tok) {
        float r;
        asm("ld.shared.f32 %0, [%1];\n" : "=f"(r) : "r"(a), "r"(tok));
        return r;
    }
    static __device__ __forceinline__ float ld1t_if(bool p, uint32_t a, uint32_t tok) {
        float r = 0.f;
        asm("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f32 %0, [%2];\n}\n"
            : "+f"(r) : "r"((unsigned)p), "r"(a), "r"(tok));
        return r;
    }
    // predicated forms: no branch; the load leaves 0 where p is false
    static __device__ __forceinline__ float ld1_if(bool p, uint32_t a) {
        float r = 0.f;
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f32 %0, [%2];\n}\n"
                     : "+f"(r) : "r"((unsigned)p), "r"(a));
        return r;
    }
    static __device__ __forceinline__ void st_if(bool p, uint32_t a, const Vec<float, 4>& x) {
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.v4.f32 [%1], {%2, %3, %4, %5};\n}\n"
                     ::"r"((unsigned)p), "r"(a), "f"(x.v[0]), "f"(x.v[1]), "f"(x.v[2]), "f"(x.v[3]));
    }
    static __device__ __forceinline__ Vec<float, 4> ld(uint32_t a) {
        Vec<float, 4> r;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "r"(a));
        return r;
    }
    static __device__ __forceinline__ void st(uint32_t a, const Vec<float, 4>& x) {
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x.v[0]), "f"(x.v[1]), "f"(x.v[2]),
                     "f"(x.v[3]));
    }
};
template <> struct Lds<double, 2> {
    static __device__ __forceinline__ Vec<double, 2> ldt(uint32_t a, uint32_t tok) {
        Vec<double, 2> r;
        asm("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.v[0]), "=d"(r.v[1]) : "r"(a), "r"(tok));
        return r;
    }
    static __device__ __forceinline__ double ld1t(uint32_t a, uint32_t tok) {
        double r;
        asm("ld.shared.f64 %0, [%1];\n" : "=d"(r) : "r"(a), "r"(tok));
        return r;
    }
    static __device__ __forceinline__ double ld1t_if(bool p, uint32_t a, uint32_t tok) {
        double r = 0.0;
        asm("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f64 %0, [%2];\n}\n"
            : "+d"(r) : "r"((unsigned)p), "r"(a), "r"(tok));
        return r;
    }
    static __device__ __forceinline__ double ld1_if(bool p, uint32_t a) {
        double r = 0.0;
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f64 %0, [%2];\n}\n"
                     : "+d"(r) : "r"((unsigned)p), "r"(a));
        return r;
    }
    static __device__ __forceinline__ void st_if(bool p, uint32_t a, const Vec<double, 2>& x) {
        asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n @q st.shared.v2.f64 [%1], {%2, %3};\n}\n"
                     ::"r"((unsigned)p), "r"(a), "d"(x.v[0]), "d"(x.v[1]));
    }
    static __device__ __forceinline__ Vec<double, 2> ld(uint32_t a) {
        Vec<double, 2> r;
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.v[0]), "=d"(r.v[1]) : "r"(a));
        return r;
    }
    static __device__ __forceinline__ void st(uint32_t a, const Vec<double, 2>& x) {
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(x.v[0]), "d"(x.v[1]));
    }
};
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int pmod(int a, int q) {
    int r = a % q;
    return r < 0 ? r + q : r;
}
__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int cdiv(int a, int b) { return -fdiv(-a, b); }
__device__ __forceinline__ int wrap_inc(int s, int q) { return s + 1 == q ? 0 : s + 1; }
constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }


// Per-warp state of one owned item (level l, RB adjacent rows y0.., one 32-vector
// chunk): pointers and lane flags.
template <typename TF, int V, int RB>
struct Item {
    const TF* rowp;    // ring row y0 of level l, slot 0, this lane's vector
    bool hasd[RB];     // row y0+i has a ring row at level l+1
    TF* gdst;          // HBM array receiving u_{t+1}
    uint32_t g0[RB];   // element index of (xg, y0+i, z = 0) (< (R + 1) planes, checked on the host)
    char* gst[RB];     // address of (xg, y0+i, z = 0) in gdst
    int PS, dPS;       // ring plane strides (elements)
    int zb0;           // z of the item's first plane at step 0 (= -l d)
    int slz;           // ring slot of the item's first plane at the current step
    int qr;            // vectors available to the right of this lane's vector
    int xg;            // interior x of the lane's element 0
    int nr;            // valid rows (1..RB)
    uint32_t ar;       // shared address of rowp
    uint32_t ad[RB];   // shared address of row y0+i of level l+1, slot 0, this lane's vector
    int rq;            // right-neighbour vector offset (1, or 0 at the end of the ring row)
    bool valid, active, indom, full;
    bool store[RB];
    bool wr[RB];       // lane writes row i to the next level's ring (fast path)
    bool fastok;       // warp-uniform: RB real rows and no lane straddles the x boundary
};

// One tile (row k, diamond b) of one grid, x tile xti, all z; the whole CTA
// participates. lock: the x tiles of the diamond run as a lockstep cluster.
// p0: array holding u_0 of this run. ring / M: the CTA's shared memory.
template <int KIND, typename TF, typename TC, int K, int NF>
__device__ __forceinline__ void run_tile(const GridArgs<TF, TC>& P, const int k, const int b, const int xti,
                                         const bool lock, const int p0, TileMeta& M, TF* ring) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int NC = KindTraits<KIND>::NC;
    constexpr int V = 16 / sizeof(TF);
    constexpr int J = (R + V - 1) / V;
    constexpr int HV = J * V;
    constexpr bool PERSIST = (R == 1);  // keep z-windows in registers across steps
    constexpr int RB = PERSIST ? 2 : 1;   // adjacent rows per item (diamond widths are multiples of 2R)
    static_assert(RB == 1 || R == 1, "two-row items assume radius 1");
    constexpr int WIN = 2 * R + NF;
    using VT = Vec<TF, V>;

    const Layout& L = P.L;
    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int NW = NT >> 5;
    const int warp = tid >> 5, lane = tid & 31;
    const int a = b + k;
    const int D = P.D, Xs = P.Xs, Xt = P.Xt, EH = P.EH;
    constexpr int d = NF + R;
    // ring depth (planes per level): with register windows the ring is read from the
    // current plane up, otherwise from R planes below it
    constexpr int Q = PERSIST ? 3 * NF + R : 3 * NF + 2 * R;
    // x tiles: interior tiles are Xt wide; with R = 1 the first and last tiles, which need no
    // trapezoid overlap on the grid's side, are Xe = Xt + overlap wide (the host sets Xe = Xt
    // otherwise), so their rows fit the same lanes
    const int x0 = xti == 0 ? 0 : P.Xe + (xti - 1) * Xt;
    const int Wt = (xti == 0 || xti == P.CX - 1) ? P.Xe : Xt;
    const int Ny = L.ny, Nz = L.nz, Nx = L.nx;
    __syncthreads();  // the previous tile of this CTA has finished with M and the ring
    const int rnx = ((Nx + V - 1) / V) * V;
    const int nvs = Xs / V;  // vectors per ring row

    if (tid == 0) {
        int tlo, thi;
        row_trange(D, R, P.T, k, tlo, thi);
        int Lt = thi > tlo ? thi - tlo : 0;
        if (Lt > MAXLV) Lt = MAXLV;  // host guarantees D/R - 1 <= MAXLV
        M.Lt = Lt;
        M.t0 = tlo;
        int off = 0, ntask = 0, nitem = 0;
        for (int l = 0; l < Lt; ++l) {
            int lo, hi;
            level_rows(D, R, Ny, a, b, tlo + l, lo, hi);
            M.clo[l] = lo;
            M.chi[l] = hi;
            int nlo = 0, nhi = 0;
            if (hi > lo) {
                nlo = lo - R;
                nhi = hi + R;
            }
            M.nlo[l] = nlo;
            M.nhi[l] = nhi;
            M.roff[l] = off;
            off += Q * (nhi - nlo) * Xs;
            // x extent: level l computes [x0 - e, x0 + Wt + e), e = R (Lt - 1 - l), clipped
            // to the vectors that hold interior columns when the ring is prefilled with the
            // Dirichlet value (R = 1), else to [-HV, rnx + HV); its input spans R more on each
            // side.
            const int e = R * (Lt - 1 - l);
            const int clo = PERSIST ? 0 : -HV, chi = PERSIST ? rnx : rnx + HV;
            int xl = x0 - e, xh = x0 + Wt + e;
            if (xl < clo) xl = clo;
            if (xh > chi) xh = chi;
            M.xlo[l] = xl;
            M.xhi[l] = xh;
            M.vlo[l] = fdiv(xl - x0 + EH, V);
            int il_ = x0 - e - R, ih_ = x0 + Wt + e + R;
            if (il_ < -HV) il_ = -HV;
            if (ih_ > rnx + HV) ih_ = rnx + HV;
            M.ldlo[l] = fdiv(il_ - x0 + EH, V);
            M.ldhi[l] = cdiv(ih_ - x0 + EH, V);
            // load tasks: interior rows of N_l that level l-1 does not compute, and halo rows
            if (hi > lo) {
                const bool prev = l > 0 && M.chi[l - 1] > M.clo[l - 1];
                const int blo = prev ? M.clo[l - 1] : 1 << 30, bhi = prev ? M.chi[l - 1] : 1 << 30;
                for (int y = nlo; y < nhi; ++y) {
                    const bool halo_row = y < 0 || y >= Ny;
                    const bool computed = !halo_row && y >= blo && y < bhi;
                    if (computed || ntask >= MAXTASK) continue;
                    M.tl[ntask] = (short)l;
                    M.ty[ntask] = (short)y;
                    M.tfill[ntask] = halo_row ? 1 : 0;
                    ++ntask;
                }
                const int nch = (cdiv(xh - x0 + EH, V) - M.vlo[l] + 31) / 32;
                for (int y = lo; y < hi; y += RB)
                    for (int c = 0; c < nch && nitem < MAXITEM; ++c) {
                        M.il[nitem] = (short)l;
                        M.iy[nitem] = (short)y;
                        M.ich[nitem] = (unsigned char)c;
                        M.inr[nitem] = (unsigned char)(hi - y < RB ? hi - y : RB);
                        ++nitem;
                    }
            }
        }
        M.ntask = ntask;
        M.nitem = nitem;
        M.nring = off;
        M.tpre[0] = 0;
        for (int i = 0; i < ntask; ++i) M.tpre[i + 1] = M.tpre[i] + (M.ldhi[M.tl[i]] - M.ldlo[M.tl[i]]);
        for (int l = 0; l < Lt; ++l) {
            const int t = tlo + l;
            const bool all = (t == P.T - 1) || (l + 1 >= Lt) || (M.chi[l + 1] <= M.clo[l + 1]);
            if (all) {
                M.wlo[l] = M.whi[l] = 0;
            } else {
                const int c2lo = M.clo[l + 1], c2hi = M.chi[l + 1];
                M.wlo[l] = c2lo > 0 ? c2lo + R : 0;
                M.whi[l] = c2hi < Ny ? c2hi - R : Ny;
                if (M.whi[l] < M.wlo[l]) M.whi[l] = M.wlo[l];
            }
        }
    }
    __syncthreads();
    const int Lt = M.Lt;
    if (Lt == 0) return;
    const TF hv = P.halo;
    uint32_t tok = 0;  // barrier token of the fast path's shared-memory loads
    if constexpr (PERSIST) {
        // Dirichlet value everywhere: ring cells of lanes outside the domain are never
        // written by the fast path and must read as the boundary value
        VT h;
#pragma unroll
        for (int e = 0; e < V; ++e) h.v[e] = hv;
        const uint32_t rb = smem_u32(ring);
        for (int i = tid; i < M.nring / V; i += NT) Lds<TF, V>::st(rb + (uint32_t)(i * V * (int)sizeof(TF)), h);
        tok = bar_sync_token(tok);
    }
    const int ntask = M.ntask;
    const int s_begin = -((2 * R + NF + NF - 1) / NF);
    const int s_end = (Nz - 1 + (Lt - 1) * d) / NF + 1;
    const size_t gplane = L.plane();

    // ---- per-warp owned items
    Item<TF, V, RB> it[K];
    VT win[K][RB][WIN];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        Item<TF, V, RB>& I = it[kk];
        const int id = warp + kk * NW;
        I.valid = id < M.nitem;
        if (!I.valid) continue;
        const int l = M.il[id], y0 = M.iy[id];
        I.nr = M.inr[id];
        const int nlo = M.nlo[l];
        I.PS = (M.nhi[l] - nlo) * Xs;
        const int v = M.vlo[l] + 32 * M.ich[id] + lane;
        const int vr = v < nvs ? v : nvs - 1;  // clamped read vector (inactive lanes only)
        I.qr = nvs - 1 - vr;
        I.rowp = ring + M.roff[l] + (y0 - nlo) * Xs + vr * V;
        I.xg = x0 - EH + v * V;
        I.active = (I.xg + V > M.xlo[l]) && (I.xg < M.xhi[l]);
        I.indom = I.xg >= 0 && I.xg < Nx;
        I.full = I.xg >= 0 && I.xg + V <= Nx;
        I.dPS = 0;
        const bool nxt = l + 1 < Lt;
        if (nxt) I.dPS = (M.nhi[l + 1] - M.nlo[l + 1]) * Xs;
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int y = y0 + (i < I.nr ? i : I.nr - 1);
            I.hasd[i] = nxt && y >= M.nlo[l + 1] && y < M.nhi[l + 1];
            I.ad[i] = I.hasd[i] ? smem_u32(ring + M.roff[l + 1] + (y - M.nlo[l + 1]) * Xs + v * V) : 0u;
            I.store[i] = i < I.nr && I.active && I.indom && !(y >= M.wlo[l] && y < M.whi[l]) && I.xg >= x0 &&
                         I.xg < x0 + Wt;
            I.g0[i] = I.indom ? (uint32_t)L.at(I.xg, y, 0) : 0u;
        }
        I.gdst = P.f[(p0 + M.t0 + l + 1) & 1];
#pragma unroll
        for (int i = 0; i < RB; ++i) I.gst[i] = reinterpret_cast<char*>(I.gdst + I.g0[i]);
        I.zb0 = -l * d;
        I.slz = pmod(s_begin * NF + I.zb0, Q);
        I.ar = smem_u32(I.rowp);
        I.rq = I.qr < 1 ? I.qr : 1;
#pragma unroll
        for (int i = 0; i < RB; ++i) I.wr[i] = I.active && I.indom && I.hasd[i];
        // the fast path writes nothing for lanes outside the domain (the ring is
        // pre-filled with the Dirichlet value) and has no per-element x mask
        I.fastok = I.nr == RB && !__any_sync(0xffffffffu, I.indom && !I.full);
    }

    if constexpr (PERSIST) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk)
#pragma unroll
            for (int i = 0; i < RB; ++i)
#pragma unroll
                for (int r = 0; r < WIN; ++r)
#pragma unroll
                    for (int e = 0; e < V; ++e) win[kk][i][r].v[e] = hv;
    }

    // ---- producer: HBM loads (cp.async) and Dirichlet fills of planes P_l(s) = [s NF - l d + NF + R, +NF)
    // The (task row, vector) pairs of the tile are spread over all threads, so every
    // thread moves about the same number of vectors per step: pair q = tid + j NT,
    // j < KT, is kept in registers for the whole sweep (with the ring slot of its
    // next plane, advanced as the calls proceed); any further pairs are re-derived.
    // (one pair per thread covers the 7-point variable tiles and frees registers for
    // their coefficient loads; measured on GB300)
    constexpr int KT = KIND == K7V ? 1 : 2;
    const int npair = M.tpre[ntask];
    uint32_t pa_dst[KT];   // shared address: task row, slot 0, the pair's vector
    uint32_t pa_psb[KT];   // plane stride of the task's ring (bytes)
    const TF* pa_src[KT];  // the pair's vector of the task row at z = 0 (any valid address: fill)
    int pa_zb0[KT];        // first plane at step 0
    int pa_sl[KT];         // ring slot of the first plane of the next call
    bool pa_ok[KT];
    bool pa_fill[KT];      // a halo row: Dirichlet value, no load
    {
        int ti = 0;
#pragma unroll
        for (int j = 0; j < KT; ++j) {
            const int q = tid + j * NT;
            pa_ok[j] = q < npair;
            pa_fill[j] = true;
            pa_dst[j] = 0;
            pa_psb[j] = 0;
            pa_src[j] = P.f[0];
            pa_zb0[j] = 0;
            pa_sl[j] = 0;
            if (!pa_ok[j]) continue;
            while (M.tpre[ti + 1] <= q) ++ti;
            const int l = M.tl[ti], y = M.ty[ti];
            const int nlo = M.nlo[l];
            const int c = M.ldlo[l] + (q - M.tpre[ti]);
            pa_psb[j] = (uint32_t)((M.nhi[l] - nlo) * Xs * (int)sizeof(TF));
            pa_dst[j] = smem_u32(ring + M.roff[l] + (y - nlo) * Xs + c * V);
            pa_zb0[j] = -l * d + NF + R;
            pa_sl[j] = pmod(s_begin * NF + pa_zb0[j], Q);
            pa_fill[j] = M.tfill[ti] != 0;
            if (!pa_fill[j])
                pa_src[j] = P.f[(p0 + M.t0 + l) & 1] + L.at(0, y, 0) + (ptrdiff_t)(x0 - EH) + (ptrdiff_t)c * V;
        }
    }
    // produce(s) touches the Dirichlet z-halo of some level only if s < fill_lo (the
    // deepest level's planes s NF + NF + R - (Lt - 1) d start below 0) or s >= fill_hi
    // (level 0's planes reach Nz); the per-level test below is exact
    const int fill_lo = cdiv((Lt - 1) * d - NF - R, NF);
    const int fill_hi = fdiv(Nz - 2 * NF - R, NF) + 1;

    // produce(s) is called for consecutive s (the ring slots advance by N_F per call)
    const int gplaneB = (int)(gplane * sizeof(TF));  // a plane has fewer than 2^28 elements (checked on the host)
    const bool pa_fast = npair <= KT * NT;
    auto produce = [&](int s) {
        if constexpr (PERSIST) {
            if (pa_fast && s >= fill_lo && s < fill_hi) {  // block-uniform
                // steady state: every plane of the call is a real plane of every level, and
                // halo rows keep the value the ring was filled with, so every thread issues
                // its pairs' copies predicated, with no branch
#pragma unroll
                for (int j = 0; j < KT; ++j) {
                    const char* const gp = reinterpret_cast<const char*>(pa_src[j]);
                    const int z0 = s * NF + pa_zb0[j];
                    const bool live = pa_ok[j] && !pa_fill[j];
                    int sl = pa_sl[j];
#pragma unroll
                    for (int fz = 0; fz < NF; ++fz) {
                        cp_async16_if(live, pa_dst[j] + (uint32_t)sl * pa_psb[j], gp + (long long)(z0 + fz) * gplaneB);
                        sl = sl + 1 == Q ? 0 : sl + 1;
                    }
                    pa_sl[j] = pa_sl[j] + NF >= Q ? pa_sl[j] + NF - Q : pa_sl[j] + NF;
                }
                return;
            }
        }
        VT hvv;
#pragma unroll
        for (int e = 0; e < V; ++e) hvv.v[e] = hv;
#pragma unroll
        for (int j = 0; j < KT; ++j) {
            if (pa_ok[j]) {
                const int z0 = s * NF + pa_zb0[j];
                int sl = pa_sl[j];
                if (z0 >= 0 && z0 + NF <= Nz) {  // every plane of the call is a real plane
                    if (!pa_fill[j]) {
                        const TF* gp = pa_src[j] + (size_t)z0 * gplane;
#pragma unroll
                        for (int fz = 0; fz < NF; ++fz) {
                            cp_async16_u32(pa_dst[j] + (uint32_t)sl * pa_psb[j], gp + (size_t)fz * gplane);
                            sl = sl + 1 == Q ? 0 : sl + 1;
                        }
                    } else {
#pragma unroll
                        for (int fz = 0; fz < NF; ++fz) {
                            Lds<TF, V>::st(pa_dst[j] + (uint32_t)sl * pa_psb[j], hvv);
                            sl = sl + 1 == Q ? 0 : sl + 1;
                        }
                    }
                } else {
#pragma unroll
                    for (int fz = 0; fz < NF; ++fz) {
                        const int z = z0 + fz;
                        const uint32_t dst = pa_dst[j] + (uint32_t)sl * pa_psb[j];
                        sl = sl + 1 == Q ? 0 : sl + 1;
                        if (z < 0 || z >= Nz) continue;
                        if (pa_fill[j]) Lds<TF, V>::st(dst, hvv);
                        else cp_async16_u32(dst, pa_src[j] + (size_t)z * gplane);
                    }
                }
            }
            pa_sl[j] = pa_sl[j] + NF >= Q ? pa_sl[j] + NF - Q : pa_sl[j] + NF;
        }
        for (int q = tid + KT * NT, ti = 0; q < npair; q += NT) {
            while (M.tpre[ti + 1] <= q) ++ti;
            const int l = M.tl[ti], y = M.ty[ti];
            const int nlo = M.nlo[l];
            const int c = M.ldlo[l] + (q - M.tpre[ti]);
            const int PS = (M.nhi[l] - nlo) * Xs;
            TF* rowv = ring + M.roff[l] + (y - nlo) * Xs + c * V;
            const int zb = s * NF - l * d + NF + R;
#pragma unroll
            for (int fz = 0; fz < NF; ++fz) {
                const int z = zb + fz;
                if (z < 0 || z >= Nz) continue;
                TF* dst = rowv + pmod(z, Q) * PS;
                if (M.tfill[ti]) {
                    stv<TF, V>(dst, hvv);
                } else {
                    const TF* src = P.f[(p0 + M.t0 + l) & 1] + L.at(0, y, 0) + (ptrdiff_t)(x0 - EH) + (ptrdiff_t)c * V;
                    cp_async16(dst, src + (size_t)z * gplane);
                }
            }
        }
        // Dirichlet z-halo planes: every row of the level's ring (only in the first
        // and last few steps of the wavefront)
        if (s < fill_lo || s >= fill_hi)
        for (int l = 0; l < Lt; ++l) {
            const int zb = s * NF - l * d + NF + R;
            if (zb + NF <= -R || zb >= Nz + R || (zb >= 0 && zb + NF <= Nz)) continue;
            const int nlo = M.nlo[l], nrows = M.nhi[l] - nlo;
            if (nrows <= 0) continue;
            const int ldlo = M.ldlo[l], ldhi = M.ldhi[l];
            for (int fz = 0; fz < NF; ++fz) {
                const int z = zb + fz;
                if (!((z >= -R && z < 0) || (z >= Nz && z < Nz + R))) continue;
                TF* slotb = ring + M.roff[l] + pmod(z, Q) * nrows * Xs;
                for (int r = warp; r < nrows; r += NW)
                    for (int c = ldlo + lane; c < ldhi; c += 32) stv<TF, V>(slotb + r * Xs + c * V, hvv);
            }
        }
    };

    // One wavefront step. With register windows (R = 1) the window of an item is a
    // rotating set of WIN registers: logical plane r of step phase PH lives in register
    // (r + PH N_F) mod WIN, so the windows never move; NPH phases return to the start.
    auto step = [&](const int s, auto phase) {
        constexpr int PH = decltype(phase)::value;
        produce(s + 1);
        cp_async_commit();
        // The stores below may overwrite (same parity array) values that another
        // x-tile of this diamond loads in its overlap; those loads were issued at
        // step s-2 or earlier and completed before that CTA's arrive of step s-1.
        if (lock) cluster_wait();
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            Item<TF, V, RB>& I = it[kk];
            if (!I.valid) continue;
            const int zb = s * NF + I.zb0;
            const int slz = I.slz;  // = zb mod Q
            I.slz = slz + NF >= Q ? slz + NF - Q : slz + NF;
            if constexpr (PERSIST) {
                // the windows advance every step from the start; planes below 0 are the
                // Dirichlet value, so the ring is never read below the current plane
                if (zb + NF + R <= 0 || zb >= Nz) continue;  // warp-uniform
            } else {
                if (zb + NF <= 0 || zb >= Nz) continue;  // warp-uniform
            }
            bool fast = false;
            if constexpr (PERSIST) fast = I.fastok && zb >= 0 && zb + NF + R <= Nz;  // warp-uniform
            if constexpr (PERSIST) if (fast) {
                // steady state: every plane of the step and its z + R neighbour are real
                // planes, both rows are real; straight-line code with predicated accesses
                constexpr int XB = (int)sizeof(TF);
                constexpr uint32_t VB = (uint32_t)(V * XB);
                const uint32_t XsB = (uint32_t)(Xs * XB);
                const uint32_t PSB = (uint32_t)(I.PS * XB), dPSB = (uint32_t)(I.dPS * XB);
                (void)dPSB;
                int sc = slz;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    int sn = sc + R;
                    if (sn >= Q) sn -= Q;
                    const uint32_t an = I.ar + (uint32_t)sn * PSB;
                    win[kk][0][(2 * R + f + PH * NF) % WIN] = Lds<TF, V>::ldt(an, tok);
                    win[kk][1][(2 * R + f + PH * NF) % WIN] = Lds<TF, V>::ldt(an + XsB, tok);
                    const uint32_t acb = I.ar + (uint32_t)sc * PSB;
                    const VT ydn = Lds<TF, V>::ldt(acb - XsB, tok);
                    const VT yup = Lds<TF, V>::ldt(acb + 2 * XsB, tok);
                    const size_t zoff = (size_t)(zb + f) * gplane;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const VT& ctr = win[kk][i][(f + R + PH * NF) % WIN];
                        const uint32_t ac = acb + (uint32_t)i * XsB;
                        // x neighbours of the lane's first and last element. Variable
                        // coefficients: straight from the ring row (fewer issue slots than
                        // shuffles plus edge loads; the word before a chunk's first vector is
                        // in the shared window and only feeds columns outside the level's
                        // range). Constant coefficients: shuffles, with the edge lanes'
                        // neighbours loaded (the direct loads' 4-way bank conflicts cost this
                        // shared-memory-heavier kernel more than they save; measured).
                        TF xm0, xpl;
                        if constexpr (NC > 0) {
                            xm0 = Lds<TF, V>::ld1t(ac - (uint32_t)XB, tok);
                            xpl = Lds<TF, V>::ld1t(ac + (uint32_t)I.rq * VB, tok);
                        } else {
                            const TF lf = Lds<TF, V>::ld1t_if(lane == 0, ac - (uint32_t)XB, tok);
                            const TF rt = Lds<TF, V>::ld1t_if(lane == 31, ac + (uint32_t)I.rq * VB, tok);
                            xm0 = __shfl_up_sync(0xffffffffu, ctr.v[V - 1], 1);
                            xpl = __shfl_down_sync(0xffffffffu, ctr.v[0], 1);
                            xm0 = lane == 0 ? lf : xm0;
                            xpl = lane == 31 ? rt : xpl;
                        }
                        const VT& ym = i == 0 ? ydn : win[kk][0][(f + R + PH * NF) % WIN];
                        const VT& yp = i == 0 ? win[kk][1][(f + R + PH * NF) % WIN] : yup;
                        const VT& zp1 = win[kk][i][(f + R + 1 + PH * NF) % WIN];
                        const VT& zm1 = win[kk][i][(f + R - 1 + PH * NF) % WIN];
                        const size_t gidx = (size_t)I.g0[i] + zoff;  // in bounds for every lane
                        Vec<TC, V> cv[NC > 0 ? NC : 1];
                        (void)cv;
                        (void)gidx;
                        if constexpr (NC > 0) {
#pragma unroll
                            for (int m = 0; m < NC; ++m) cv[m] = ldv_ro<TC, V>(P.C[m] + gidx);
                        }
                        if constexpr (NC > 0 && sizeof(TC) < sizeof(TF)) {
                            // BF16 coefficients: ask L2 for this row's coefficients N_F planes
                            // ahead (the item's next step), so that the first level touching a
                            // plane does not wait on HBM; measured +23 % on GB300 (no gain for
                            // FP32 coefficients, whose kernel is short of registers instead).
                            // In bounds: z + N_F + R <= Nz - 1 + N_F < Nz + 2R planes.
                            static_assert(NF <= 2 * R, "prefetch plane inside the array");
#pragma unroll
                            for (int m = 0; m < NC; ++m)
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.C[m] + gidx + (size_t)NF * gplane));
                        }
                        VT out;
                        if constexpr (KIND == K7C && std::is_same<TF, float>::value) {
                            // packed pairs of points (e, e + 1); the x sums are scalar
                            const F2 c0p = F2::pack(P.c0, P.c0), c1p = F2::pack(P.c1, P.c1);
#pragma unroll
                            for (int e = 0; e < V; e += 2) {
                                const float xpb = e + 2 < V ? ctr.v[e + 2 < V ? e + 2 : 0] : xpl;
                                const float xma = e > 0 ? ctr.v[e > 0 ? e - 1 : 0] : xm0;
                                const F2 sx = F2::pack(Ar<float>::add(ctr.v[e + 1], xma), Ar<float>::add(xpb, ctr.v[e]));
                                const F2 r = upd7c_x2(c0p, c1p, F2::pack(ctr.v[e], ctr.v[e + 1]), sx,
                                                      F2::pack(yp.v[e], yp.v[e + 1]), F2::pack(ym.v[e], ym.v[e + 1]),
                                                      F2::pack(zp1.v[e], zp1.v[e + 1]), F2::pack(zm1.v[e], zm1.v[e + 1]));
                                r.unpack(out.v[e], out.v[e + 1]);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < V; ++e) {
                                const TF xp = e + 1 < V ? ctr.v[e + 1 < V ? e + 1 : 0] : xpl;
                                const TF xm = e > 0 ? ctr.v[e > 0 ? e - 1 : 0] : xm0;
                                if constexpr (KIND == K7C) {
                                    out.v[e] = upd7c<TF>(P.c0, P.c1, ctr.v[e], xp, xm, yp.v[e], ym.v[e], zp1.v[e], zm1.v[e]);
                                } else {
                                    TF c[7];
#pragma unroll
                                    for (int m = 0; m < 7; ++m) c[m] = Cvt<TF, TC>::f(cv[m < NC ? m : 0].v[e]);
                                    out.v[e] = upd7v<TF>(c, ctr.v[e], xp, xm, yp.v[e], ym.v[e], zp1.v[e], zm1.v[e]);
                                }
                            }
                        }
                        Lds<TF, V>::st_if(I.wr[i], I.ad[i] + (uint32_t)sc * dPSB, out);
                        TF* const gp = reinterpret_cast<TF*>(I.gst[i] + (long long)(zb + f) * gplaneB);
                        Stg<TF, V>::st_if(I.store[i], gp, out);
                    }
                    sc = sc + 1 == Q ? 0 : sc + 1;
                }
            }
            const int s0 = slz;  // ring slot of plane zb
#pragma unroll
            for (int f = 0; f < NF && !fast; ++f) {
                const int z = zb + f;
                int sc = s0 + f;
                if (sc >= Q) sc -= Q;  // slot of plane z
                if constexpr (PERSIST) {
                    int sn = sc + R;
                    if (sn >= Q) sn -= Q;  // slot of plane z + R
                    const bool loadnew = z + R >= 0 && z < Nz;
                    const uint32_t an = I.ar + (uint32_t)(sn * I.PS * (int)sizeof(TF));
#pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        if (loadnew) {
                            const int ri = i < I.nr ? i : I.nr - 1;
                            win[kk][i][(2 * R + f + PH * NF) % WIN] =
                                Lds<TF, V>::ld(an + (uint32_t)(ri * Xs * (int)sizeof(TF)));
                        } else {
#pragma unroll
                            for (int e = 0; e < V; ++e) win[kk][i][(2 * R + f + PH * NF) % WIN].v[e] = hv;
                        }
                    }
                } else {
                    if (z >= 0 && z < Nz) {
                        // reload the window of planes z - R .. z + R from the ring
                        int sw = sc - R;
                        if (sw < 0) sw += Q;
#pragma unroll
                        for (int r = 0; r < 2 * R + 1; ++r) {
                            win[kk][0][f + r] = ldv<TF, V>(I.rowp + sw * I.PS);
                            sw = wrap_inc(sw, Q);
                        }
                    }
                }
                if (z < 0 || z >= Nz) continue;
                const uint32_t acb = I.ar + (uint32_t)(sc * I.PS * (int)sizeof(TF));
                constexpr int XB = (int)sizeof(TF);
                VT ydn[R], yup[R];                   // rows y0 - r and y0 + nr - 1 + r
#pragma unroll
                for (int r = 1; r <= R; ++r) {
                    ydn[r - 1] = Lds<TF, V>::ld(acb - (uint32_t)(r * Xs * XB));
                    yup[r - 1] = Lds<TF, V>::ld(acb + (uint32_t)((I.nr - 1 + r) * Xs * XB));
                }
                const size_t zoff = (size_t)z * gplane;
                // window register of logical plane r (rotating for R = 1, fixed otherwise)
                auto W = [&](int i, int r) -> VT& {
                    return win[kk][i][PERSIST ? (r + PH * NF) % WIN : r];
                };
#pragma unroll
                for (int i = 0; i < RB; ++i) {
                    if (i >= I.nr) continue;  // warp-uniform
                    const VT& ctr = W(i, f + R);
                    const uint32_t ac = acb + (uint32_t)(i * Xs * XB);
                    TF xl[(2 * J + 1) * V];
#pragma unroll
                    for (int e = 0; e < V; ++e) xl[J * V + e] = ctr.v[e];
#pragma unroll
                    for (int q = 1; q <= J; ++q) {
                        VT lf{}, rt{};
                        if (lane < q) lf = Lds<TF, V>::ld(ac - (uint32_t)(q * V * XB));
                        if (lane >= 32 - q) rt = Lds<TF, V>::ld(ac + (uint32_t)((q <= I.qr ? q : I.qr) * V * XB));
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            if ((J - q) * V + e >= J * V - R) {  // within R to the left
                                const TF w = __shfl_up_sync(0xffffffffu, ctr.v[e], q);
                                xl[(J - q) * V + e] = lane < q ? lf.v[e] : w;
                            }
                            if ((J + q) * V + e <= J * V + V - 1 + R) {  // within R to the right
                                const TF w = __shfl_down_sync(0xffffffffu, ctr.v[e], q);
                                xl[(J + q) * V + e] = lane >= 32 - q ? rt.v[e] : w;
                            }
                        }
                    }
                    // y neighbours: other rows of this item from the windows, the rest loaded
                    VT ypv[R], ymv[R];
#pragma unroll
                    for (int r = 1; r <= R; ++r) {
                        if constexpr (RB == 1) {
                            ymv[r - 1] = ydn[r - 1];
                            ypv[r - 1] = yup[r - 1];
                        } else {  // two rows, R = 1
                            ymv[0] = i == 0 ? ydn[0] : W(0, f + R);
                            ypv[0] = (i == 0 && I.nr == 2) ? W(RB - 1, f + R) : yup[0];
                        }
                    }
                    const size_t gidx = (size_t)I.g0[i] + zoff;
                    Vec<TC, V> cv[NC > 0 ? NC : 1];
                    (void)cv;
                    (void)gidx;
                    if constexpr (NC > 0) {
                        if (I.active && I.indom) {
#pragma unroll
                            for (int m = 0; m < NC; ++m) cv[m] = ldv_ro<TC, V>(P.C[m] + gidx);
                        } else {
#pragma unroll
                            for (int m = 0; m < NC; ++m)
#pragma unroll
                                for (int e = 0; e < V; ++e) cv[m].v[e] = TC(0);
                        }
                    }
                    VT out;
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int xc = J * V + e;
                        const VT& zp1 = W(i, f + R + 1);
                        const VT& zm1 = W(i, f + R - 1);
                        if constexpr (KIND == K7C) {
                            out.v[e] = upd7c<TF>(P.c0, P.c1, ctr.v[e], xl[xc + 1], xl[xc - 1], ypv[0].v[e],
                                                 ymv[0].v[e], zp1.v[e], zm1.v[e]);
                        } else if constexpr (KIND == K7V) {
                            TF c[7];
#pragma unroll
                            for (int m = 0; m < 7; ++m) c[m] = Cvt<TF, TC>::f(cv[m].v[e]);
                            out.v[e] = upd7v<TF>(c, ctr.v[e], xl[xc + 1], xl[xc - 1], ypv[0].v[e], ymv[0].v[e],
                                                 zp1.v[e], zm1.v[e]);
                        } else {
                            TF c[13], xp[4], xm[4], yp4[4], ym4[4], zp[4], zm[4];
#pragma unroll
                            for (int m = 0; m < 13; ++m) c[m] = Cvt<TF, TC>::f(cv[m].v[e]);
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                xp[q] = xl[xc + q + 1];
                                xm[q] = xl[xc - q - 1];
                                yp4[q] = ypv[q].v[e];
                                ym4[q] = ymv[q].v[e];
                                zp[q] = W(i, f + R + q + 1).v[e];
                                zm[q] = W(i, f + R - q - 1).v[e];
                            }
                            out.v[e] = upd25v<TF>(c, ctr.v[e], xp, xm, yp4, ym4, zp, zm);
                        }
                    }
                    if (!I.full) {
#pragma unroll
                        for (int e = 0; e < V; ++e)
                            if (!(I.xg + e >= 0 && I.xg + e < Nx)) out.v[e] = hv;
                    }
                    if (I.active && I.hasd[i]) Lds<TF, V>::st(I.ad[i] + (uint32_t)(sc * I.dPS * XB), out);
                    if (I.store[i]) {
                        TF* const gp = reinterpret_cast<TF*>(I.gst[i] + (long long)z * gplaneB);
                        if (I.full) {
                            stv<TF, V>(gp, out);
                        } else {
#pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (I.xg + e < Nx) gp[e] = out.v[e];
                        }
                    }
                }
            }
        }
        cp_async_wait_1();
        tok = bar_sync_token(tok + 1);
        if (lock) cluster_arrive_relaxed();
    };

    produce(s_begin);
    cp_async_commit();
    if (lock) cluster_arrive_relaxed();
    constexpr int NPH = PERSIST ? WIN / cgcd(WIN, NF) : 1;
    for (int s = s_begin; s < s_end; s += NPH) {
        step(s, std::integral_constant<int, 0>{});
        if constexpr (NPH > 1) if (s + 1 < s_end) step(s + 1, std::integral_constant<int, 1 % NPH>{});
        if constexpr (NPH > 2) if (s + 2 < s_end) step(s + 2, std::integral_constant<int, 2 % NPH>{});
        static_assert(NPH <= 3, "window rotation period");
    }
    if (lock) cluster_wait();
    cp_async_wait_all();
}

template <int KIND, typename TF, typename TC, int K, int NF>
__global__ void __launch_bounds__(BLK_MAXT, 1) blocked_kernel(const BlkParams<TF, TC> P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ TileMeta M;
    run_tile<KIND, TF, TC, K, NF>(P.G, P.row, P.bmin + (int)blockIdx.y, (int)blockIdx.x, P.G.CX > 1, P.G.p0, M,
                                  reinterpret_cast<TF*>(smem_raw));
}


// ------------------------------------------------------------- persistent batch
// Many independent grids in one launch. Every tile (grid g, row k, diamond b)
// covers its grid's whole x extent. Tiles are listed in row order; a CTA pops
// the next tile from an atomic counter and waits (bounded) until the tiles it
// depends on have published their results: (g, k-1, b), (g, k-1, b+1) and
// (g, k-2, b+1) (the last one matters only when the first two are empty). This
// is the GPU form of the paper's queue of ready diamonds (Section II-A). Every
// popped tile is held by a running CTA and waits only on earlier tiles, so the
// persistent grid (at most the co-resident CTAs) cannot deadlock; a wait that
// exceeds its limit sets the status word and the CTA leaves the loop.

template <typename TF, typename TC>
struct BatchArgs {
    const GridArgs<TF, TC>* grids;  // per grid
    const BatchItem* items;         // dependency order
    int nitems;
    int* head;         // next item to pop
    int* status;       // 0 ok, 1 a dependency wait gave up
    int* done;         // per item: published
    int* gdone;        // per grid: tiles finished in this launch
    const int* ntiles; // per grid: tiles per launch
    int* parity;       // per grid: array holding the current time level
    unsigned spin_limit;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

template <int KIND, typename TF, typename TC, int K, int NF>
__global__ void __launch_bounds__(BLK_MAXT, 1) blocked_batch_kernel(const BatchArgs<TF, TC> A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ TileMeta M;
    __shared__ int s_item, s_abort, s_p0;
    TF* ring = reinterpret_cast<TF*>(smem_raw);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int i = atomicAdd(A.head, 1);
            int abort = 0;
            if (i < A.nitems) {
                const BatchItem it = A.items[i];
                for (int q = 0; q < 3 && !abort; ++q) {
                    const int dd = it.dep[q];
                    if (dd < 0) continue;
                    unsigned n = 0;
                    while (ld_acquire_gpu(A.done + dd) == 0) {
                        if (++n > A.spin_limit || ld_volatile(A.status) != 0) {
                            abort = 1;
                            break;
                        }
                        __nanosleep(200);
                    }
                }
                if (abort) atomicCAS(A.status, 0, 1);
                s_p0 = ld_volatile(A.parity + it.g);
            }
            s_item = i;
            s_abort = abort;
        }
        __syncthreads();
        const int i = s_item;
        if (i >= A.nitems || s_abort) break;
        const BatchItem it = A.items[i];
        const int p0 = s_p0;
        run_tile<KIND, TF, TC, K, NF>(A.grids[it.g], it.k, it.b, 0, false, p0, M, ring);
        __threadfence();  // this thread's HBM stores of the tile are visible GPU-wide
        __syncthreads();
        if (threadIdx.x == 0) {
            st_release_gpu(A.done + i, 1);
            if (atomicAdd(A.gdone + it.g, 1) == A.ntiles[it.g] - 1)
                A.parity[it.g] = (p0 + A.grids[it.g].T) & 1;  // every tile of g has read p0
        }
    }
}


// ------------------------------------------------------- persistent single grid
// The tiles of one grid in row order; cluster c (the x tiles of a diamond, in
// lockstep) processes tiles c, c + NC, c + 2 NC, ... Every tile waits until the
// tiles it depends on have been published by all of their x tiles. Clusters
// are launched only as many as can be resident, and each walks its tiles in
// increasing order while depending only on smaller indices, so the smallest
// unfinished tile can always proceed. A wait that exceeds its limit sets the
// (sticky) status word and proceeds (the results are then invalid but every CTA
// of the cluster keeps to the same barriers, so nothing can hang).
//
// The tile list is not stored: row k of the list holds the diamonds
// b = bmin[k] .. bmin[k] + (base[k+1] - base[k]) - 1 as tiles base[k] ..
// base[k+1] - 1, and the table is a __grid_constant__ kernel parameter, so a
// run needs no host-to-device copy of a plan (it stays asynchronous and can be
// captured in a CUDA graph).
constexpr int MAXPROWS = 960;  // diamond rows of one persistent launch (longer runs are split)

struct PlanRows {
    int nrows, nitems;
    int bmin[MAXPROWS];
    int base[MAXPROWS + 1];
};

// Tile i of the plan: its row k, diamond b and the tiles it waits for.
__device__ __forceinline__ void plan_tile(const PlanRows& P, int i, int& k, int& b) {
    int lo = 0, hi = P.nrows - 1;  // the last row whose first tile is <= i (empty rows share a base)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.base[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    k = lo;
    b = P.bmin[lo] + (i - P.base[lo]);
}
__device__ __forceinline__ int plan_index(const PlanRows& P, int k, int b) {
    if (k < 0 || k >= P.nrows) return -1;
    const int o = b - P.bmin[k];
    return (o >= 0 && o < P.base[k + 1] - P.base[k]) ? P.base[k] + o : -1;
}

template <typename TF, typename TC>
struct PersistArgs {
    GridArgs<TF, TC> G;
    int* status;      // sticky: 1 once a dependency wait gave up
    int* never;       // a flag no tile sets (the stall hook waits on it)
    int* done;        // per tile: x tiles finished
    unsigned spin_limit;
    int stall_item;   // test hook: this tile also waits on *never (-1: none)
    PlanRows P;
};

template <int KIND, typename TF, typename TC, int K, int NF>
__global__ void __launch_bounds__(BLK_MAXT, 1) blocked_persist_kernel(const __grid_constant__ PersistArgs<TF, TC> A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ TileMeta M;
    TF* ring = reinterpret_cast<TF*>(smem_raw);
    const int CX = A.G.CX;
    const int nclusters = (int)gridDim.y;
    for (int i = (int)blockIdx.y; i < A.P.nitems; i += nclusters) {
        int k, b;
        plan_tile(A.P, i, k, b);
        if (threadIdx.x == 0) {
            const int dep[4] = {plan_index(A.P, k - 1, b), plan_index(A.P, k - 1, b + 1),
                                plan_index(A.P, k - 2, b + 1), i == A.stall_item ? -2 : -1};
            for (int q = 0; q < 4; ++q) {
                if (dep[q] == -1) continue;
                const int* flag = dep[q] >= 0 ? A.done + dep[q] : A.never;
                unsigned n = 0;
                while (ld_acquire_gpu(flag) < CX) {
                    if (ld_volatile(A.status) != 0) break;
                    if (++n > A.spin_limit) {
                        atomicCAS(A.status, 0, 1);
                        break;
                    }
                    __nanosleep(128);
                }
            }
        }
        __syncthreads();
        run_tile<KIND, TF, TC, K, NF>(A.G, k, b, (int)blockIdx.x, CX > 1, A.G.p0, M, ring);
        __threadfence();  // this thread's HBM stores of the tile are visible GPU-wide
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(A.done + i, 1);
    }
}

// ------------------------------------------------------------------- host side

static int ring_rows_bound(int D, int R) {
    // full (unclipped) diamond: widths 2R, 4R, ..., D, ..., 2R over 2m-1 levels, each + 2R rows
    int m = D / (2 * R);
    int rows = 0;
    for (int l = 1; l <= 2 * m - 1; ++l) {
        int w = l <= m ? 2 * R * l : 2 * R * (2 * m - l);
        rows += w + 2 * R;
    }
    return rows;
}

static int item_bound(int D, int R) { return D * D / (2 * R); }

struct BlkShape {
    int V, HV, Xt, EH, Xs, Q, K, nch;
    int Xe, CX;  // width of the first and last x tiles, x tiles per row
    size_t smem;
    bool ok;
};

// Shape of the rings and the work split for one grid and tuning. With xtile >= nx
// the whole row is one tile (no cluster); rows wider than one warp of vectors are
// split into 32-vector chunks, each one item.
static BlkShape blk_shape_x(int kind, int fdt, int nx, int dw, int nf, int warps, int xtile);

// The kernel keeps the element index of (x, y, z = 0) and a plane's size in bytes in 32 bits.
static bool index32_ok(const Layout& L) {
    return (size_t)(L.R + 2) * L.plane() < ((size_t)1 << 32) && L.plane() < ((size_t)1 << 28);
}

static BlkShape blk_shape_x(int kind, int fdt, int nx, int dw, int nf, int warps, int xtile) {
    BlkShape s{};
    int R = kind_radius(kind);
    int eb = dtype_bytes(fdt);
    s.V = 16 / eb;
    int J = (R + s.V - 1) / s.V;
    s.HV = J * s.V;
    s.ok = false;
    if (dw < 2 * R || dw % (2 * R) != 0) return s;
    if (nf < 1 || nf > 2) return s;
    int ltmax = dw / R - 1;
    if (ltmax > MAXLV) return s;
    if (warps < 1 || warps * 32 > BLK_MAXT) return s;
    if (xtile < s.V || xtile % s.V != 0 || xtile > 4096) return s;
    int ov = ltmax > 1 ? (R * (ltmax - 1) + s.V - 1) / s.V : 0;
    // x tiles per row: one when the row fits; else, with R = 1, two edge tiles of xtile + ov V
    // columns (no overlap on the grid's side; the same lanes as an interior tile) around
    // ceil((nx - 2 Xe) / xtile) interior tiles; with R = 4, ceil(nx / xtile) equal tiles
    if (nx <= xtile) {
        s.CX = 1;
        s.Xe = xtile;
    } else if (R == 1) {
        s.Xe = xtile + ov * s.V;
        s.CX = nx <= 2 * s.Xe ? 2 : 2 + (nx - 2 * s.Xe + xtile - 1) / xtile;
    } else {
        s.Xe = xtile;
        s.CX = (nx + xtile - 1) / xtile;
    }
    if (s.CX > MAXCLUSTER) return s;
    s.nch = (xtile / s.V + 2 * ov + 31) / 32;
    // rows per item, as in the kernel; unclipped widths are multiples of 2R, and clipping
    // only removes rows, so ceil(w / rb) summed over the levels never exceeds D^2/(2R rb)
    const int rb = R == 1 ? 2 : 1;
    int items = item_bound(dw, R) / rb * s.nch;
    if (items > MAXITEM) return s;
    if (ring_rows_bound(dw, R) > MAXTASK) return s;  // load / fill tasks are ring rows
    int K = (items + warps - 1) / warps;
    if (K > 4) return s;
    s.K = K <= 1 ? 1 : (K <= 2 ? 2 : 4);
    s.Xt = xtile;
    s.EH = ((R * ltmax + s.V - 1) / s.V) * s.V + s.HV;
    s.Xs = s.Xe + 2 * s.EH;  // the widest tile's ring row
    s.Q = R == 1 ? 3 * nf + R : 3 * nf + 2 * R;  // matches the kernel's ring depth
    s.smem = (size_t)s.Q * ring_rows_bound(dw, R) * s.Xs * eb;
    s.ok = true;
    return s;
}

static BlkShape blk_shape(const SweepArgs& a, const BlockedTune& tn) {
    BlkShape s = blk_shape_x(a.kind, a.fdt, a.L.nx, tn.dw, tn.nf, tn.warps, tn.xtile);
    if (!index32_ok(a.L)) s.ok = false;
    return s;
}

#ifdef STG_BLOCKED_MAIN
size_t blocked_smem_bytes(const SweepArgs& a, const BlockedTune& tn) {
    BlkShape s = blk_shape(a, tn);
    if (!s.ok) return 0;
    return s.smem + sizeof(TileMeta);
}
#endif  // STG_BLOCKED_MAIN

template <typename TF, typename TC>
static GridArgs<TF, TC> grid_args(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                                  const BlkShape& sh) {
    GridArgs<TF, TC> G{};
    G.L = a.L;
    G.f[0] = static_cast<TF*>(field[0]);
    G.f[1] = static_cast<TF*>(field[1]);
    for (int m = 0; m < kind_ncoef(a.kind); ++m) G.C[m] = static_cast<const TC*>(a.coef[m]);
    G.c0 = (TF)a.c0;
    G.c1 = (TF)a.c1;
    G.halo = (TF)a.halo;
    G.p0 = p0;
    G.T = T;
    G.D = tn.dw;
    G.Xt = sh.Xt;
    G.Xe = sh.Xe;
    G.EH = sh.EH;
    G.Xs = sh.Xs;
    G.CX = 1;
    return G;
}

template <int KIND, typename TF, typename TC, int K, int NF>
static cudaError_t launch_blocked_k(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                                    const BlkShape& sh, cudaStream_t st, long long* launches) {
    const int R = KindTraits<KIND>::R;
    auto kfn = blocked_kernel<KIND, TF, TC, K, NF>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e != cudaSuccess) return e;
    const int nxt = sh.CX;
    if (nxt > 8) {
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    BlkParams<TF, TC> P{};
    P.G = grid_args<TF, TC>(a, field, p0, T, tn, sh);
    P.G.CX = nxt;
    const int D = tn.dw, Ny = a.L.ny;
    for (int k = 0;; ++k) {
        int tlo, thi;
        row_trange(D, R, T, k, tlo, thi);
        if (tlo >= T) break;
        if (thi <= tlo) continue;
        // tiles of row k that own at least one update
        int bmin = 1 << 30, bmax = -(1 << 30);
        int blo = -(k + 2) / 2 - 2, bhi = (2 * Ny / D - k) / 2 + 2;
        for (int b = blo; b <= bhi; ++b) {
            bool any = false;
            for (int t = tlo; t < thi && !any; ++t) {
                int lo, hi;
                level_rows(D, R, Ny, b + k, b, t, lo, hi);
                any = hi > lo;
            }
            if (any) {
                if (b < bmin) bmin = b;
                if (b > bmax) bmax = b;
            }
        }
        if (bmax < bmin) continue;
        P.row = k;
        P.bmin = bmin;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)nxt, (unsigned)(bmax - bmin + 1), 1);
        cfg.blockDim = dim3((unsigned)(tn.warps * 32), 1, 1);
        cfg.dynamicSmemBytes = sh.smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)nxt;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = nxt > 1 ? 1 : 0;
        e = cudaLaunchKernelEx(&cfg, kfn, P);
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    return cudaSuccess;
}

template <int KIND, typename TF, typename TC>
cudaError_t launch_blocked(const SweepArgs& a, void* const field[2], int p0, int T,
                                  const BlockedTune& tn, cudaStream_t st, long long* launches) {
    BlkShape sh = blk_shape(a, tn);
    if (!sh.ok) return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sh.smem + sizeof(TileMeta) > (size_t)optin) return cudaErrorInvalidValue;
#define STG_BLK(KK, NFF)                                                                                      \
    if (sh.K == KK && tn.nf == NFF)                                                                           \
        return launch_blocked_k<KIND, TF, TC, KK, NFF>(a, field, p0, T, tn, sh, st, launches);
    STG_BLK(1, 1) STG_BLK(2, 1) STG_BLK(4, 1) STG_BLK(1, 2) STG_BLK(2, 2) STG_BLK(4, 2)
#undef STG_BLK
    return cudaErrorInvalidValue;
}

#ifdef STG_BLOCKED_MAIN
cudaError_t blocked_run(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                        cudaStream_t s, long long* launches) {
    if (T <= 0 || a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) return launch_blocked<K7C, float, float>(a, field, p0, T, tn, s, launches);
            if (a.fdt == DT_F64) return launch_blocked<K7C, double, double>(a, field, p0, T, tn, s, launches);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32)
                return launch_blocked<K7V, float, float>(a, field, p0, T, tn, s, launches);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_blocked<K7V, float, __nv_bfloat16>(a, field, p0, T, tn, s, launches);
            if (a.fdt == DT_F64) return launch_blocked<K7V, double, double>(a, field, p0, T, tn, s, launches);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32)
                return launch_blocked<K25V, float, float>(a, field, p0, T, tn, s, launches);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_blocked<K25V, float, __nv_bfloat16>(a, field, p0, T, tn, s, launches);
            if (a.fdt == DT_F64) return launch_blocked<K25V, double, double>(a, field, p0, T, tn, s, launches);
            break;
    }
    return cudaErrorInvalidValue;
}
#endif  // STG_BLOCKED_MAIN


// ------------------------------------------------------------- batch host side

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename TF, typename TC>
static size_t grid_args_bytes() { return sizeof(GridArgs<TF, TC>); }

static size_t gridargs_size(int fdt, int cdt) {
    if (fdt == DT_F64) return grid_args_bytes<double, double>();
    if (cdt == DT_BF16) return grid_args_bytes<float, __nv_bfloat16>();
    return grid_args_bytes<float, float>();
}

// Host plan: the items (in row order) and their dependencies.
static int batch_items(const BatchGrid* g, int n, int dw, std::vector<BatchItem>& items, std::vector<int>& ntiles) {
    const int R = kind_radius(g[0].a.kind);
    items.clear();
    ntiles.assign(n, 0);
    // per grid, per row: [bmin, bmax] and the item index of bmin
    std::vector<std::vector<int>> rbmin(n), rbmax(n), rbase(n);
    int kmax = 0;
    for (int q = 0; q < n; ++q) {
        for (int k = 0;; ++k) {
            int tlo, thi;
            row_trange(dw, R, g[q].T, k, tlo, thi);
            if (tlo >= g[q].T) break;
            kmax = k > kmax ? k : kmax;
        }
    }
    for (int q = 0; q < n; ++q) {
        rbmin[q].assign(kmax + 1, 1);
        rbmax[q].assign(kmax + 1, 0);
        rbase[q].assign(kmax + 1, -1);
    }
    auto nonempty = [&](int q, int k, int b) {
        int tlo, thi;
        row_trange(dw, R, g[q].T, k, tlo, thi);
        for (int t = tlo; t < thi; ++t) {
            int lo, hi;
            level_rows(dw, R, g[q].a.L.ny, b + k, b, t, lo, hi);
            if (hi > lo) return true;
        }
        return false;
    };
    auto index_of = [&](int q, int k, int b) -> int {
        if (k < 0 || k > kmax || rbase[q][k] < 0 || b < rbmin[q][k] || b > rbmax[q][k]) return -1;
        return rbase[q][k] + (b - rbmin[q][k]);
    };
    for (int k = 0; k <= kmax; ++k) {
        for (int q = 0; q < n; ++q) {
            const int Ny = g[q].a.L.ny;
            int tlo, thi;
            row_trange(dw, R, g[q].T, k, tlo, thi);
            if (tlo >= g[q].T || thi <= tlo) continue;
            int bmin = 1 << 30, bmax = -(1 << 30);
            for (int b = -(k + 2) / 2 - 2; b <= (2 * Ny / dw - k) / 2 + 2; ++b)
                if (nonempty(q, k, b)) {
                    bmin = b < bmin ? b : bmin;
                    bmax = b > bmax ? b : bmax;
                }
            if (bmax < bmin) continue;
            rbmin[q][k] = bmin;
            rbmax[q][k] = bmax;
            rbase[q][k] = (int)items.size();
            for (int b = bmin; b <= bmax; ++b) {
                BatchItem it{};
                it.g = q;
                it.k = k;
                it.b = b;
                it.dep[0] = index_of(q, k - 1, b);
                it.dep[1] = index_of(q, k - 1, b + 1);
                it.dep[2] = index_of(q, k - 2, b + 1);
                items.push_back(it);
                ntiles[q]++;
            }
        }
    }
    return (int)items.size();
}

#ifdef STG_BLOCKED_MAIN
cudaError_t batch_plan(const BatchGrid* g, int n, const BlockedTune& tn, BatchLaunch* bl) {
    if (n < 1) return cudaErrorInvalidValue;
    const SweepArgs& a0 = g[0].a;
    int K = 1;
    size_t smem = 0;
    for (int q = 0; q < n; ++q) {
        const SweepArgs& a = g[q].a;
        if (a.kind != a0.kind || a.fdt != a0.fdt || a.cdt != a0.cdt) return cudaErrorInvalidValue;
        const int V = 16 / dtype_bytes(a.fdt);
        const int xt = ((a.L.nx + V - 1) / V) * V;
        BlkShape sh = blk_shape_x(a.kind, a.fdt, a.L.nx, tn.dw, tn.nf, tn.warps, xt);
        if (!sh.ok || !index32_ok(a.L)) return cudaErrorInvalidValue;
        K = sh.K > K ? sh.K : K;
        smem = sh.smem > smem ? sh.smem : smem;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + sizeof(TileMeta) > (size_t)optin) return cudaErrorInvalidValue;
    std::vector<BatchItem> items;
    std::vector<int> ntiles;
    const int nitems = batch_items(g, n, tn.dw, items, ntiles);
    bl->kind = a0.kind;
    bl->fdt = a0.fdt;
    bl->cdt = a0.cdt;
    bl->K = K;
    bl->nf = tn.nf;
    bl->threads = tn.warps * 32;
    bl->smem = smem;
    bl->ngrids = n;
    bl->nitems = nitems;
    // workspace layout
    size_t off = 0;
    bl->off_grids = off;
    off += align256(gridargs_size(a0.fdt, a0.cdt) * n);
    bl->off_items = off;
    off += align256(sizeof(BatchItem) * (size_t)nitems);
    bl->off_ntiles = off;
    off += align256(sizeof(int) * (size_t)n);
    bl->off_parity = off;
    off += align256(sizeof(int) * (size_t)n);
    bl->off_counters = off;  // head, status, gdone[n], done[nitems + 1] (the extra flag is never set)
    bl->counter_bytes = sizeof(int) * (size_t)(2 + n + nitems + 1);
    off += align256(bl->counter_bytes);
    bl->bytes = off;
    bl->items = items;
    bl->ntiles = ntiles;
    return cudaSuccess;
}
#endif  // STG_BLOCKED_MAIN

template <typename TF, typename TC>
static cudaError_t batch_upload_t(const BatchGrid* g, int n, const BlockedTune& tn, BatchLaunch* bl, char* ws,
                                  cudaStream_t s) {
    std::vector<GridArgs<TF, TC>> ga(n);
    std::vector<int> par(n);
    for (int q = 0; q < n; ++q) {
        const int V = 16 / sizeof(TF);
        const int xt = ((g[q].a.L.nx + V - 1) / V) * V;
        BlockedTune t = tn;
        t.xtile = xt;
        BlkShape sh = blk_shape_x(g[q].a.kind, g[q].a.fdt, g[q].a.L.nx, tn.dw, tn.nf, tn.warps, xt);
        ga[q] = grid_args<TF, TC>(g[q].a, g[q].field, g[q].parity, g[q].T, t, sh);
        par[q] = g[q].parity;
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ws + bl->off_grids, ga.data(), sizeof(GridArgs<TF, TC>) * n, cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(ws + bl->off_items, bl->items.data(), sizeof(BatchItem) * bl->items.size(),
                             cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(ws + bl->off_ntiles, bl->ntiles.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(ws + bl->off_parity, par.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s))) return e;
    return cudaStreamSynchronize(s);  // host vectors are freed on return
}

#ifdef STG_BLOCKED_MAIN
cudaError_t batch_upload(const BatchGrid* g, int n, const BlockedTune& tn, BatchLaunch* bl, void* ws,
                         cudaStream_t s) {
    char* w = static_cast<char*>(ws);
    bl->ws = w;
    if (bl->fdt == DT_F64) return batch_upload_t<double, double>(g, n, tn, bl, w, s);
    if (bl->cdt == DT_BF16) return batch_upload_t<float, __nv_bfloat16>(g, n, tn, bl, w, s);
    return batch_upload_t<float, float>(g, n, tn, bl, w, s);
}
#endif  // STG_BLOCKED_MAIN

#ifdef STG_BLOCKED_MAIN
cudaError_t batch_reupload_items(BatchLaunch* bl, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(bl->ws + bl->off_items, bl->items.data(), sizeof(BatchItem) * bl->items.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e) return e;
    return cudaStreamSynchronize(s);
}
#endif  // STG_BLOCKED_MAIN

template <int KIND, typename TF, typename TC, int K, int NF>
static cudaError_t batch_launch_k(const BatchLaunch& bl, cudaStream_t s) {
    auto kfn = blocked_batch_kernel<KIND, TF, TC, K, NF>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bl.smem);
    if (e) return e;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, bl.threads, bl.smem);
    if (e) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    long long ctas = (long long)per * sms;
    if (ctas > bl.nitems) ctas = bl.nitems;
    if (ctas < 1) return cudaSuccess;
    BatchArgs<TF, TC> A{};
    char* ws = bl.ws;
    int* cnt = reinterpret_cast<int*>(ws + bl.off_counters);
    A.grids = reinterpret_cast<const GridArgs<TF, TC>*>(ws + bl.off_grids);
    A.items = reinterpret_cast<const BatchItem*>(ws + bl.off_items);
    A.nitems = bl.nitems;
    A.head = cnt;
    A.status = cnt + 1;
    A.gdone = cnt + 2;
    A.done = cnt + 2 + bl.ngrids;
    A.ntiles = reinterpret_cast<const int*>(ws + bl.off_ntiles);
    A.parity = reinterpret_cast<int*>(ws + bl.off_parity);
    A.spin_limit = bl.spin_limit;
    if ((e = cudaMemsetAsync(cnt, 0, bl.counter_bytes, s))) return e;
    kfn<<<(unsigned)ctas, bl.threads, bl.smem, s>>>(A);
    return cudaGetLastError();
}

template <int KIND, typename TF, typename TC>
cudaError_t batch_launch_t(const BatchLaunch& bl, cudaStream_t s) {
#define STG_BAT(KK, NFF) \
    if (bl.K == KK && bl.nf == NFF) return batch_launch_k<KIND, TF, TC, KK, NFF>(bl, s);
    STG_BAT(1, 1) STG_BAT(2, 1) STG_BAT(4, 1) STG_BAT(1, 2) STG_BAT(2, 2) STG_BAT(4, 2)
#undef STG_BAT
    return cudaErrorInvalidValue;
}

#ifdef STG_BLOCKED_MAIN
cudaError_t batch_launch(const BatchLaunch& bl, cudaStream_t s) {
    switch (bl.kind) {
        case K7C:
            if (bl.fdt == DT_F32) return batch_launch_t<K7C, float, float>(bl, s);
            if (bl.fdt == DT_F64) return batch_launch_t<K7C, double, double>(bl, s);
            break;
        case K7V:
            if (bl.fdt == DT_F32 && bl.cdt == DT_F32) return batch_launch_t<K7V, float, float>(bl, s);
            if (bl.fdt == DT_F32 && bl.cdt == DT_BF16) return batch_launch_t<K7V, float, __nv_bfloat16>(bl, s);
            if (bl.fdt == DT_F64) return batch_launch_t<K7V, double, double>(bl, s);
            break;
        case K25V:
            if (bl.fdt == DT_F32 && bl.cdt == DT_F32) return batch_launch_t<K25V, float, float>(bl, s);
            if (bl.fdt == DT_F32 && bl.cdt == DT_BF16) return batch_launch_t<K25V, float, __nv_bfloat16>(bl, s);
            if (bl.fdt == DT_F64) return batch_launch_t<K25V, double, double>(bl, s);
            break;
    }
    return cudaErrorInvalidValue;
}
#endif  // STG_BLOCKED_MAIN


// Row table of the persistent single-grid plan (rows whose tiles own no update are
// empty). false: more rows than one launch can carry.
static bool plan_rows(const SweepArgs& a, int T, int dw, PlanRows* P) {
    const int R = kind_radius(a.kind), Ny = a.L.ny;
    int n = 0, k = 0;
    for (;; ++k) {
        int tlo, thi;
        row_trange(dw, R, T, k, tlo, thi);
        if (tlo >= T) break;
        if (k >= MAXPROWS) return false;
        int bmin = 1 << 30, bmax = -(1 << 30);
        for (int b = -(k + 2) / 2 - 2; b <= (2 * Ny / dw - k) / 2 + 2; ++b) {
            bool any = false;
            for (int t = tlo; t < thi && !any; ++t) {
                int lo, hi;
                level_rows(dw, R, Ny, b + k, b, t, lo, hi);
                any = hi > lo;
            }
            if (any) {
                bmin = b < bmin ? b : bmin;
                bmax = b > bmax ? b : bmax;
            }
        }
        P->base[k] = n;
        P->bmin[k] = bmax >= bmin ? bmin : 0;
        if (bmax >= bmin) n += bmax - bmin + 1;
    }
    P->nrows = k;
    P->base[k] = n;
    P->nitems = n;
    return true;
}

// Persistent single-grid run. The workspace holds the status word, the never-set
// flag and one completion counter per tile (PERSIST_WS_* in internal.h). Returns
// cudaErrorNotReady when the plan does not fit one launch (more diamond rows than
// the parameter table holds, or more tiles than the workspace has counters for);
// the caller then runs T in parts.
template <int KIND, typename TF, typename TC, int K, int NF>
static cudaError_t persist_k(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                             const BlkShape& sh, void* ws, size_t ws_bytes, const PersistCtl& ctl, cudaStream_t st,
                             long long* launches) {
    PersistArgs<TF, TC> A{};
    if (!plan_rows(a, T, tn.dw, &A.P)) return cudaErrorNotReady;
    const int n = A.P.nitems;
    if (n == 0) return cudaSuccess;
    if (sizeof(int) * ((size_t)PERSIST_WS_DONE + n) > ws_bytes) return cudaErrorNotReady;
    auto kfn = blocked_persist_kernel<KIND, TF, TC, K, NF>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e) return e;
    const int nxt = sh.CX;
    if (nxt > 8 && (e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1))) return e;
    cudaLaunchConfig_t cfg{};
    cfg.blockDim = dim3((unsigned)(tn.warps * 32), 1, 1);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)nxt;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)nxt, 1, 1);
    int nclusters = 0;
    if (nxt > 1) {
        e = cudaOccupancyMaxActiveClusters(&nclusters, (void*)kfn, &cfg);
        if (e) return e;
    } else {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, tn.warps * 32, sh.smem))) return e;
        nclusters = per * sms;
    }
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    if (nclusters > n) nclusters = n;
    int* w = static_cast<int*>(ws);
    // the never-set flag and the completion counters start at 0; the status word is kept
    if ((e = cudaMemsetAsync(w + PERSIST_WS_NEVER, 0, sizeof(int) * (size_t)(PERSIST_WS_DONE - PERSIST_WS_NEVER + n),
                             st)))
        return e;
    A.G = grid_args<TF, TC>(a, field, p0, T, tn, sh);
    A.G.CX = nxt;
    A.status = w + PERSIST_WS_STATUS;
    A.never = w + PERSIST_WS_NEVER;
    A.done = w + PERSIST_WS_DONE;
    A.spin_limit = ctl.spin_limit;
    A.stall_item = ctl.stall_item;
    cfg.gridDim = dim3((unsigned)nxt, (unsigned)nclusters, 1);
    cfg.numAttrs = nxt > 1 ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kfn, A);
    if (e) return e;
    if (launches) *launches += 1;  // the library's kernels only (the counter reset is a memset)
    return cudaSuccess;
}

template <int KIND, typename TF, typename TC>
cudaError_t persist_t(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn, void* ws,
                      size_t ws_bytes, const PersistCtl& ctl, cudaStream_t st, long long* launches) {
    BlkShape sh = blk_shape(a, tn);
    if (!sh.ok) return cudaErrorInvalidValue;
#define STG_PER(KK, NFF) \
    if (sh.K == KK && tn.nf == NFF) \
        return persist_k<KIND, TF, TC, KK, NFF>(a, field, p0, T, tn, sh, ws, ws_bytes, ctl, st, launches);
    STG_PER(1, 1) STG_PER(2, 1) STG_PER(4, 1) STG_PER(1, 2) STG_PER(2, 2) STG_PER(4, 2)
#undef STG_PER
    return cudaErrorInvalidValue;
}

#ifdef STG_BLOCKED_MAIN
cudaError_t blocked_run_persistent(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                                   void* ws, size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s,
                                   long long* launches) {
    if (T <= 0 || a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) return persist_t<K7C, float, float>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            if (a.fdt == DT_F64) return persist_t<K7C, double, double>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32)
                return persist_t<K7V, float, float>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return persist_t<K7V, float, __nv_bfloat16>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            if (a.fdt == DT_F64) return persist_t<K7V, double, double>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32)
                return persist_t<K25V, float, float>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return persist_t<K25V, float, __nv_bfloat16>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            if (a.fdt == DT_F64) return persist_t<K25V, double, double>(a, field, p0, T, tn, ws, ws_bytes, ctl, s, launches);
            break;
    }
    return cudaErrorInvalidValue;
}
#endif  // STG_BLOCKED_MAIN

}  // namespace stg
