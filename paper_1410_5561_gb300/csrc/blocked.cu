// Temporally blocked sweep: diamond tiling in (y, t), wavefront along z,
// x split across the CTAs of a thread-block cluster.
//
// Paper: Section II-A (multicore wavefront diamond blocking, MWD): extruded
// diamonds in the (y, t) plane, traversed as a wavefront along z, with a group
// of threads sharing one cache block; "frontlines" N_F planes per level per
// wavefront step; Section III-A (leading-dimension tiling). The GPU version:
//
// * Tile geometry. With slope R per step and width D (a multiple of 2R),
//   update (y, t) (producing u_{t+1}(y)) belongs to tile (a, b) with
//   a = floor((y + R t) / D), b = floor((y - R t) / D). Row k = a - b holds
//   tiles that are mutually independent; tile (k, b) depends on (k-1, b) and
//   (k-1, b+1). Each row advances D/(2R) steps on average (Eq. 5's volume
//   N_z D^2 / (2R)). Rows run as successive launches on one stream, which is
//   the GPU counterpart of the paper's FIFO queue of ready diamonds.
// * One cluster of CX CTAs processes one tile for all z (the paper's thread
//   group). CTA c owns x in [c*Xt, (c+1)*Xt) and pushes its edge vectors into
//   its neighbours' rings through distributed shared memory.
// * Each time level l of the tile keeps a ring of Q = 2(N_F + R) planes in
//   shared memory holding u_{t_l} on rows N_l = Yc(t_l) +- R. Level l computes
//   planes [s N_F - l d, s N_F - l d + N_F) at step s with d = N_F + R, so all
//   levels of one step are independent and one cluster barrier per step
//   suffices.
// * HBM traffic is only the diamond boundary (Section III-C): rows of N_l not
//   computed by level l-1 are loaded from array (p0 + t_l) & 1 with cp.async;
//   an update is stored to array (p0 + t + 1) & 1 only if a point of another
//   tile reads it (or t = T-1). Coefficients are read through L2.
// * The per-point arithmetic is the shared update of common.cuh, so results
//   are bit-identical to the plain sweep.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace stg {

constexpr int MAXLV = 64;        // levels per tile (D/R - 1 <= 63)
constexpr int BLK_MAXT = 512;    // threads per CTA

struct TileMeta {
    int Lt, t0;
    int clo[MAXLV], chi[MAXLV];        // computed rows (interior), empty: clo == chi
    int nlo[MAXLV], nhi[MAXLV];        // ring rows [nlo, nhi) in [-R, Ny + R)
    int l0lo[MAXLV], l0hi[MAXLV];      // interior rows loaded from HBM, interval 0
    int l1lo[MAXLV], l1hi[MAXLV];      // interval 1
    int wlo[MAXLV], whi[MAXLV];        // computed rows NOT stored to HBM
    int roff[MAXLV];                   // ring element offset in shared memory
    int ipre[MAXLV + 1];               // prefix sums of computed rows
};

template <typename TF, typename TC>
struct BlkParams {
    Layout L;
    TF* f[2];
    const TC* C[13];
    TF c0, c1, halo;
    int p0, T, D, NF, row, bmin, Xt, CX, Q, Xs;
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
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int pmod(int a, int q) {
    int r = a % q;
    return r < 0 ? r + q : r;
}

template <int KIND, typename TF, typename TC>
__global__ void __launch_bounds__(BLK_MAXT, 1) blocked_kernel(const BlkParams<TF, TC> P) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int NC = KindTraits<KIND>::NC;
    constexpr int V = 16 / sizeof(TF);
    constexpr int J = (R + V - 1) / V;
    constexpr int HV = J * V;
    using VT = Vec<TF, V>;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ TileMeta M;
    TF* ring = reinterpret_cast<TF*>(smem_raw);

    const Layout& L = P.L;
    const int tid = threadIdx.x;
    const int NT = blockDim.x;
    const int NW = NT >> 5;
    const int warp = tid >> 5, lane = tid & 31;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = P.CX > 1 ? (int)cluster.block_rank() : 0;
    const int k = P.row;
    const int b = P.bmin + (int)blockIdx.y;
    const int a = b + k;
    const int D = P.D, NF = P.NF, Q = P.Q, Xs = P.Xs, Xt = P.Xt;
    const int d = NF + R;
    const int x0 = crank * Xt;
    const int Ny = L.ny, Nz = L.nz, Nx = L.nx;

    if (tid == 0) {
        int tlo, thi;
        row_trange(D, R, P.T, k, tlo, thi);
        int Lt = thi > tlo ? thi - tlo : 0;
        if (Lt > MAXLV) Lt = MAXLV;  // host guarantees D/R - 1 <= MAXLV
        M.Lt = Lt;
        M.t0 = tlo;
        int off = 0;
        M.ipre[0] = 0;
        for (int l = 0; l < Lt; ++l) {
            int lo, hi;
            level_rows(D, R, Ny, a, b, tlo + l, lo, hi);
            M.clo[l] = lo;
            M.chi[l] = hi;
            M.ipre[l + 1] = M.ipre[l] + (hi - lo);
            int nlo = 0, nhi = 0;
            if (hi > lo) {
                nlo = lo - R;
                nhi = hi + R;
            }
            M.nlo[l] = nlo;
            M.nhi[l] = nhi;
            M.roff[l] = off;
            off += Q * (nhi - nlo) * Xs;
            // interior rows of N_l that level l-1 does not compute
            int alo = nlo < 0 ? 0 : nlo, ahi = nhi > Ny ? Ny : nhi;
            if (ahi < alo) ahi = alo;
            int blo = 1 << 30, bhi = 1 << 30;
            if (l > 0 && M.chi[l - 1] > M.clo[l - 1]) {
                blo = M.clo[l - 1];
                bhi = M.chi[l - 1];
            }
            M.l0lo[l] = alo;
            M.l0hi[l] = ahi < blo ? ahi : blo;
            if (M.l0hi[l] < M.l0lo[l]) M.l0hi[l] = M.l0lo[l];
            M.l1lo[l] = alo > bhi ? alo : bhi;
            M.l1hi[l] = ahi;
            if (M.l1hi[l] < M.l1lo[l]) M.l1hi[l] = M.l1lo[l];
        }
        for (int l = 0; l < Lt; ++l) {
            int t = tlo + l;
            bool all = (t == P.T - 1) || (l + 1 >= Lt) || (M.chi[l + 1] <= M.clo[l + 1]);
            if (all) {
                M.wlo[l] = M.whi[l] = 0;
            } else {
                int c2lo = M.clo[l + 1], c2hi = M.chi[l + 1];
                M.wlo[l] = c2lo > 0 ? c2lo + R : 0;
                M.whi[l] = c2hi < Ny ? c2hi - R : Ny;
                if (M.whi[l] < M.wlo[l]) M.whi[l] = M.wlo[l];
            }
        }
    }
    __syncthreads();
    const int Lt = M.Lt;
    const TF hv = P.halo;

    // Outer x-halo columns of the cluster's end CTAs hold the Dirichlet value for good.
    if (crank == 0 || crank == P.CX - 1) {
        int totrows = 0;
        for (int l = 0; l < Lt; ++l) totrows += Q * (M.nhi[l] - M.nlo[l]);
        for (int i = tid; i < totrows * (2 * HV); i += NT) {
            int r = i / (2 * HV), c = i % (2 * HV);
            int col = c < HV ? c : Xt + c;  // [0,HV) or [HV+Xt, Xs)
            if ((c < HV && crank == 0) || (c >= HV && crank == P.CX - 1)) ring[(size_t)r * Xs + col] = hv;
        }
    }
    if (P.CX > 1) cluster.sync(); else __syncthreads();
    if (Lt == 0) return;

    // Work decomposition for the compute phase: G lanes per row (one vector each).
    const int G = Xt / V;
    const int nslots = NT / G;
    const int slot = tid / G;
    const int xv = tid - slot * G;
    const int xg = x0 + xv * V;  // interior x of this lane's vector element 0
    const int totitems = M.ipre[Lt];

    const int s_begin = -((2 * R + NF + NF - 1) / NF);
    const int s_end = (Nz - 1 + (Lt - 1) * d) / NF + 1;

    // global vector range to load: [x0 - HV, min(x0 + Xt + HV, roundup(Nx, V) + HV))
    const int xend = ((Nx + V - 1) / V) * V + HV;
    const int lv_hi = (min(x0 + Xt + HV, xend) - (x0 - HV)) / V;  // vectors per loaded row

    for (int s = s_begin; s < s_end; ++s) {
        // ---------------- producer: HBM loads and Dirichlet fills (one warp per row)
        {
            int g = 0;
            for (int l = 0; l < Lt; ++l) {
                const int nlo = M.nlo[l], nhi = M.nhi[l];
                if (nhi <= nlo) continue;
                const int nrows = nhi - nlo;
                TF* rb = ring + M.roff[l];
                const TF* src = P.f[(P.p0 + M.t0 + l) & 1];
                const int zb = s * NF - l * d + NF + R;
                for (int f = 0; f < NF; ++f) {
                    const int z = zb + f;
                    if (z < -R || z >= Nz + R) continue;
                    const bool hplane = (z < 0 || z >= Nz);
                    const int n0 = M.l0hi[l] - M.l0lo[l], n1 = M.l1hi[l] - M.l1lo[l];
                    const int hlo = nlo < 0 ? -nlo : 0;            // halo rows below 0: [nlo, 0)
                    const int hhi = nhi > Ny ? nhi - Ny : 0;       // halo rows at/after Ny
                    const int cnt = hplane ? nrows : (n0 + n1 + hlo + hhi);
                    TF* slotb = rb + (size_t)pmod(z, Q) * nrows * Xs;
                    int i0 = pmod(warp - g, NW);
                    for (int i = i0; i < cnt; i += NW) {
                        int y;
                        bool fill;
                        if (hplane) {
                            y = nlo + i;
                            fill = true;
                        } else if (i < n0) {
                            y = M.l0lo[l] + i;
                            fill = false;
                        } else if (i < n0 + n1) {
                            y = M.l1lo[l] + (i - n0);
                            fill = false;
                        } else if (i < n0 + n1 + hlo) {
                            y = nlo + (i - n0 - n1);
                            fill = true;
                        } else {
                            y = Ny + (i - n0 - n1 - hlo);
                            fill = true;
                        }
                        TF* rowp = slotb + (size_t)(y - nlo) * Xs;
                        if (fill) {
                            VT hvv;
#pragma unroll
                            for (int e = 0; e < V; ++e) hvv.v[e] = hv;
                            for (int c = lane; c < Xs / V; c += 32) stv<TF, V>(rowp + c * V, hvv);
                        } else {
                            const TF* gp = src + L.at(x0 - HV, y, z);
                            for (int c = lane; c < lv_hi; c += 32) cp_async16(rowp + c * V, gp + c * V);
                        }
                    }
                    g += cnt;
                }
            }
        }
        // ---------------- compute: items (level, row), N_F planes each
        if (slot < nslots) {
            int l = 0;
            for (int it = slot; it < totitems; it += nslots) {
                while (it >= M.ipre[l + 1]) ++l;
                const int y = M.clo[l] + (it - M.ipre[l]);
                const int zb = s * NF - l * d;
                if (zb + NF <= 0 || zb >= Nz) continue;
                const int nlo = M.nlo[l];
                const int nrows = M.nhi[l] - nlo;
                const TF* rb = ring + M.roff[l];
                const int t = M.t0 + l;
                // destination ring (level l+1), if it holds row y
                TF* rdst = nullptr;
                int dnlo = 0, dnrows = 0;
                if (l + 1 < Lt && y >= M.nlo[l + 1] && y < M.nhi[l + 1]) {
                    rdst = ring + M.roff[l + 1];
                    dnlo = M.nlo[l + 1];
                    dnrows = M.nhi[l + 1] - dnlo;
                }
                const bool store = !(y >= M.wlo[l] && y < M.whi[l]);
                TF* gdst = P.f[(P.p0 + t + 1) & 1];
                auto at = [&](int z, int yy, int col) -> const TF* {
                    return rb + ((size_t)pmod(z, Q) * nrows + (yy - nlo)) * Xs + col;
                };
                const int col = HV + xv * V;
                VT zr[2 * R + 1];
                const int zfirst = zb < 0 ? 0 : zb;
                const int zlast = (zb + NF < Nz ? zb + NF : Nz);
#pragma unroll
                for (int r = 0; r < 2 * R; ++r) zr[r] = ldv<TF, V>(at(zfirst - R + r, y, col));
                for (int z = zfirst; z < zlast; ++z) {
                    zr[2 * R] = ldv<TF, V>(at(z + R, y, col));
                    TF xl[(2 * J + 1) * V];
#pragma unroll
                    for (int q = -J; q <= J; ++q) {
                        VT w = (q == 0) ? zr[R] : ldv<TF, V>(at(z, y, col + q * V));
#pragma unroll
                        for (int e = 0; e < V; ++e) xl[(q + J) * V + e] = w.v[e];
                    }
                    VT ypv[R], ymv[R];
#pragma unroll
                    for (int r = 1; r <= R; ++r) {
                        ypv[r - 1] = ldv<TF, V>(at(z, y + r, col));
                        ymv[r - 1] = ldv<TF, V>(at(z, y - r, col));
                    }
                    const size_t gidx = L.at(xg, y, z);
                    Vec<TC, V> cv[NC > 0 ? NC : 1];
                    if constexpr (NC > 0) {
                        if (xg < Nx) {
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
                        TF r_;
                        if constexpr (KIND == K7C) {
                            r_ = upd7c<TF>(P.c0, P.c1, zr[R].v[e], xl[xc + 1], xl[xc - 1], ypv[0].v[e],
                                           ymv[0].v[e], zr[R + 1].v[e], zr[R - 1].v[e]);
                        } else if constexpr (KIND == K7V) {
                            TF c[7];
#pragma unroll
                            for (int m = 0; m < 7; ++m) c[m] = Cvt<TF, TC>::f(cv[m].v[e]);
                            r_ = upd7v<TF>(c, zr[R].v[e], xl[xc + 1], xl[xc - 1], ypv[0].v[e], ymv[0].v[e],
                                           zr[R + 1].v[e], zr[R - 1].v[e]);
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
                                zp[q] = zr[R + q + 1].v[e];
                                zm[q] = zr[R - q - 1].v[e];
                            }
                            r_ = upd25v<TF>(c, zr[R].v[e], xp, xm, yp4, ym4, zp, zm);
                        }
                        out.v[e] = (xg + e < Nx) ? r_ : hv;
                    }
                    if (rdst) {
                        TF* dp = rdst + ((size_t)pmod(z, Q) * dnrows + (y - dnlo)) * Xs;
                        stv<TF, V>(dp + col, out);
                        if (P.CX > 1) {
                            if (xv < J && crank > 0) {
                                TF* rp = cluster.map_shared_rank(dp + HV + Xt + xv * V, crank - 1);
                                stv<TF, V>(rp, out);
                            }
                            if (xv >= G - J && crank < P.CX - 1) {
                                TF* rp = cluster.map_shared_rank(dp + (xv - (G - J)) * V, crank + 1);
                                stv<TF, V>(rp, out);
                            }
                        }
                    }
                    if (store && xg < Nx) {
                        if (xg + V <= Nx) {
                            stv<TF, V>(gdst + gidx, out);
                        } else {
#pragma unroll
                            for (int e = 0; e < V; ++e)
                                if (xg + e < Nx) gdst[gidx + e] = out.v[e];
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 2 * R; ++r) zr[r] = zr[r + 1];
                }
            }
        }
        cp_async_wait_all();
        if (P.CX > 1) cluster.sync(); else __syncthreads();
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

struct BlkShape {
    int V, HV, Xt, Xs, Q, G;
    size_t smem;
    bool ok;
};

static BlkShape blk_shape(const SweepArgs& a, const BlockedTune& tn) {
    BlkShape s{};
    int R = kind_radius(a.kind);
    int eb = dtype_bytes(a.fdt);
    s.V = 16 / eb;
    int J = (R + s.V - 1) / s.V;
    s.HV = J * s.V;
    s.ok = false;
    if (tn.dw < 2 * R || tn.dw % (2 * R) != 0 || tn.nf < 1 || tn.cx < 1 || tn.cx > 16) return s;
    if (tn.dw / R - 1 > MAXLV) return s;
    if (tn.warps < 1 || tn.warps * 32 > BLK_MAXT) return s;
    int per = (a.L.nx + tn.cx - 1) / tn.cx;
    s.Xt = ((per + s.V - 1) / s.V) * s.V;
    if (s.Xt < s.HV) s.Xt = s.HV;
    s.G = s.Xt / s.V;
    if (s.G > tn.warps * 32) return s;
    s.Xs = s.Xt + 2 * s.HV;
    s.Q = 2 * (tn.nf + R);
    s.smem = (size_t)s.Q * ring_rows_bound(tn.dw, R) * s.Xs * eb;
    s.ok = true;
    return s;
}

size_t blocked_smem_bytes(const SweepArgs& a, const BlockedTune& tn) {
    BlkShape s = blk_shape(a, tn);
    if (!s.ok) return 0;
    return s.smem + sizeof(TileMeta);
}

template <int KIND, typename TF, typename TC>
static cudaError_t launch_blocked(const SweepArgs& a, void* const field[2], int p0, int T,
                                  const BlockedTune& tn, cudaStream_t st) {
    const int R = KindTraits<KIND>::R;
    BlkShape sh = blk_shape(a, tn);
    if (!sh.ok) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sh.smem + sizeof(TileMeta) > (size_t)optin) return cudaErrorInvalidValue;
    auto kfn = blocked_kernel<KIND, TF, TC>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e != cudaSuccess) return e;
    if (tn.cx > 8) {
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    BlkParams<TF, TC> P{};
    P.L = a.L;
    P.f[0] = static_cast<TF*>(field[0]);
    P.f[1] = static_cast<TF*>(field[1]);
    for (int m = 0; m < KindTraits<KIND>::NC; ++m) P.C[m] = static_cast<const TC*>(a.coef[m]);
    P.c0 = (TF)a.c0;
    P.c1 = (TF)a.c1;
    P.halo = (TF)a.halo;
    P.p0 = p0;
    P.T = T;
    P.D = tn.dw;
    P.NF = tn.nf;
    P.Xt = sh.Xt;
    P.CX = tn.cx;
    P.Q = sh.Q;
    P.Xs = sh.Xs;
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
        cfg.gridDim = dim3((unsigned)tn.cx, (unsigned)(bmax - bmin + 1), 1);
        cfg.blockDim = dim3((unsigned)(tn.warps * 32), 1, 1);
        cfg.dynamicSmemBytes = sh.smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)tn.cx;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kfn, P);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t blocked_run(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tn,
                        cudaStream_t s) {
    if (T <= 0 || a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    switch (a.kind) {
        case K7C:
            if (a.fdt == DT_F32) return launch_blocked<K7C, float, float>(a, field, p0, T, tn, s);
            if (a.fdt == DT_F64) return launch_blocked<K7C, double, double>(a, field, p0, T, tn, s);
            break;
        case K7V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) return launch_blocked<K7V, float, float>(a, field, p0, T, tn, s);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_blocked<K7V, float, __nv_bfloat16>(a, field, p0, T, tn, s);
            if (a.fdt == DT_F64) return launch_blocked<K7V, double, double>(a, field, p0, T, tn, s);
            break;
        case K25V:
            if (a.fdt == DT_F32 && a.cdt == DT_F32) return launch_blocked<K25V, float, float>(a, field, p0, T, tn, s);
            if (a.fdt == DT_F32 && a.cdt == DT_BF16)
                return launch_blocked<K25V, float, __nv_bfloat16>(a, field, p0, T, tn, s);
            if (a.fdt == DT_F64) return launch_blocked<K25V, double, double>(a, field, p0, T, tn, s);
            break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace stg
