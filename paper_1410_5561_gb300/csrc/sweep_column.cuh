// One thread's share of a one-step sweep: the updates of one column of V
// consecutive x values (one 128-bit vector) at row j, planes [k0, k1), from
// array src into array dst (Listings 1-3 through the shared update functions of
// common.cuh, so every schedule that uses it is bit-identical to the others).
//
// The thread keeps the 2R+1 planes of its column in a register ring, so each
// z-neighbour is loaded once, plus PF planes loaded ahead so that several loads
// per thread are in flight. x- and y-neighbours are plain aligned vector loads
// that hit L1/L2 (the neighbouring threads read them too). Coefficients are
// read once per update: with COEF_STREAM through evict-first loads (the plain
// sweep, which never reads them again), otherwise through the read-only path
// with the default L2 policy (the wavefront schedule, whose next time level
// reads the same planes soon after, from L2).
//
// With COHERENT the field is read with explicit weak global loads (never the
// read-only path the compiler may pick for a const __restrict__ pointer): in the
// wavefront schedule other CTAs of the same launch write src, and a CTA reads
// it only after acquiring their completion flags.
#pragma once
#include "internal.h"

namespace stg {

template <typename TC>
struct CoefPtrs {
    const TC* c[13];
};

// Field vector load: coherent (COH: ld.global, L1-cacheable; volatile so that it is never
// moved above the barrier that follows a dependency wait) or unconstrained.
template <bool COH, typename T, int V> struct FieldLd {
    static __device__ __forceinline__ Vec<T, V> ld(const T* p) { return ldv<T, V>(p); }
};
template <> struct FieldLd<true, float, 4> {
    static __device__ __forceinline__ Vec<float, 4> ld(const float* p) {
        Vec<float, 4> r;
        asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(p));
        return r;
    }
};
template <> struct FieldLd<true, double, 2> {
    static __device__ __forceinline__ Vec<double, 2> ld(const double* p) {
        Vec<double, 2> r;
        asm volatile("ld.global.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p));
        return r;
    }
};

// The column walk as a resumable state: begin() loads the planes below the first
// plane, plane() updates the next plane (planes in increasing order, starting at
// begin's k0; no plane at or beyond k1 is loaded). Loads reach R + PF planes above
// the plane being updated.
template <int KIND, typename TF, typename TC, int PF, bool COEF_STREAM, bool COHERENT>
struct Column {
    static constexpr int R = KindTraits<KIND>::R;
    static constexpr int NC = KindTraits<KIND>::NC;
    static constexpr int V = 16 / sizeof(TF);
    static constexpr int J = (R + V - 1) / V;  // neighbour vectors needed on each side along x
    Vec<TF, V> ring[2 * R + 1];                 // planes k-R .. k+R of this thread's column
    Vec<TF, V> ahead[PF > 0 ? PF : 1];          // planes k+R .. k+R+PF-1 (loaded while k - 1 computes)
    size_t base;                                // element index of (i0, j, k)
    int k1;

    __device__ __forceinline__ void begin(const Layout& L, const TF* __restrict__ src, int i0, int j, int k0,
                                          int k1_) {
        const size_t sz = L.plane();
        base = L.at(i0, j, k0);
        k1 = k1_;
#pragma unroll
        for (int r = 0; r < 2 * R; ++r) ring[r] = FieldLd<COHERENT, TF, V>::ld(src + base + (ptrdiff_t)(r - R) * (ptrdiff_t)sz);
#pragma unroll
        for (int p = 0; p < PF; ++p)
            if (k0 + p < k1) ahead[p] = FieldLd<COHERENT, TF, V>::ld(src + base + (size_t)(R + p) * sz);
    }

    __device__ __forceinline__ void plane(const Layout& L, const TF* __restrict__ src, TF* __restrict__ dst,
                                          const CoefPtrs<TC>& C, TF c0, TF c1, int i0, int k) {
        const size_t sy = (size_t)L.px;
        const size_t sz = L.plane();
        if constexpr (PF > 0) {
            ring[2 * R] = ahead[0];
#pragma unroll
            for (int p = 0; p + 1 < PF; ++p) ahead[p] = ahead[p + 1];
            // plane k+R+PF exists (interior or upper halo) while k + PF <= nz - 1
            if (k + PF < k1) ahead[PF - 1] = FieldLd<COHERENT, TF, V>::ld(src + base + (size_t)(R + PF) * sz);
        } else {
            ring[2 * R] = FieldLd<COHERENT, TF, V>::ld(src + base + (size_t)R * sz);
        }
        // x line around the vector: [i0 - J*V, i0 + (J+1)*V)
        TF xl[(2 * J + 1) * V];
#pragma unroll
        for (int q = -J; q <= J; ++q) {
            Vec<TF, V> w = (q == 0) ? ring[R] : FieldLd<COHERENT, TF, V>::ld(src + base + (ptrdiff_t)q * V);
#pragma unroll
            for (int e = 0; e < V; ++e) xl[(q + J) * V + e] = w.v[e];
        }
        Vec<TF, V> yp[R], ym[R];
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            yp[r - 1] = FieldLd<COHERENT, TF, V>::ld(src + base + (size_t)r * sy);
            ym[r - 1] = FieldLd<COHERENT, TF, V>::ld(src + base - (size_t)r * sy);
        }
        Vec<TC, V> cv[NC > 0 ? NC : 1];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            if constexpr (COEF_STREAM) cv[m] = ldv_stream<TC, V>(C.c[m] + base);
            else cv[m] = ldv_ro<TC, V>(C.c[m] + base);
        }

        Vec<TF, V> out;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int xc = J * V + e;
            if constexpr (KIND == K7C) {
                out.v[e] = upd7c<TF>(c0, c1, ring[R].v[e], xl[xc + 1], xl[xc - 1], yp[0].v[e],
                                     ym[0].v[e], ring[R + 1].v[e], ring[R - 1].v[e]);
            } else if constexpr (KIND == K7V) {
                TF c[7];
#pragma unroll
                for (int m = 0; m < 7; ++m) c[m] = Cvt<TF, TC>::f(cv[m].v[e]);
                out.v[e] = upd7v<TF>(c, ring[R].v[e], xl[xc + 1], xl[xc - 1], yp[0].v[e], ym[0].v[e],
                                     ring[R + 1].v[e], ring[R - 1].v[e]);
            } else {
                TF c[13], xp[4], xm[4], ypp[4], ymm[4], zp[4], zm[4];
#pragma unroll
                for (int m = 0; m < 13; ++m) c[m] = Cvt<TF, TC>::f(cv[m].v[e]);
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    xp[d] = xl[xc + d + 1];
                    xm[d] = xl[xc - d - 1];
                    ypp[d] = yp[d].v[e];
                    ymm[d] = ym[d].v[e];
                    zp[d] = ring[R + d + 1].v[e];
                    zm[d] = ring[R - d - 1].v[e];
                }
                out.v[e] = upd25v<TF>(c, ring[R].v[e], xp, xm, ypp, ymm, zp, zm);
            }
        }
        if (i0 + V <= L.nx) {
            stv<TF, V>(dst + base, out);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (i0 + e < L.nx) dst[base + e] = out.v[e];
        }
#pragma unroll
        for (int r = 0; r < 2 * R; ++r) ring[r] = ring[r + 1];
        base += sz;
    }
};

template <int KIND, typename TF, typename TC, int PF, bool COEF_STREAM, bool COHERENT = false>
__device__ __forceinline__ void sweep_column(const Layout& L, const TF* __restrict__ src, TF* __restrict__ dst,
                                             const CoefPtrs<TC>& C, TF c0, TF c1, int i0, int j, int k0, int k1) {
    Column<KIND, TF, TC, PF, COEF_STREAM, COHERENT> col;
    col.begin(L, src, i0, j, k0, k1);
    for (int k = k0; k < k1; ++k) col.plane(L, src, dst, C, c0, c1, i0, k);
}

}  // namespace stg
