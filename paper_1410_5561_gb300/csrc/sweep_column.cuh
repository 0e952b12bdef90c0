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

// Per-thread asynchronous copy of one coefficient vector into shared memory (16 bytes through
// L2 only, or 8 bytes for a BF16 vector), and the group bookkeeping.
template <int BYTES> struct CoefCp;
template <> struct CoefCp<16> {
    static __device__ __forceinline__ void cp(uint32_t s, const void* g) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
    }
};
template <> struct CoefCp<8> {
    static __device__ __forceinline__ void cp(uint32_t s, const void* g) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
    }
};
__device__ __forceinline__ void coef_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void coef_cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// Shared-memory vector load of the field type.
template <typename TF, int V> struct Lds16;
template <> struct Lds16<float, 4> {
    static __device__ __forceinline__ Vec<float, 4> ld(uint32_t a) {
        Vec<float, 4> r;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "r"(a) : "memory");
        return r;
    }
};
template <> struct Lds16<double, 2> {
    static __device__ __forceinline__ Vec<double, 2> ld(uint32_t a) {
        Vec<double, 2> r;
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.v[0]), "=d"(r.v[1]) : "r"(a) : "memory");
        return r;
    }
};
template <typename TC, int V> struct CoefLds;
template <> struct CoefLds<float, 4> {
    static __device__ __forceinline__ Vec<float, 4> ld(uint32_t a) {
        Vec<float, 4> r;
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                     : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "r"(a) : "memory");
        return r;
    }
};
template <> struct CoefLds<double, 2> {
    static __device__ __forceinline__ Vec<double, 2> ld(uint32_t a) {
        Vec<double, 2> r;
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(r.v[0]), "=d"(r.v[1]) : "r"(a) : "memory");
        return r;
    }
};
template <> struct CoefLds<__nv_bfloat16, 4> {
    static __device__ __forceinline__ Vec<__nv_bfloat16, 4> ld(uint32_t a) {
        uint2 u;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];\n" : "=r"(u.x), "=r"(u.y) : "r"(a) : "memory");
        Vec<__nv_bfloat16, 4> r;
        memcpy(&r, &u, sizeof(r));
        return r;
    }
};

// The column walk as a resumable state: begin() loads the planes below the first
// plane, plane() updates the next plane (planes in increasing order, starting at
// begin's k0; no plane at or beyond k1 is loaded). Loads reach R + PF planes above
// the plane being updated.
//
// With CP > 0 the coefficient vectors of the next CP planes are copied ahead, by this thread,
// into its own slots of a shared-memory ring (cslot: shared address of the thread's slot for
// ring position 0 and array 0; cstep: bytes between consecutive (position, array) slots), so
// the copies in flight hold shared memory instead of registers. Each thread reads only the
// slots it filled, after its own cp.async.wait_group: no CTA barrier is needed.
template <int KIND, typename TF, typename TC, int PF, bool COEF_STREAM, bool COHERENT, int CP = 0>
struct Column {
    static constexpr int R = KindTraits<KIND>::R;
    static constexpr int NC = KindTraits<KIND>::NC;
    static constexpr int V = 16 / sizeof(TF);
    static constexpr int J = (R + V - 1) / V;  // neighbour vectors needed on each side along x
    static constexpr int CB = (int)sizeof(Vec<TC, V>);  // bytes of one coefficient vector
    Vec<TF, V> ring[2 * R + 1];                 // planes k-R .. k+R of this thread's column
    Vec<TF, V> ahead[PF > 0 ? PF : 1];          // planes k+R .. k+R+PF-1 (loaded while k - 1 computes)
    size_t base;                                // element index of (i0, j, k)
    int k1;
    uint32_t cslot, cstep;                      // coefficient ring (CP > 0)
    int cpos;                                   // ring position of the plane being updated

    // copies of the coefficient vectors of plane kk (element index b) into ring position pos
    __device__ __forceinline__ void coef_fetch(const CoefPtrs<TC>& C, size_t b, int pos) {
#pragma unroll
        for (int m = 0; m < NC; ++m)
            CoefCp<CB>::cp(cslot + (uint32_t)(pos * NC + m) * cstep, C.c[m] + b);
    }

    __device__ __forceinline__ void begin_coef(const Layout& L, const CoefPtrs<TC>& C, uint32_t cslot_,
                                               uint32_t cstep_, int k0) {
        cslot = cslot_;
        cstep = cstep_;
        cpos = 0;
        if constexpr (CP > 0) {
#pragma unroll
            for (int p = 0; p < CP; ++p) {
                if (k0 + p < k1) coef_fetch(C, base + (size_t)p * L.plane(), p);
                coef_cp_commit();
            }
        }
    }

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
        if constexpr (CP > 0) {
            coef_cp_wait<CP - 1>();  // this thread's copies of plane k have landed
#pragma unroll
            for (int m = 0; m < NC; ++m) cv[m] = CoefLds<TC, V>::ld(cslot + (uint32_t)(cpos * NC + m) * cstep);
        } else {
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                if constexpr (COEF_STREAM) cv[m] = ldv_stream<TC, V>(C.c[m] + base);
                else cv[m] = ldv_ro<TC, V>(C.c[m] + base);
            }
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
        if constexpr (CP > 0) {
            // refill the position just read (its values are consumed) with plane k + CP
            if (k + CP < k1) coef_fetch(C, base + (size_t)CP * sz, cpos);
            coef_cp_commit();
            cpos = cpos + 1 == CP ? 0 : cpos + 1;
        }
        base += sz;
    }
};


// The column walk with every load of a plane copied ahead: each thread copies, D planes ahead,
// the vectors its update of plane k reads (the new z plane k+R, the x-neighbour vectors, the
// y-neighbour rows at distance 1..R, the n_c coefficient vectors) into its own slots of a
// shared-memory ring, with cp.async (field through L1, coefficients through L2 only). A plane
// then waits only for its own copies, issued D planes earlier, instead of a full memory latency,
// and the copies in flight hold shared memory, not registers. No CTA barrier is needed: a
// thread reads only the slots it filled. Loads reach plane k + D + R at most.
// Shared memory per thread: D x (SF x 16 + n_c x sizeof(coefficient vector)) bytes, SF = 1 + 2J + 2R.
template <int KIND, typename TF, typename TC, bool COEF_STREAM, int D>
struct ColumnAsync {
    static constexpr int R = KindTraits<KIND>::R;
    static constexpr int NC = KindTraits<KIND>::NC;
    static constexpr int V = 16 / sizeof(TF);
    static constexpr int J = (R + V - 1) / V;
    static constexpr int SF = 1 + 2 * J + 2 * R;  // field vectors per plane: z new, x -J..-1, 1..J, y -R..-1, 1..R
    static constexpr int CB = (int)sizeof(Vec<TC, V>);
    static_assert(D >= 1, "prefetch depth");
    Vec<TF, V> ring[2 * R + 1];
    size_t base;
    int k1, pos;
    uint32_t fslot, fstep, cslot, cstep;  // shared addresses: this thread's slot (position 0, vector 0); strides

    __device__ __forceinline__ void fetch(const Layout& L, const TF* src, const CoefPtrs<TC>& C, size_t b, int p) {
        const size_t sy = (size_t)L.px, sz = L.plane();
        const uint32_t f0 = fslot + (uint32_t)(p * SF) * fstep;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(f0), "l"(src + b + (size_t)R * sz) : "memory");
#pragma unroll
        for (int q = 1; q <= J; ++q) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(f0 + (uint32_t)(2 * q - 1) * fstep),
                         "l"(src + b - (ptrdiff_t)q * V) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(f0 + (uint32_t)(2 * q) * fstep),
                         "l"(src + b + (ptrdiff_t)q * V) : "memory");
        }
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(f0 + (uint32_t)(2 * J + 2 * r - 1) * fstep),
                         "l"(src + b - (size_t)r * sy) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(f0 + (uint32_t)(2 * J + 2 * r) * fstep),
                         "l"(src + b + (size_t)r * sy) : "memory");
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) CoefCp<CB>::cp(cslot + (uint32_t)(p * NC + m) * cstep, C.c[m] + b);
    }

    __device__ __forceinline__ void begin(const Layout& L, const TF* __restrict__ src, const CoefPtrs<TC>& C, int i0,
                                          int j, int k0, int k1_, uint32_t fslot_, uint32_t fstep_, uint32_t cslot_,
                                          uint32_t cstep_) {
        const size_t sz = L.plane();
        base = L.at(i0, j, k0);
        k1 = k1_;
        pos = 0;
        fslot = fslot_;
        fstep = fstep_;
        cslot = cslot_;
        cstep = cstep_;
#pragma unroll
        for (int r = 0; r < 2 * R; ++r)
            ring[r] = FieldLd<true, TF, V>::ld(src + base + (ptrdiff_t)(r - R) * (ptrdiff_t)sz);
#pragma unroll
        for (int p = 0; p < D; ++p) {
            if (k0 + p < k1) fetch(L, src, C, base + (size_t)p * sz, p);
            coef_cp_commit();
        }
    }

    __device__ __forceinline__ void plane(const Layout& L, const TF* __restrict__ src, TF* __restrict__ dst,
                                          const CoefPtrs<TC>& C, TF c0, TF c1, int i0, int k) {
        const size_t sz = L.plane();
        coef_cp_wait<D - 1>();  // this thread's copies for plane k have landed
        const uint32_t f0 = fslot + (uint32_t)(pos * SF) * fstep;
        ring[2 * R] = Lds16<TF, V>::ld(f0);
        TF xl[(2 * J + 1) * V];
#pragma unroll
        for (int e = 0; e < V; ++e) xl[J * V + e] = ring[R].v[e];
#pragma unroll
        for (int q = 1; q <= J; ++q) {
            const Vec<TF, V> a = Lds16<TF, V>::ld(f0 + (uint32_t)(2 * q - 1) * fstep);
            const Vec<TF, V> b = Lds16<TF, V>::ld(f0 + (uint32_t)(2 * q) * fstep);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                xl[(J - q) * V + e] = a.v[e];
                xl[(J + q) * V + e] = b.v[e];
            }
        }
        Vec<TF, V> yp[R], ym[R];
#pragma unroll
        for (int r = 1; r <= R; ++r) {
            ym[r - 1] = Lds16<TF, V>::ld(f0 + (uint32_t)(2 * J + 2 * r - 1) * fstep);
            yp[r - 1] = Lds16<TF, V>::ld(f0 + (uint32_t)(2 * J + 2 * r) * fstep);
        }
        Vec<TC, V> cv[NC > 0 ? NC : 1];
#pragma unroll
        for (int m = 0; m < NC; ++m) cv[m] = CoefLds<TC, V>::ld(cslot + (uint32_t)(pos * NC + m) * cstep);
        Vec<TF, V> out;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int xc = J * V + e;
            if constexpr (KIND == K7C) {
                out.v[e] = upd7c<TF>(c0, c1, ring[R].v[e], xl[xc + 1], xl[xc - 1], yp[0].v[e], ym[0].v[e],
                                     ring[R + 1].v[e], ring[R - 1].v[e]);
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
        // refill the position just read (its values are consumed) with plane k + D
        if (k + D < k1) fetch(L, src, C, base + (size_t)D * sz, pos);
        coef_cp_commit();
        pos = pos + 1 == D ? 0 : pos + 1;
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
