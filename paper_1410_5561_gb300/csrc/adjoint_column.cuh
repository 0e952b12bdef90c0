// One thread's share of a transposed step of the variable-coefficient stencils
// (the adjoint's cotangent recursion lambda_t = A^T lambda_{t+1}, Listings 2 and 3):
// the V points of one 128-bit vector at row j, planes [k0, k1).
//
//   (A^T l)(q) = C0(q) l(q) + sum over d = 1..R and axis a of
//                C_minus(q - d e_a) l(q - d e_a) + C_plus(q + d e_a) l(q + d e_a)
//
// where C_minus / C_plus are the arrays that weigh the +/- neighbour in the forward
// update (7-point: C(2a+1) weighs p + e_a and C(2a+2) weighs p - e_a, so the point
// q - e_a reaches q through C(2a+1); 25-point: the axis coefficient weighs both
// sides). The terms are summed in this order with explicitly rounded operations, so
// every schedule that uses this function gives the same bits. Zero halos in lambda
// and in the coefficient arrays make the "p is interior" condition of the
// transpose automatic.
//
// With COHERENT lambda is read with explicit weak global loads (other CTAs of the
// same launch write it in the wavefront schedule); otherwise through the read-only
// path. Coefficients are read-only for the whole launch either way.
#pragma once
#include "internal.h"
#include "sweep_column.cuh"

namespace stg {

template <int KIND>
struct AdjSides {
    // coefficient arrays weighing the minus and plus neighbour of axis a at distance d
    static __device__ __forceinline__ int minus(int d, int a) { return KIND == K7V ? 1 + 2 * a : 3 * (d - 1) + a + 1; }
    static __device__ __forceinline__ int plus(int d, int a) { return KIND == K7V ? 2 + 2 * a : 3 * (d - 1) + a + 1; }
};

template <bool COH, typename T, int V>
__device__ __forceinline__ Vec<T, V> lam_ld(const T* p) {
    if constexpr (COH) return FieldLd<true, T, V>::ld(p);
    else return ldv_ro<T, V>(p);
}

template <int KIND, typename TF, typename TC, bool COHERENT>
__device__ __forceinline__ void lambda_column(const Layout& L, const TF* __restrict__ lam_in,
                                              TF* __restrict__ lam_out, const CoefPtrs<TC>& C, int i0, int j, int k0,
                                              int k1) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int V = 16 / sizeof(TF);
    constexpr int J = (R + V - 1) / V;  // neighbour vectors on each side along x
    constexpr int XL = (2 * J + 1) * V;
    using A = Ar<TF>;
    using SD = AdjSides<KIND>;
    const size_t sy = (size_t)L.px, sz = L.plane();
    const bool full = i0 + V <= L.nx;
    for (int k = k0; k < k1; ++k) {
        const size_t p = L.at(i0, j, k);
        TF lx[XL];  // x line around the vector: [i0 - J V, i0 + (J + 1) V)
#pragma unroll
        for (int q = -J; q <= J; ++q) {
            const Vec<TF, V> wl = lam_ld<COHERENT, TF, V>(lam_in + p + (ptrdiff_t)q * V);
#pragma unroll
            for (int e = 0; e < V; ++e) lx[(q + J) * V + e] = wl.v[e];
        }
        TF r[V];
        {
            const Vec<TC, V> c0 = ldv_ro<TC, V>(C.c[0] + p);
#pragma unroll
            for (int e = 0; e < V; ++e) r[e] = A::mul(Cvt<TF, TC>::f(c0.v[e]), lx[J * V + e]);
        }
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            // x: coefficient lines of the two arrays at this distance
            {
                const TC* cm = C.c[SD::minus(d, 0)];
                const TC* cpl = C.c[SD::plus(d, 0)];
                TF cxm[XL], cxp[XL];
#pragma unroll
                for (int q = -J; q <= J; ++q) {
                    const Vec<TC, V> a = ldv_ro<TC, V>(cm + p + (ptrdiff_t)q * V);
                    const Vec<TC, V> b = ldv_ro<TC, V>(cpl + p + (ptrdiff_t)q * V);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        cxm[(q + J) * V + e] = Cvt<TF, TC>::f(a.v[e]);
                        cxp[(q + J) * V + e] = Cvt<TF, TC>::f(b.v[e]);
                    }
                }
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const int xc = J * V + e;
                    r[e] = A::fma(cxm[xc - d], lx[xc - d], r[e]);
                    r[e] = A::fma(cxp[xc + d], lx[xc + d], r[e]);
                }
            }
            // y and z
#pragma unroll
            for (int a = 1; a < 3; ++a) {
                const size_t o = (size_t)d * (a == 1 ? sy : sz);
                const Vec<TC, V> cmv = ldv_ro<TC, V>(C.c[SD::minus(d, a)] + p - o);
                const Vec<TF, V> lmv = lam_ld<COHERENT, TF, V>(lam_in + p - o);
                const Vec<TC, V> cpv = ldv_ro<TC, V>(C.c[SD::plus(d, a)] + p + o);
                const Vec<TF, V> lpv = lam_ld<COHERENT, TF, V>(lam_in + p + o);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    r[e] = A::fma(Cvt<TF, TC>::f(cmv.v[e]), lmv.v[e], r[e]);
                    r[e] = A::fma(Cvt<TF, TC>::f(cpv.v[e]), lpv.v[e], r[e]);
                }
            }
        }
        if (full) {
            Vec<TF, V> o;
#pragma unroll
            for (int e = 0; e < V; ++e) o.v[e] = r[e];
            stv<TF, V>(lam_out + p, o);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (i0 + e < L.nx) lam_out[p + e] = r[e];
        }
    }
}

}  // namespace stg
