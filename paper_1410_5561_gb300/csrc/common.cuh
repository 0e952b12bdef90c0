// Shared device helpers for the stencil kernels (sm_103a).
//
// Every kernel computes one lattice-site update (LUP) with the functions in
// this file, in the term order of the paper's Listings 1-3 (Section I-A), with
// explicitly rounded operations (__fmul_rn / __fmaf_rn / __fadd_rn and their
// double counterparts) so that the compiler cannot re-associate or contract
// them differently in different kernels. The plain and the temporally blocked
// sweeps therefore produce bit-identical results.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace stg {

enum Kind { K7C = 0, K7V = 1, K25V = 2 };

template <int KIND> struct KindTraits;
template <> struct KindTraits<K7C> { static constexpr int R = 1; static constexpr int NC = 0; };
template <> struct KindTraits<K7V> { static constexpr int R = 1; static constexpr int NC = 7; };
template <> struct KindTraits<K25V> { static constexpr int R = 4; static constexpr int NC = 13; };

// Element-index layout shared by every array of one grid (field and coefficients):
// interior (i, j, k) lives at ((k + R) * py + (j + R)) * px + (xo + i).
struct Layout {
    int nx, ny, nz;   // interior sizes
    int R;            // halo width
    int xo;           // elements before interior x = 0 (multiple of the vector width)
    int px;           // elements per row
    int py;           // rows per plane (ny + 2R)
    int pz;           // planes (nz + 2R)
    __host__ __device__ size_t plane() const { return (size_t)px * py; }
    __host__ __device__ size_t count() const { return plane() * pz; }
    __host__ __device__ size_t at(int i, int j, int k) const {
        return ((size_t)(k + R) * py + (size_t)(j + R)) * px + (size_t)(xo + i);
    }
};

// ----------------------------------------------------------------- arithmetic
template <typename T> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ar<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// Coefficient element -> field arithmetic type (BF16 widens exactly to FP32).
template <typename TF, typename TC> struct Cvt {
    static __device__ __forceinline__ TF f(TC c) { return (TF)c; }
};
template <> struct Cvt<float, __nv_bfloat16> {
    static __device__ __forceinline__ float f(__nv_bfloat16 c) { return __bfloat162float(c); }
};

// Listing 1: U = c0*V + c1*(x+ + x-) + c1*(y+ + y-) + c1*(z+ + z-)
template <typename T>
__device__ __forceinline__ T upd7c(T c0, T c1, T v, T xp, T xm, T yp, T ym, T zp, T zm) {
    using A = Ar<T>;
    T r = A::mul(c0, v);
    r = A::fma(c1, A::add(xp, xm), r);
    r = A::fma(c1, A::add(yp, ym), r);
    r = A::fma(c1, A::add(zp, zm), r);
    return r;
}

// Two FP32 lanes in one 64-bit register: sm_100-family packed add / mul / fma,
// each lane rounded exactly like the scalar operation (round to nearest, no
// flush), so a packed evaluation gives the scalar one's bits.
struct F2 {
    unsigned long long r;
    static __device__ __forceinline__ F2 pack(float a, float b) {
        F2 x;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x.r) : "f"(a), "f"(b));
        return x;
    }
    __device__ __forceinline__ void unpack(float& a, float& b) const {
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    }
    static __device__ __forceinline__ F2 add(F2 a, F2 b) {
        F2 x;
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(x.r) : "l"(a.r), "l"(b.r));
        return x;
    }
    static __device__ __forceinline__ F2 mul(F2 a, F2 b) {
        F2 x;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(x.r) : "l"(a.r), "l"(b.r));
        return x;
    }
    static __device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) {
        F2 x;
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(x.r) : "l"(a.r), "l"(b.r), "l"(c.r));
        return x;
    }
};

// Listing 1 for the points e and e+1 of a vector, packed: the same operations in
// the same order as upd7c on each point. sx: the x pair sums (xp + xm), formed
// by the caller because the x neighbours are not register pairs.
__device__ __forceinline__ F2 upd7c_x2(F2 c0, F2 c1, F2 v, F2 sx, F2 yp, F2 ym, F2 zp, F2 zm) {
    F2 r = F2::mul(c0, v);
    r = F2::fma(c1, sx, r);
    r = F2::fma(c1, F2::add(yp, ym), r);
    r = F2::fma(c1, F2::add(zp, zm), r);
    return r;
}

// Listing 2: U = C0*V + C1*x+ + C2*x- + C3*y+ + C4*y- + C5*z+ + C6*z-
template <typename T>
__device__ __forceinline__ T upd7v(const T* c, T v, T xp, T xm, T yp, T ym, T zp, T zm) {
    using A = Ar<T>;
    T r = A::mul(c[0], v);
    r = A::fma(c[1], xp, r);
    r = A::fma(c[2], xm, r);
    r = A::fma(c[3], yp, r);
    r = A::fma(c[4], ym, r);
    r = A::fma(c[5], zp, r);
    r = A::fma(c[6], zm, r);
    return r;
}

// Listing 3: U = C00*V + sum_{d=1..4} [C(3d-2)*(x+d + x-d) + C(3d-1)*(y+d + y-d) + C(3d)*(z+d + z-d)]
// xs[d-1] etc. hold the pair sums' operands: xp[d-1] = V(x+d), xm[d-1] = V(x-d).
template <typename T>
__device__ __forceinline__ T upd25v(const T* c, T v, const T* xp, const T* xm, const T* yp,
                                    const T* ym, const T* zp, const T* zm) {
    using A = Ar<T>;
    T r = A::mul(c[0], v);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        r = A::fma(c[3 * d + 1], A::add(xp[d], xm[d]), r);
        r = A::fma(c[3 * d + 2], A::add(yp[d], ym[d]), r);
        r = A::fma(c[3 * d + 3], A::add(zp[d], zm[d]), r);
    }
    return r;
}

// ------------------------------------------------------------ vector access
template <typename T, int V> struct alignas(sizeof(T) * V) Vec { T v[V]; };

template <int BYTES> struct Raw;
template <> struct Raw<16> { using t = uint4; };
template <> struct Raw<8> { using t = uint2; };
template <> struct Raw<4> { using t = unsigned int; };
template <> struct Raw<2> { using t = unsigned short; };

// Plain (coherent) vector load.
template <typename T, int V>
__device__ __forceinline__ Vec<T, V> ldv(const T* p) {
    return *reinterpret_cast<const Vec<T, V>*>(p);
}
// Read-only-path vector load: only for data no thread of the launch writes.
template <typename T, int V>
__device__ __forceinline__ Vec<T, V> ldv_ro(const T* p) {
    using R = typename Raw<sizeof(T) * V>::t;
    R r = __ldg(reinterpret_cast<const R*>(p));
    Vec<T, V> out;
    static_assert(sizeof(R) == sizeof(out), "size");
    memcpy(&out, &r, sizeof(out));
    return out;
}
// Streaming read-only load (evict-first): coefficients that are used once per pass.
template <typename T, int V>
__device__ __forceinline__ Vec<T, V> ldv_stream(const T* p) {
    using R = typename Raw<sizeof(T) * V>::t;
    R r = __ldcs(reinterpret_cast<const R*>(p));
    Vec<T, V> out;
    memcpy(&out, &r, sizeof(out));
    return out;
}
template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const Vec<T, V>& x) {
    *reinterpret_cast<Vec<T, V>*>(p) = x;
}

}  // namespace stg
