// Adjoint (reverse-mode) sweep of the variable-coefficient stencils.
//
// Forward (Listings 2 and 3): u_{t+1} = A(C) u_t on the interior, Dirichlet halo.
// For L = 0.5 ||u_T - target||^2 (or any cotangent lambda_T of u_T):
//   lambda_t = A^T lambda_{t+1},
//   (A^T l)(q) = sum over the terms of every point p that reads q of C(p) l(p):
//     7-point:  C0(q) l(q) + C1(q-x) l(q-x) + C2(q+x) l(q+x) + C3(q-y) l(q-y)
//               + C4(q+y) l(q+y) + C5(q-z) l(q-z) + C6(q+z) l(q+z)
//     25-point: C00(q) l(q) + sum_{d,a} [C_da(q - d e_a) l(q - d e_a) + C_da(q + d e_a) l(q + d e_a)]
//   dL/dC_m(p) = sum_t lambda_{t+1}(p) * (the field value that multiplies C_m(p) at step t),
//   dL/du_0 = lambda_0.
// Zero halos in lambda and in the coefficient arrays make the "p is interior"
// condition of the transpose automatic. Coefficient gradients accumulate in FP64.
#include "internal.h"

namespace stg {

template <typename TC>
struct AdjCoef {
    const TC* c[13];
};
struct AdjGrad {
    double* g[13];
};

template <typename TF, typename TC>
__device__ __forceinline__ TF cf(const TC* p, size_t i) {
    return Cvt<TF, TC>::f(__ldg(p + i));
}

// One adjoint step over the interior: lam_out = A^T lam_in (interior), gC += lam_in * u terms.
template <int KIND, typename TF, typename TC>
__global__ void __launch_bounds__(256) adjoint_step_kernel(Layout L, const TF* __restrict__ lam_in,
                                                           const TF* __restrict__ u, TF* __restrict__ lam_out,
                                                           AdjCoef<TC> C, AdjGrad G, int accumulate) {
    constexpr int R = KindTraits<KIND>::R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int k = blockIdx.z;
    if (i >= L.nx) return;
    const size_t p = L.at(i, j, k);
    const size_t sx = 1, sy = (size_t)L.px, sz = L.plane();
    using A = Ar<TF>;
    const TF l = __ldg(lam_in + p);
    if constexpr (KIND == K7V) {
        TF r = A::mul(cf<TF, TC>(C.c[0], p), l);
        r = A::fma(cf<TF, TC>(C.c[1], p - sx), __ldg(lam_in + p - sx), r);
        r = A::fma(cf<TF, TC>(C.c[2], p + sx), __ldg(lam_in + p + sx), r);
        r = A::fma(cf<TF, TC>(C.c[3], p - sy), __ldg(lam_in + p - sy), r);
        r = A::fma(cf<TF, TC>(C.c[4], p + sy), __ldg(lam_in + p + sy), r);
        r = A::fma(cf<TF, TC>(C.c[5], p - sz), __ldg(lam_in + p - sz), r);
        r = A::fma(cf<TF, TC>(C.c[6], p + sz), __ldg(lam_in + p + sz), r);
        lam_out[p] = r;
        if (accumulate) {
            const double ld = (double)l;
            G.g[0][p] += ld * (double)__ldg(u + p);
            G.g[1][p] += ld * (double)__ldg(u + p + sx);
            G.g[2][p] += ld * (double)__ldg(u + p - sx);
            G.g[3][p] += ld * (double)__ldg(u + p + sy);
            G.g[4][p] += ld * (double)__ldg(u + p - sy);
            G.g[5][p] += ld * (double)__ldg(u + p + sz);
            G.g[6][p] += ld * (double)__ldg(u + p - sz);
        }
    } else {
        TF r = A::mul(cf<TF, TC>(C.c[0], p), l);
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            const size_t o[3] = {d * sx, d * sy, d * sz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const TC* cp = C.c[3 * (d - 1) + a + 1];
                r = A::fma(cf<TF, TC>(cp, p - o[a]), __ldg(lam_in + p - o[a]), r);
                r = A::fma(cf<TF, TC>(cp, p + o[a]), __ldg(lam_in + p + o[a]), r);
            }
        }
        lam_out[p] = r;
        if (accumulate) {
            const double ld = (double)l;
            G.g[0][p] += ld * (double)__ldg(u + p);
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const size_t o[3] = {d * sx, d * sy, d * sz};
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    G.g[3 * (d - 1) + a + 1][p] +=
                        ld * ((double)__ldg(u + p + o[a]) + (double)__ldg(u + p - o[a]));
            }
        }
    }
}

// dst(interior) = src(interior); every other cell of dst = 0.
template <typename TF>
__global__ void copy_interior_zero_halo_kernel(Layout L, const TF* __restrict__ src, TF* __restrict__ dst) {
    const size_t n = L.count();
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const size_t row = q / (size_t)L.px;
        const int x = (int)(q - row * (size_t)L.px) - L.xo;
        const int y = (int)(row % (size_t)L.py) - L.R;
        const int z = (int)(row / (size_t)L.py) - L.R;
        const bool in = x >= 0 && x < L.nx && y >= 0 && y < L.ny && z >= 0 && z < L.nz;
        dst[q] = in ? src[q] : TF(0);
    }
}

template <int KIND, typename TF, typename TC>
static cudaError_t adj_step(const SweepArgs& a, const void* lam_in, const void* u, void* lam_out,
                            double* const* gC, bool accumulate, cudaStream_t s) {
    const Layout& L = a.L;
    AdjCoef<TC> C{};
    AdjGrad G{};
    for (int m = 0; m < KindTraits<KIND>::NC; ++m) {
        C.c[m] = static_cast<const TC*>(a.coef[m]);
        G.g[m] = gC[m];
    }
    dim3 block(256, 1, 1);
    dim3 grid((unsigned)((L.nx + 255) / 256), (unsigned)L.ny, (unsigned)L.nz);
    adjoint_step_kernel<KIND, TF, TC><<<grid, block, 0, s>>>(L, static_cast<const TF*>(lam_in),
                                                             static_cast<const TF*>(u), static_cast<TF*>(lam_out),
                                                             C, G, accumulate ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t adjoint_step(const SweepArgs& a, const void* lam_in, const void* u, void* lam_out, double* const* gC,
                         bool accumulate, cudaStream_t s) {
    if (a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    if (a.kind == K7V) {
        if (a.fdt == DT_F32 && a.cdt == DT_F32) return adj_step<K7V, float, float>(a, lam_in, u, lam_out, gC, accumulate, s);
        if (a.fdt == DT_F32 && a.cdt == DT_BF16)
            return adj_step<K7V, float, __nv_bfloat16>(a, lam_in, u, lam_out, gC, accumulate, s);
        if (a.fdt == DT_F64) return adj_step<K7V, double, double>(a, lam_in, u, lam_out, gC, accumulate, s);
    } else if (a.kind == K25V) {
        if (a.fdt == DT_F32 && a.cdt == DT_F32)
            return adj_step<K25V, float, float>(a, lam_in, u, lam_out, gC, accumulate, s);
        if (a.fdt == DT_F32 && a.cdt == DT_BF16)
            return adj_step<K25V, float, __nv_bfloat16>(a, lam_in, u, lam_out, gC, accumulate, s);
        if (a.fdt == DT_F64) return adj_step<K25V, double, double>(a, lam_in, u, lam_out, gC, accumulate, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t copy_interior_zero_halo(const Layout& L, int dt, const void* src, void* dst, cudaStream_t s) {
    unsigned blocks = (unsigned)((L.count() + 255) / 256);
    if (blocks > 152u * 32u) blocks = 152u * 32u;
    if (dt == DT_F32)
        copy_interior_zero_halo_kernel<float><<<blocks, 256, 0, s>>>(L, (const float*)src, (float*)dst);
    else if (dt == DT_F64)
        copy_interior_zero_halo_kernel<double><<<blocks, 256, 0, s>>>(L, (const double*)src, (double*)dst);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace stg
