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
#include "adjoint_column.cuh"
#include "internal.h"

namespace stg {

struct AdjGrad {
    double* g[13];
};

// One transposed step over the interior: lam_out = A^T lam_in (lambda_column). A warp covers
// 32 x vectors of V = 16/sizeof(field) points (128-bit loads), warps are stacked along y, and
// each thread walks a chunk of z planes.
template <int KIND, typename TF, typename TC, int BY>
__global__ void __launch_bounds__(32 * BY) adjoint_vec_kernel(Layout L, const TF* __restrict__ lam_in,
                                                              TF* __restrict__ lam_out, CoefPtrs<TC> C, int zchunk) {
    constexpr int V = 16 / sizeof(TF);
    const int i0 = (blockIdx.x * 32 + threadIdx.x) * V;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zchunk;
    const int k1 = min(L.nz, k0 + zchunk);
    lambda_column<KIND, TF, TC, false>(L, lam_in, lam_out, C, i0, j, k0, k1);
}

// Coefficient gradients of several steps in one pass: for the steps t = t_hi, t_hi - 1,
// ..., t_lo (in that order, the order of the backward walk), gC_m(p) += lam_{t+1}(p) x
// (the field value(s) C_m(p) weighs in step t), one FP64 fma per step on an accumulator
// kept in registers, so each gradient array is read and written once per pass instead of
// once per step. The fma sequence per element is the one the one-step kernel performs, so
// the result is the same bit for bit. lam[g] = lam_{t_hi + 1 - g}, u[g] = u_{t_hi - g}.
constexpr int ADJ_GROUP = 16;  // steps per gradient pass

template <typename TF>
struct AdjSteps {
    const TF* lam[ADJ_GROUP];
    const TF* u[ADJ_GROUP];
};

template <int KIND, typename TF, int BY>
__global__ void __launch_bounds__(32 * BY) adjoint_grad_kernel(Layout L, AdjSteps<TF> S, int nsteps, AdjGrad G,
                                                               int zchunk) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int NC = KindTraits<KIND>::NC;
    constexpr int V = 16 / sizeof(TF);
    constexpr int J = (R + V - 1) / V;
    constexpr int XL = (2 * J + 1) * V;
    using A = Ar<TF>;
    const int i0 = (blockIdx.x * 32 + threadIdx.x) * V;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i0 >= L.nx || j >= L.ny) return;
    const int k0 = blockIdx.z * zchunk;
    const int k1 = min(L.nz, k0 + zchunk);
    const size_t sy = (size_t)L.px, sz = L.plane();
    const bool full = i0 + V <= L.nx;
    for (int k = k0; k < k1; ++k) {
        const size_t p = L.at(i0, j, k);
        // all accumulators in registers: every gradient array read once and written once
        double gv[NC][V];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const double* gp = G.g[m] + p;
            if (full) {
#pragma unroll
                for (int h = 0; h < V; h += 2) {
                    const double2 g = *reinterpret_cast<const double2*>(gp + h);
                    gv[m][h] = g.x;
                    gv[m][h + 1] = g.y;
                }
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) gv[m][e] = i0 + e < L.nx ? gp[e] : 0.0;
            }
        }
        // steps outermost: the neighbours of each state are loaded once per step
        for (int g = 0; g < nsteps; ++g) {
            const TF* u = S.u[g];
            const Vec<TF, V> lv = ldv_ro<TF, V>(S.lam[g] + p);
            TF ux[XL];
#pragma unroll
            for (int q = -J; q <= J; ++q) {
                const Vec<TF, V> wu = ldv_ro<TF, V>(u + p + (ptrdiff_t)q * V);
#pragma unroll
                for (int e = 0; e < V; ++e) ux[(q + J) * V + e] = wu.v[e];
            }
            double lam[V];
#pragma unroll
            for (int e = 0; e < V; ++e) lam[e] = (double)lv.v[e];
            // weight of array m: 7-point C0 u(p), C(2a+1) u(p + e_a), C(2a+2) u(p - e_a);
            // 25-point C00 u(p), C(3(d-1)+a+1) (u(p + d e_a) + u(p - d e_a)), the pair sum
            // in the field precision as the forward step forms it
#pragma unroll
            for (int e = 0; e < V; ++e) gv[0][e] = __fma_rn(lam[e], (double)ux[J * V + e], gv[0][e]);
#pragma unroll
            for (int d = 1; d <= R; ++d) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    TF up[V], um[V];
                    if (a == 0) {
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            up[e] = ux[J * V + e + d];
                            um[e] = ux[J * V + e - d];
                        }
                    } else {
                        const size_t o = (size_t)d * (a == 1 ? sy : sz);
                        const Vec<TF, V> vp = ldv_ro<TF, V>(u + p + o);
                        const Vec<TF, V> vm = ldv_ro<TF, V>(u + p - o);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            up[e] = vp.v[e];
                            um[e] = vm.v[e];
                        }
                    }
                    if constexpr (KIND == K7V) {
                        // C(2a+1) weighs u(p + e_a), C(2a+2) weighs u(p - e_a)
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            gv[1 + 2 * a][e] = __fma_rn(lam[e], (double)up[e], gv[1 + 2 * a][e]);
                            gv[2 + 2 * a][e] = __fma_rn(lam[e], (double)um[e], gv[2 + 2 * a][e]);
                        }
                    } else {
                        const int m = 3 * (d - 1) + a + 1;
#pragma unroll
                        for (int e = 0; e < V; ++e) gv[m][e] = __fma_rn(lam[e], (double)A::add(up[e], um[e]), gv[m][e]);
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            double* gp = G.g[m] + p;
            if (full) {
#pragma unroll
                for (int h = 0; h < V; h += 2) *reinterpret_cast<double2*>(gp + h) = make_double2(gv[m][h], gv[m][h + 1]);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (i0 + e < L.nx) gp[e] = gv[m][e];
            }
        }
    }
}

template <int KIND, typename TF>
static cudaError_t adj_grads(const Layout& L, const void* const* lam, const void* const* u, int n,
                             double* const* gC, cudaStream_t s) {
    constexpr int BY = 4;
    constexpr int V = 16 / sizeof(TF);
    const int zchunk = 16;
    dim3 block(32, BY, 1);
    dim3 grid((unsigned)((L.nx + 32 * V - 1) / (32 * V)), (unsigned)((L.ny + BY - 1) / BY),
              (unsigned)((L.nz + zchunk - 1) / zchunk));
    AdjGrad G{};
    for (int m = 0; m < KindTraits<KIND>::NC; ++m) G.g[m] = gC[m];
    for (int g0 = 0; g0 < n; g0 += ADJ_GROUP) {
        AdjSteps<TF> S{};
        const int ng = n - g0 < ADJ_GROUP ? n - g0 : ADJ_GROUP;
        for (int g = 0; g < ng; ++g) {
            S.lam[g] = static_cast<const TF*>(lam[g0 + g]);
            S.u[g] = static_cast<const TF*>(u[g0 + g]);
        }
        adjoint_grad_kernel<KIND, TF, BY><<<grid, block, 0, s>>>(L, S, ng, G, zchunk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t adjoint_grads(const SweepArgs& a, const void* const* lam, const void* const* u, int n, double* const* gC,
                          cudaStream_t s) {
    if (a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0 || n <= 0) return cudaSuccess;
    if (a.kind == K7V) {
        if (a.fdt == DT_F32) return adj_grads<K7V, float>(a.L, lam, u, n, gC, s);
        if (a.fdt == DT_F64) return adj_grads<K7V, double>(a.L, lam, u, n, gC, s);
    } else if (a.kind == K25V) {
        if (a.fdt == DT_F32) return adj_grads<K25V, float>(a.L, lam, u, n, gC, s);
        if (a.fdt == DT_F64) return adj_grads<K25V, double>(a.L, lam, u, n, gC, s);
    }
    return cudaErrorInvalidValue;
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
static cudaError_t adj_step(const SweepArgs& a, const void* lam_in, void* lam_out, cudaStream_t s) {
    const Layout& L = a.L;
    CoefPtrs<TC> C{};
    for (int m = 0; m < KindTraits<KIND>::NC; ++m) C.c[m] = static_cast<const TC*>(a.coef[m]);
    constexpr int BY = 4;
    constexpr int V = 16 / sizeof(TF);
    const int zchunk = 16;
    dim3 block(32, BY, 1);
    dim3 grid((unsigned)((L.nx + 32 * V - 1) / (32 * V)), (unsigned)((L.ny + BY - 1) / BY),
              (unsigned)((L.nz + zchunk - 1) / zchunk));
    adjoint_vec_kernel<KIND, TF, TC, BY><<<grid, block, 0, s>>>(L, static_cast<const TF*>(lam_in),
                                                                static_cast<TF*>(lam_out), C, zchunk);
    return cudaGetLastError();
}

cudaError_t adjoint_step(const SweepArgs& a, const void* lam_in, void* lam_out, cudaStream_t s) {
    if (a.L.nx == 0 || a.L.ny == 0 || a.L.nz == 0) return cudaSuccess;
    if (a.kind == K7V) {
        if (a.fdt == DT_F32 && a.cdt == DT_F32) return adj_step<K7V, float, float>(a, lam_in, lam_out, s);
        if (a.fdt == DT_F32 && a.cdt == DT_BF16) return adj_step<K7V, float, __nv_bfloat16>(a, lam_in, lam_out, s);
        if (a.fdt == DT_F64) return adj_step<K7V, double, double>(a, lam_in, lam_out, s);
    } else if (a.kind == K25V) {
        if (a.fdt == DT_F32 && a.cdt == DT_F32) return adj_step<K25V, float, float>(a, lam_in, lam_out, s);
        if (a.fdt == DT_F32 && a.cdt == DT_BF16) return adj_step<K25V, float, __nv_bfloat16>(a, lam_in, lam_out, s);
        if (a.fdt == DT_F64) return adj_step<K25V, double, double>(a, lam_in, lam_out, s);
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
