/*
 * FP64 CPU oracle for the three stencil sweeps of Malas, Ltaief, Hager, Keyes,
 * "Towards energy efficiency and maximum computational intensity for stencil
 * algorithms using wavefront diamond temporal blocking" (arXiv:1410.5561).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
 * baseline leg use this file. It shares no code with the CUDA library and is
 * built with -ffp-contract=off, so every product and sum is rounded once, in
 * the order the paper's listings write them.
 *
 * Layout (oracle-private): a grid with interior nx*ny*nz and halo H = R is a
 * dense FP64 array of (nz+2H)*(ny+2H)*(nx+2H) values, x fastest. Interior
 * point (i, j, k), 0-based, lives at ((k+H)*(ny+2H) + (j+H))*(nx+2H) + (i+H).
 * Coefficient arrays use the same padded shape; their halo is never read by
 * the forward sweep.
 *
 * What each function follows:
 *   oracle_step / oracle_sweep : Section I-A, Listings 1 (7-point constant),
 *       2 (7-point variable) and 3 (25-point variable): one Jacobi update of
 *       every interior point from the previous array, repeated over T steps
 *       with the two arrays swapped (Section I, "sweep ... repeated over many
 *       time steps"; two domain-sized arrays, Section I-A). The halo is never
 *       written (the listings' loops stop R cells from each face).
 *   oracle_step_transpose : the transpose of the same linear map, written as
 *       a scatter of each interior point's terms (not derived from the GPU's
 *       gather form).
 *   oracle_adjoint : reverse-mode derivative of L = 0.5*||u_T - target||^2
 *       over the interior, by storing every state and running the transposed
 *       steps backwards; coefficient gradients accumulate lambda_{t+1}(p) times
 *       the field value that multiplies C_m(p) in the listing.
 *   oracle_points : u_T at selected interior points, computed by the same
 *       update restricted to the shrinking box that the point depends on.
 */
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { K_7PT_CONST = 0, K_7PT_VAR = 1, K_25PT_VAR = 2 };

int oracle_radius(int kind) { return kind == K_25PT_VAR ? 4 : 1; }
int oracle_ncoef(int kind) { return kind == K_7PT_CONST ? 0 : (kind == K_7PT_VAR ? 7 : 13); }

static int valid_kind(int kind) { return kind >= 0 && kind <= 2; }

/* One interior point of Listing 1/2/3, terms in listing order. */
static inline double point_update(int kind, const double* V, size_t p, size_t sx, size_t sy,
                                  size_t sz, const double* scal, const double* const* C) {
    if (kind == K_7PT_CONST) {
        double c0 = scal[0], c1 = scal[1];
        double r = c0 * V[p];
        r = r + c1 * (V[p + sx] + V[p - sx]);
        r = r + c1 * (V[p + sy] + V[p - sy]);
        r = r + c1 * (V[p + sz] + V[p - sz]);
        return r;
    }
    if (kind == K_7PT_VAR) {
        double r = C[0][p] * V[p];
        r = r + C[1][p] * V[p + sx];
        r = r + C[2][p] * V[p - sx];
        r = r + C[3][p] * V[p + sy];
        r = r + C[4][p] * V[p - sy];
        r = r + C[5][p] * V[p + sz];
        r = r + C[6][p] * V[p - sz];
        return r;
    }
    /* 25-point: C00 centre, then distance d = 1..4, axis x, y, z. */
    double r = C[0][p] * V[p];
    for (int d = 1; d <= 4; ++d) {
        size_t ox = (size_t)d * sx, oy = (size_t)d * sy, oz = (size_t)d * sz;
        r = r + C[3 * (d - 1) + 1][p] * (V[p + ox] + V[p - ox]);
        r = r + C[3 * (d - 1) + 2][p] * (V[p + oy] + V[p - oy]);
        r = r + C[3 * (d - 1) + 3][p] * (V[p + oz] + V[p - oz]);
    }
    return r;
}

static void coef_ptrs(int kind, const double* coef, size_t n, const double** C) {
    int nc = oracle_ncoef(kind);
    for (int m = 0; m < nc; ++m) C[m] = coef + (size_t)m * n;
}

/* dst(interior) = A src; dst halo untouched. */
int oracle_step(int kind, int nx, int ny, int nz, const double* scal, const double* coef,
                const double* src, double* dst, int nthreads) {
    if (!valid_kind(kind) || nx < 0 || ny < 0 || nz < 0) return -1;
    int H = oracle_radius(kind);
    size_t px = (size_t)nx + 2 * H, py = (size_t)ny + 2 * H, pz = (size_t)nz + 2 * H;
    size_t n = px * py * pz;
    const double* C[13];
    coef_ptrs(kind, coef, n, C);
    size_t sx = 1, sy = px, sz = px * py;
    (void)pz;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)(k + H) * py + (size_t)(j + H)) * px + (size_t)(i + H);
                dst[p] = point_update(kind, src, p, sx, sy, sz, scal, C);
            }
    (void)nthreads;
    return 0;
}

/* u holds u_0 (interior and halo) on entry and u_T on exit; work is a second
 * padded array (its contents are overwritten; its halo is set from u). */
int oracle_sweep(int kind, int nx, int ny, int nz, int T, const double* scal, const double* coef,
                 double* u, double* work, int nthreads) {
    if (!valid_kind(kind) || T < 0) return -1;
    int H = oracle_radius(kind);
    size_t n = ((size_t)nx + 2 * H) * ((size_t)ny + 2 * H) * ((size_t)nz + 2 * H);
    memcpy(work, u, n * sizeof(double));
    double* V = u;
    double* U = work;
    for (int t = 0; t < T; ++t) {
        int rc = oracle_step(kind, nx, ny, nz, scal, coef, V, U, nthreads);
        if (rc) return rc;
        double* tmp = V; V = U; U = tmp;
    }
    if (V != u) memcpy(u, V, n * sizeof(double));
    return 0;
}

/* dst = A^T src over the interior: every interior point p scatters
 * weight(p, q) * src(p) to each interior q it reads. dst is fully
 * overwritten (halo set to 0). src's halo is ignored. */
int oracle_step_transpose(int kind, int nx, int ny, int nz, const double* scal,
                          const double* coef, const double* src, double* dst) {
    if (!valid_kind(kind)) return -1;
    int H = oracle_radius(kind);
    size_t px = (size_t)nx + 2 * H, py = (size_t)ny + 2 * H, pz = (size_t)nz + 2 * H;
    size_t n = px * py * pz;
    const double* C[13];
    coef_ptrs(kind, coef, n, C);
    memset(dst, 0, n * sizeof(double));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)(k + H) * py + (size_t)(j + H)) * px + (size_t)(i + H);
                double l = src[p];
                /* neighbour offsets (di, dj, dk) and weights, as read by point p */
                int nt = 0;
                int off[25][3];
                double w[25];
                if (kind == K_7PT_CONST) {
                    static const int o7[7][3] = {{0,0,0},{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
                    for (int m = 0; m < 7; ++m) {
                        off[m][0] = o7[m][0]; off[m][1] = o7[m][1]; off[m][2] = o7[m][2];
                        w[m] = m == 0 ? scal[0] : scal[1];
                    }
                    nt = 7;
                } else if (kind == K_7PT_VAR) {
                    static const int o7[7][3] = {{0,0,0},{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
                    for (int m = 0; m < 7; ++m) {
                        off[m][0] = o7[m][0]; off[m][1] = o7[m][1]; off[m][2] = o7[m][2];
                        w[m] = C[m][p];
                    }
                    nt = 7;
                } else {
                    off[0][0] = off[0][1] = off[0][2] = 0;
                    w[0] = C[0][p];
                    nt = 1;
                    for (int d = 1; d <= 4; ++d)
                        for (int a = 0; a < 3; ++a)
                            for (int sgn = -1; sgn <= 1; sgn += 2) {
                                off[nt][0] = a == 0 ? sgn * d : 0;
                                off[nt][1] = a == 1 ? sgn * d : 0;
                                off[nt][2] = a == 2 ? sgn * d : 0;
                                w[nt] = C[3 * (d - 1) + a + 1][p];
                                ++nt;
                            }
                }
                for (int m = 0; m < nt; ++m) {
                    int qi = i + off[m][0], qj = j + off[m][1], qk = k + off[m][2];
                    if (qi < 0 || qi >= nx || qj < 0 || qj >= ny || qk < 0 || qk >= nz) continue;
                    size_t q = ((size_t)(qk + H) * py + (size_t)(qj + H)) * px + (size_t)(qi + H);
                    dst[q] += w[m] * l;
                }
            }
    return 0;
}

/* Reverse-mode gradient of L = 0.5 * sum_interior (u_T - target)^2 with
 * respect to u_0 (interior) and every coefficient array (interior; halo of
 * g_coef set to 0). States are all stored (small grids only).
 * u0: padded u_0 with its Dirichlet halo; target: padded (halo ignored).
 * g_u0: padded output (halo 0). g_coef: ncoef padded outputs. */
int oracle_adjoint(int kind, int nx, int ny, int nz, int T, const double* coef,
                   const double* u0, const double* target, double* g_u0, double* g_coef,
                   double* loss_out) {
    if (kind != K_7PT_VAR && kind != K_25PT_VAR) return -1;
    if (T < 0) return -1;
    int H = oracle_radius(kind);
    int nc = oracle_ncoef(kind);
    size_t px = (size_t)nx + 2 * H, py = (size_t)ny + 2 * H, pz = (size_t)nz + 2 * H;
    size_t n = px * py * pz;
    size_t sx = 1, sy = px, sz = px * py;
    (void)pz;
    double* states = (double*)malloc((size_t)(T + 1) * n * sizeof(double));
    double* lam = (double*)malloc(n * sizeof(double));
    double* lam2 = (double*)malloc(n * sizeof(double));
    if (!states || !lam || !lam2) { free(states); free(lam); free(lam2); return -2; }
    memcpy(states, u0, n * sizeof(double));
    for (int t = 0; t < T; ++t) {
        memcpy(states + (size_t)(t + 1) * n, states + (size_t)t * n, n * sizeof(double));
        oracle_step(kind, nx, ny, nz, NULL, coef, states + (size_t)t * n,
                    states + (size_t)(t + 1) * n, 1);
    }
    const double* C[13];
    coef_ptrs(kind, coef, n, C);
    memset(lam, 0, n * sizeof(double));
    memset(g_coef, 0, (size_t)nc * n * sizeof(double));
    double loss = 0.0;
    const double* uT = states + (size_t)T * n;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t p = ((size_t)(k + H) * py + (size_t)(j + H)) * px + (size_t)(i + H);
                double r = uT[p] - target[p];
                lam[p] = r;
                loss += 0.5 * r * r;
            }
    for (int t = T - 1; t >= 0; --t) {
        const double* ut = states + (size_t)t * n;
        /* dL/dC_m(p) += lambda_{t+1}(p) * (field value multiplying C_m(p) at step t) */
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t p = ((size_t)(k + H) * py + (size_t)(j + H)) * px + (size_t)(i + H);
                    double l = lam[p];
                    if (kind == K_7PT_VAR) {
                        g_coef[0 * n + p] += l * ut[p];
                        g_coef[1 * n + p] += l * ut[p + sx];
                        g_coef[2 * n + p] += l * ut[p - sx];
                        g_coef[3 * n + p] += l * ut[p + sy];
                        g_coef[4 * n + p] += l * ut[p - sy];
                        g_coef[5 * n + p] += l * ut[p + sz];
                        g_coef[6 * n + p] += l * ut[p - sz];
                    } else {
                        g_coef[p] += l * ut[p];
                        for (int d = 1; d <= 4; ++d) {
                            size_t ox = (size_t)d * sx, oy = (size_t)d * sy, oz = (size_t)d * sz;
                            g_coef[(size_t)(3 * (d - 1) + 1) * n + p] += l * (ut[p + ox] + ut[p - ox]);
                            g_coef[(size_t)(3 * (d - 1) + 2) * n + p] += l * (ut[p + oy] + ut[p - oy]);
                            g_coef[(size_t)(3 * (d - 1) + 3) * n + p] += l * (ut[p + oz] + ut[p - oz]);
                        }
                    }
                }
        oracle_step_transpose(kind, nx, ny, nz, NULL, coef, lam, lam2);
        double* tmp = lam; lam = lam2; lam2 = tmp;
    }
    memcpy(g_u0, lam, n * sizeof(double));
    if (loss_out) *loss_out = loss;
    free(states); free(lam); free(lam2);
    (void)C;
    return 0;
}

/* u_T at npts interior points pts[3*q .. 3*q+2] = (i, j, k), from padded u0.
 * Each point is computed on the box it depends on, which shrinks by R per
 * step; values outside the interior are read from u0's halo. */
int oracle_points(int kind, int nx, int ny, int nz, int T, const double* scal,
                  const double* coef, const double* u0, int npts, const int* pts, double* out,
                  int nthreads) {
    if (!valid_kind(kind) || T < 0) return -1;
    int H = oracle_radius(kind);
    size_t px = (size_t)nx + 2 * H, py = (size_t)ny + 2 * H, pz = (size_t)nz + 2 * H;
    size_t n = px * py * pz;
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (int q = 0; q < npts; ++q) {
        int ci = pts[3 * q], cj = pts[3 * q + 1], ck = pts[3 * q + 2];
        if (ci < 0 || ci >= nx || cj < 0 || cj >= ny || ck < 0 || ck >= nz) { err = -1; continue; }
        long e = (long)H * T; /* reach of the dependency box */
        /* box in padded coordinates, clipped to the padded grid */
        long lo[3], hi[3];
        long c[3] = {ci + H, cj + H, ck + H};
        long ext[3] = {(long)px, (long)py, (long)pz};
        for (int a = 0; a < 3; ++a) {
            lo[a] = c[a] - e < 0 ? 0 : c[a] - e;
            hi[a] = c[a] + e + 1 > ext[a] ? ext[a] : c[a] + e + 1;
        }
        long bx = hi[0] - lo[0], by = hi[1] - lo[1], bz = hi[2] - lo[2];
        size_t bn = (size_t)bx * by * bz;
        double* A = (double*)malloc(bn * sizeof(double));
        double* B = (double*)malloc(bn * sizeof(double));
        double* Cb = NULL;
        int nc = oracle_ncoef(kind);
        if (nc) Cb = (double*)malloc((size_t)nc * bn * sizeof(double));
        if (!A || !B || (nc && !Cb)) { free(A); free(B); free(Cb); err = -2; continue; }
        for (long k = 0; k < bz; ++k)
            for (long j = 0; j < by; ++j) {
                size_t src = ((size_t)(k + lo[2]) * py + (size_t)(j + lo[1])) * px + (size_t)lo[0];
                size_t dst = ((size_t)k * by + (size_t)j) * bx;
                memcpy(A + dst, u0 + src, (size_t)bx * sizeof(double));
                for (int m = 0; m < nc; ++m)
                    memcpy(Cb + (size_t)m * bn + dst, coef + (size_t)m * n + src,
                           (size_t)bx * sizeof(double));
            }
        memcpy(B, A, bn * sizeof(double));
        const double* Cp[13];
        for (int m = 0; m < nc; ++m) Cp[m] = Cb + (size_t)m * bn;
        double* V = A;
        double* U = B;
        for (int t = 0; t < T; ++t) {
            long r = (long)H * (T - t - 1); /* points still needed after this step */
            long ulo[3], uhi[3];
            for (int a = 0; a < 3; ++a) {
                long l = c[a] - r, h = c[a] + r + 1;
                long ilo = H, ihi = ext[a] - H; /* interior in padded coords */
                if (l < ilo) l = ilo;
                if (h > ihi) h = ihi;
                ulo[a] = l - lo[a];
                uhi[a] = h - lo[a];
            }
            for (long k = ulo[2]; k < uhi[2]; ++k)
                for (long j = ulo[1]; j < uhi[1]; ++j)
                    for (long i = ulo[0]; i < uhi[0]; ++i) {
                        size_t p = ((size_t)k * by + (size_t)j) * bx + (size_t)i;
                        U[p] = point_update(kind, V, p, 1, (size_t)bx, (size_t)bx * by, scal, Cp);
                    }
            double* tmp = V; V = U; U = tmp;
        }
        size_t pc = ((size_t)(c[2] - lo[2]) * by + (size_t)(c[1] - lo[1])) * bx + (size_t)(c[0] - lo[0]);
        out[q] = V[pc];
        free(A); free(B); free(Cb);
    }
    (void)nthreads;
    return err;
}
