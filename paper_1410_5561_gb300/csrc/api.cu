// C-ABI layer: argument checks, layout, host<->device copies and dispatch to
// the sweep kernels. Declarations and contracts are in include/stencil_gb300.h.
#include <stdint.h>
#include <string.h>
#include <math.h>

#include <new>
#include <vector>

#include "../../include/stencil_gb300.h"
#include "internal.h"

using namespace stg;

struct stencil_grid {
    int kind, fdt, cdt;
    Layout L;
    cudaStream_t stream;
    void* field[2];
    void* coef[13];
    void* ws;
    bool bound;
    double c0, c1, halo;
    int parity;
    int scheme;
    BlockedTune tune;
    WaveTune wtune;
    int plain_prefetch;  // plain sweep's prefetch depth (0 or 2)
    bool tune_set;
    long long launches;
    long long tile_passes;  // wavefront passes run with tile copies into shared memory
    bool halo_ok;        // both bound field arrays hold `halo` in every non-interior cell
    bool status_armed;   // the workspace's status word has been zeroed since bind / set_field
    PersistCtl ctl;      // dependency-wait limit and stall hook of the persistent schedule
};

static int from_cuda(cudaError_t e) { return e == cudaSuccess ? STENCIL_OK : STENCIL_ECUDA; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static SweepArgs args_of(const stencil_grid* h) {
    SweepArgs a{};
    a.kind = h->kind;
    a.fdt = h->fdt;
    a.cdt = h->cdt;
    a.L = h->L;
    for (int m = 0; m < 13; ++m) a.coef[m] = h->coef[m];
    a.c0 = h->c0;
    a.c1 = h->c1;
    a.halo = h->halo;
    a.plain_prefetch = h->plain_prefetch;
    return a;
}

// Default blocked tuning: D_w = 8 (R = 1) or 16 (R = 4), two frontlines (one for the
// 7-point variable stencil with FP32 coefficients, measured faster on GB300), 16 (8)
// warps, x tiles sized so that a tile row plus its trapezoid overlap is one warp
// of vectors; D_w is halved until the rings fit the shared-memory opt-in limit.
static BlockedTune default_tune(const stencil_grid* h) {
    BlockedTune t{};
    int R = kind_radius(h->kind);
    int eb = dtype_bytes(h->fdt);
    t.dw = R == 1 ? 8 : 16;
    t.nf = (h->kind == STENCIL_7PT_VAR && h->fdt == STENCIL_F32 && h->cdt == STENCIL_F32) ? 1 : 2;
    t.warps = R == 1 ? 16 : 8;
    {
        // widest x tile whose bottom level (tile plus trapezoid overlap) fits one warp of vectors
        int V = 16 / eb;
        int ov = ((R * (t.dw / R - 2) + V - 1) / V) * V;
        t.xtile = 32 * V - 2 * ov;
        if (t.xtile < V) t.xtile = V;
        // then the narrowest one that keeps the number of x tiles per row (less overlap work):
        // with R = 1 the first and last tiles are wider by their one-sided overlap
        const int nx = h->L.nx, lt = t.dw / R - 1;
        const int ove = lt > 1 ? ((R * (lt - 1) + V - 1) / V) * V : 0;
        auto tiles = [&](int xt) {
            if (nx <= xt) return 1;
            if (R != 1) return (nx + xt - 1) / xt;
            const int xe = xt + ove;
            return nx <= 2 * xe ? 2 : 2 + (nx - 2 * xe + xt - 1) / xt;
        };
        const int n0 = tiles(t.xtile);
        for (int xt = V; xt < t.xtile; xt += V)
            if (tiles(xt) == n0) {
                t.xtile = xt;
                break;
            }
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) optin = 0;
    SweepArgs a = args_of(h);
    auto fits = [&](const BlockedTune& x) {
        const size_t b = blocked_smem_bytes(a, x);
        return b != 0 && b <= (size_t)optin;
    };
    if (!fits(t)) t.nf = 1;
    while (t.dw > 2 * R && !fits(t)) t.dw /= 2;
    return t;
}

static int check_tune(const stencil_grid* h, const BlockedTune& t) {
    SweepArgs a = args_of(h);
    size_t need = blocked_smem_bytes(a, t);
    if (need == 0) return STENCIL_EINVAL;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return STENCIL_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return STENCIL_ECUDA;
    if (need > (size_t)optin) return STENCIL_ENOSMEM;
    return STENCIL_OK;
}

namespace stg {
int grid_batch_view(const stencil_grid* h, SweepArgs* a, void** f0, void** f1, int* parity) {
    if (!h) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    *a = args_of(h);
    *f0 = h->field[0];
    *f1 = h->field[1];
    *parity = h->parity;
    return STENCIL_OK;
}
void grid_set_parity(stencil_grid* h, int parity) { h->parity = parity & 1; }
}  // namespace stg

extern "C" {

int stencil_create(stencil_t* out, int kind, int nx, int ny, int nz, int field_dtype, int coef_dtype,
                   void* cuda_stream) {
    if (!out) return STENCIL_EINVAL;
    *out = nullptr;
    if (kind < STENCIL_7PT_CONST || kind > STENCIL_25PT_VAR) return STENCIL_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return STENCIL_EINVAL;
    if (field_dtype != STENCIL_F32 && field_dtype != STENCIL_F64) return STENCIL_EINVAL;
    if (kind == STENCIL_7PT_CONST) coef_dtype = field_dtype;
    if (coef_dtype != field_dtype && !(field_dtype == STENCIL_F32 && coef_dtype == STENCIL_BF16))
        return STENCIL_EINVAL;
    const int R = kind_radius(kind);
    const int eb = dtype_bytes(field_dtype);
    const int V = 16 / eb;
    const int J = (R + V - 1) / V;
    const long long rowal = 128 / eb;  // 128-byte rows for the field
    long long xo = (long long)J * V;
    long long px = xo + ((nx + V - 1) / V) * (long long)V + xo;
    px = ((px + rowal - 1) / rowal) * rowal;
    long long py = (long long)ny + 2 * R, pz = (long long)nz + 2 * R;
    if (px > (1LL << 30) || py > (1LL << 30) || pz > (1LL << 30)) return STENCIL_EINVAL;
    stencil_grid* h = new (std::nothrow) stencil_grid();
    if (!h) return STENCIL_EINVAL;
    h->kind = kind;
    h->fdt = field_dtype;
    h->cdt = coef_dtype;
    h->L.nx = nx;
    h->L.ny = ny;
    h->L.nz = nz;
    h->L.R = R;
    h->L.xo = (int)xo;
    h->L.px = (int)px;
    h->L.py = (int)py;
    h->L.pz = (int)pz;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->c0 = 0.4;
    h->c1 = 0.1;
    h->halo = 0.0;
    h->parity = 0;
    h->scheme = STENCIL_PLAIN;
    h->tune_set = false;
    h->launches = 0;
    h->tile_passes = 0;
    h->halo_ok = false;
    h->status_armed = false;
    h->ctl.spin_limit = 1u << 24;
    h->ctl.stall_item = -1;
    // measured on GB300: copying every load two planes ahead pays only for the 25-point sweep with
    // BF16 coefficients (+7 %); the other sweeps need more resident CTAs than its slots allow
    h->plain_prefetch = (kind == STENCIL_25PT_VAR && coef_dtype == STENCIL_BF16) ? 2 : 0;
    *out = h;
    return STENCIL_OK;
}

int stencil_layout_of(stencil_t h, int which, stencil_layout* out) {
    if (!h || !out) return STENCIL_EINVAL;
    if (which != STENCIL_FIELD_ARRAY && which != STENCIL_COEF_ARRAY && which != STENCIL_GRAD_ARRAY)
        return STENCIL_EINVAL;
    if (which != STENCIL_FIELD_ARRAY && h->kind == STENCIL_7PT_CONST) return STENCIL_EINVAL;
    int eb = which == STENCIL_FIELD_ARRAY ? dtype_bytes(h->fdt) : (which == STENCIL_COEF_ARRAY ? dtype_bytes(h->cdt) : 8);
    out->radius = h->L.R;
    out->elem_bytes = eb;
    out->x_offset = h->L.xo;
    out->pitch_x = h->L.px;
    out->pitch_y = h->L.py;
    out->planes = h->L.pz;
    out->bytes = h->L.count() * (size_t)eb;
    return STENCIL_OK;
}

size_t stencil_workspace_bytes(stencil_t h) {
    (void)h;
    return GRID_WORKSPACE_BYTES;
}

int stencil_bind(stencil_t h, void* field_a, void* field_b, void* const* coef, void* workspace) {
    if (!h || !field_a || !field_b || field_a == field_b) return STENCIL_EINVAL;
    if (!aligned16(field_a) || !aligned16(field_b)) return STENCIL_EINVAL;
    int nc = kind_ncoef(h->kind);
    if (nc > 0 && !coef) return STENCIL_EINVAL;
    for (int m = 0; m < nc; ++m)
        if (!coef[m] || !aligned16(coef[m])) return STENCIL_EINVAL;
    h->field[0] = field_a;
    h->field[1] = field_b;
    for (int m = 0; m < 13; ++m) h->coef[m] = m < nc ? coef[m] : nullptr;
    if (workspace && !aligned16(workspace)) return STENCIL_EINVAL;
    h->ws = workspace;
    h->halo_ok = false;
    h->status_armed = false;
    h->bound = true;
    return STENCIL_OK;
}

// The address the current device uses for p: device memory of that device, managed memory, or
// page-locked host memory mapped for it; null for anything else (pageable host memory, another
// device's memory, not a pointer CUDA knows), which the SM copy must not dereference.
static void* device_view(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (at.type == cudaMemoryTypeDevice) return at.device == dev ? const_cast<void*>(p) : nullptr;
    if (at.type == cudaMemoryTypeManaged) return const_cast<void*>(p);
    if (at.type == cudaMemoryTypeHost) return at.devicePointer;
    return nullptr;
}

static cudaError_t copy_interior(const stencil_grid* h, int eb, const void* dense, void* padded, bool to_padded,
                                 bool dma = false) {
    const Layout& L = h->L;
    // device memory, or page-locked host memory the device can address: the library's copy
    // kernel; pageable host memory, or dma: a pitched DMA
    cudaPointerAttributes at{};
    if (dma) {
        if (cudaPointerGetAttributes(&at, dense) != cudaSuccess) {
            cudaGetLastError();
            return cudaErrorInvalidValue;
        }
        if (at.type != cudaMemoryTypeHost) return cudaErrorInvalidValue;
    } else if (const void* dp = device_view(dense)) {
        // memory this device addresses (another device's memory and pageable memory take the DMA)
        return to_padded ? copy_rows(L, eb, dp, padded, true, h->stream)
                         : copy_rows(L, eb, padded, const_cast<void*>(dp), false, h->stream);
    }
    cudaMemcpy3DParms p{};
    cudaPitchedPtr dn = make_cudaPitchedPtr(const_cast<void*>(dense), (size_t)L.nx * eb, (size_t)L.nx, (size_t)L.ny);
    cudaPitchedPtr pd = make_cudaPitchedPtr(padded, (size_t)L.px * eb, (size_t)L.px, (size_t)L.py);
    if (to_padded) {
        p.srcPtr = dn;
        p.dstPtr = pd;
        p.dstPos = make_cudaPos((size_t)L.xo * eb, (size_t)L.R, (size_t)L.R);
    } else {
        p.srcPtr = pd;
        p.srcPos = make_cudaPos((size_t)L.xo * eb, (size_t)L.R, (size_t)L.R);
        p.dstPtr = dn;
    }
    p.extent = make_cudaExtent((size_t)L.nx * eb, (size_t)L.ny, (size_t)L.nz);
    p.kind = cudaMemcpyDefault;
    return cudaMemcpy3DAsync(&p, h->stream);
}

int stencil_set_coeffs(stencil_t h, const double* scalars, const void* const* arrays, int where) {
    if (!h) return STENCIL_EINVAL;
    if (where != STENCIL_HOST && where != STENCIL_DEVICE) return STENCIL_EINVAL;
    if (h->kind == STENCIL_7PT_CONST) {
        if (!scalars) return STENCIL_EINVAL;
        h->c0 = scalars[0];
        h->c1 = scalars[1];
        return STENCIL_OK;
    }
    if (!h->bound) return STENCIL_EUNBOUND;
    if (!arrays) return STENCIL_EINVAL;
    int nc = kind_ncoef(h->kind);
    int eb = dtype_bytes(h->cdt);
    for (int m = 0; m < nc; ++m) {
        if (!arrays[m]) return STENCIL_EINVAL;
        cudaError_t e = fill_value(h->coef[m], h->L.count(), h->cdt, 0.0, h->stream);
        if (e != cudaSuccess) return STENCIL_ECUDA;
        ++h->launches;
        e = copy_interior(h, eb, arrays[m], h->coef[m], true);
        if (e != cudaSuccess) return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

int stencil_set_field(stencil_t h, const void* src, double halo_value, int where) {
    if (!h || !src) return STENCIL_EINVAL;
    if (where != STENCIL_HOST && where != STENCIL_DEVICE && where != STENCIL_HOST_ASYNC) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    // sweeps write interior cells only, so a halo set by an earlier call on the same arrays
    // stays (the interior of the second array is written before it is read)
    const bool same = h->halo_ok && memcmp(&h->halo, &halo_value, sizeof(double)) == 0;
    if (!same) {
        h->halo_ok = false;
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = fill_value(h->field[i], h->L.count(), h->fdt, halo_value, h->stream);
            if (e != cudaSuccess) return STENCIL_ECUDA;
            ++h->launches;
        }
    }
    cudaError_t e = copy_interior(h, dtype_bytes(h->fdt), src, h->field[0], true, where == STENCIL_HOST_ASYNC);
    if (e == cudaErrorInvalidValue && where == STENCIL_HOST_ASYNC) return STENCIL_EINVAL;
    if (e != cudaSuccess) return STENCIL_ECUDA;
    h->halo = halo_value;
    h->halo_ok = true;
    h->parity = 0;
    h->status_armed = false;  // a new field: earlier timeouts no longer apply
    return STENCIL_OK;
}

int stencil_set_tuning(stencil_t h, int scheme, const stencil_tuning* tuning) {
    if (!h) return STENCIL_EINVAL;
    if (scheme == STENCIL_PLAIN) {
        if (tuning && tuning->nf != 0 && tuning->nf != 2) return STENCIL_EINVAL;
        h->scheme = STENCIL_PLAIN;
        h->plain_prefetch = tuning ? tuning->nf : (h->kind == STENCIL_25PT_VAR && h->cdt == STENCIL_BF16 ? 2 : 0);
        return STENCIL_OK;
    }
    if (scheme == STENCIL_WAVEFRONT) {
        const int R = kind_radius(h->kind);
        WaveTune w{2, R > 8 ? R : 8, 8, 2, 0};  // default: two levels per pass, 8-plane chunks, 8-row tiles
        if (tuning) {
            if (tuning->dw < 2 * R || tuning->dw % (2 * R) != 0) return STENCIL_EINVAL;
            const bool tiles = tuning->xtile == 4 && h->kind == STENCIL_25PT_VAR && h->fdt == STENCIL_F32;
            if (tuning->xtile != 0 && tuning->xtile != 2 && !tiles) return STENCIL_EINVAL;
            w.h = tuning->dw / (2 * R);
            w.zc = tuning->nf;
            w.by = tuning->warps;
            w.cp = tuning->xtile;
        }
        const size_t need = wave_workspace_bytes(args_of(h), w);
        if (need == 0) return STENCIL_EINVAL;
        if (!h->ws || need > GRID_WORKSPACE_BYTES) return STENCIL_EINVAL;
        h->scheme = STENCIL_WAVEFRONT;
        h->wtune = w;
        return STENCIL_OK;
    }
    if (scheme != STENCIL_BLOCKED && scheme != STENCIL_AUTO) return STENCIL_EINVAL;
    if (scheme == STENCIL_AUTO && (h->fdt == DT_F64 || h->kind == STENCIL_25PT_VAR)) {
        // Measured on GB300: FP64 sweeps are bound by the FP64 units (1/60 of the FP32 rate),
        // where the blocked sweep's x-tile overlap only adds work, and the 25-point rings fit
        // only narrow x tiles; the plain sweep is faster for both.
        h->scheme = STENCIL_PLAIN;
        return STENCIL_OK;
    }
    BlockedTune t = default_tune(h);
    if (tuning && scheme == STENCIL_BLOCKED) {
        t.dw = tuning->dw;
        t.nf = tuning->nf;
        t.warps = tuning->warps;
        t.xtile = tuning->xtile;
    }
    int rc = check_tune(h, t);
    if (rc != STENCIL_OK) {
        if (scheme == STENCIL_AUTO) {
            h->scheme = STENCIL_PLAIN;
            return STENCIL_OK;
        }
        return rc;
    }
    h->scheme = STENCIL_BLOCKED;
    h->tune = t;
    h->tune_set = true;
    return STENCIL_OK;
}

int stencil_run(stencil_t h, int T) {
    if (!h || T < 0) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    if (T == 0) return STENCIL_OK;
    SweepArgs a = args_of(h);
    if ((h->scheme == STENCIL_BLOCKED || h->scheme == STENCIL_WAVEFRONT) && h->ws && !h->status_armed) {
        if (cudaMemsetAsync(static_cast<int*>(h->ws) + PERSIST_WS_STATUS, 0, sizeof(int), h->stream) != cudaSuccess)
            return STENCIL_ECUDA;
        h->status_armed = true;
    }
    if (h->scheme == STENCIL_WAVEFRONT) {
        cudaError_t e = wave_run(a, h->field, h->parity, T, h->wtune, h->ws, GRID_WORKSPACE_BYTES, h->ctl, h->stream,
                                 &h->launches, &h->tile_passes);
        if (e == cudaErrorInvalidValue) return STENCIL_EINVAL;
        if (e != cudaSuccess) return STENCIL_ECUDA;
    } else if (h->scheme == STENCIL_BLOCKED) {
        cudaError_t e = cudaErrorNotReady;
        if (h->ws) {
            // one persistent launch; if the plan for T steps does not fit one launch,
            // run the steps in two parts
            e = blocked_run_persistent(a, h->field, h->parity, T, h->tune, h->ws, GRID_WORKSPACE_BYTES, h->ctl,
                                       h->stream, &h->launches);
            if (e == cudaErrorNotReady && T > 1) {
                int rc = stencil_run(h, T / 2);
                if (rc != STENCIL_OK) return rc;
                return stencil_run(h, T - T / 2);
            }
        }
        if (e == cudaErrorNotReady) e = blocked_run(a, h->field, h->parity, T, h->tune, h->stream, &h->launches);
        if (e == cudaErrorInvalidValue) return STENCIL_EINVAL;
        if (e != cudaSuccess) return STENCIL_ECUDA;
    } else {
        for (int t = 0; t < T; ++t) {
            int p = (h->parity + t) & 1;
            cudaError_t e = plain_step(a, h->field[p], h->field[p ^ 1], h->stream);
            if (e != cudaSuccess) return STENCIL_ECUDA;
            ++h->launches;
        }
    }
    h->parity = (h->parity + T) & 1;
    return STENCIL_OK;
}

int stencil_parity(stencil_t h) { return h ? h->parity : STENCIL_EINVAL; }

int stencil_get_field(stencil_t h, void* dst, int where) {
    if (!h || !dst) return STENCIL_EINVAL;
    if (where != STENCIL_HOST && where != STENCIL_DEVICE && where != STENCIL_HOST_ASYNC) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    cudaError_t e = copy_interior(h, dtype_bytes(h->fdt), dst, h->field[h->parity], false, where == STENCIL_HOST_ASYNC);
    if (e == cudaErrorInvalidValue && where == STENCIL_HOST_ASYNC) return STENCIL_EINVAL;
    if (e != cudaSuccess) return STENCIL_ECUDA;
    if (where == STENCIL_HOST) return from_cuda(cudaStreamSynchronize(h->stream));
    return STENCIL_OK;
}

static int ckpt_k(int T, int ckpt_every) {
    if (ckpt_every > 0) return ckpt_every;
    int k = (int)ceil(sqrt((double)(T > 0 ? T : 1)));
    return k < 1 ? 1 : k;
}

size_t stencil_adjoint_workspace_bytes(stencil_t h, int T, int ckpt_every) {
    if (!h || T < 0) return 0;
    int k = ckpt_k(T, ckpt_every);
    int nck = T > 0 ? (T + k - 1) / k : 1;
    // checkpoints, the states of one segment, the k + 1 cotangents of one segment
    return (size_t)(nck + 2 * k + 1) * h->L.count() * (size_t)dtype_bytes(h->fdt);
}

int stencil_run_checkpointed(stencil_t h, int T, int ckpt_every, void* workspace, size_t workspace_bytes) {
    if (!h || T < 0 || !workspace) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    if (h->kind == STENCIL_7PT_CONST) return STENCIL_ENOTSUP;
    if (workspace_bytes < stencil_adjoint_workspace_bytes(h, T, ckpt_every)) return STENCIL_EINVAL;
    if (!aligned16(workspace)) return STENCIL_EINVAL;
    const int k = ckpt_k(T, ckpt_every);
    const int nck = T > 0 ? (T + k - 1) / k : 1;
    const size_t fb = h->L.count() * (size_t)dtype_bytes(h->fdt);
    char* ws = static_cast<char*>(workspace);
    int done = 0;
    for (int c = 0; c < nck; ++c) {
        cudaError_t e = cudaMemcpyAsync(ws + (size_t)c * fb, h->field[h->parity], fb, cudaMemcpyDeviceToDevice,
                                        h->stream);
        if (e != cudaSuccess) return STENCIL_ECUDA;
        int steps = (c + 1 < nck) ? k : T - done;
        int rc = stencil_run(h, steps);
        if (rc != STENCIL_OK) return rc;
        done += steps;
    }
    return STENCIL_OK;
}

int stencil_run_adjoint(stencil_t h, int T, int ckpt_every, const void* lambda_T, void* g_u0, void* const* g_coef,
                        void* workspace, size_t workspace_bytes) {
    if (!h || T < 0 || !lambda_T || !g_u0 || !g_coef || !workspace) return STENCIL_EINVAL;
    if (!h->bound) return STENCIL_EUNBOUND;
    if (h->kind == STENCIL_7PT_CONST) return STENCIL_ENOTSUP;
    if (workspace_bytes < stencil_adjoint_workspace_bytes(h, T, ckpt_every)) return STENCIL_EINVAL;
    const int nc = kind_ncoef(h->kind);
    for (int m = 0; m < nc; ++m)
        if (!g_coef[m] || !aligned16(g_coef[m])) return STENCIL_EINVAL;
    if (!aligned16(workspace) || !aligned16(g_u0) || !aligned16(lambda_T)) return STENCIL_EINVAL;
    const int k = ckpt_k(T, ckpt_every);
    const int nck = T > 0 ? (T + k - 1) / k : 1;
    const size_t cnt = h->L.count();
    const size_t fb = cnt * (size_t)dtype_bytes(h->fdt);
    char* ws = static_cast<char*>(workspace);
    auto ckpt = [&](int c) { return (void*)(ws + (size_t)c * fb); };
    auto state = [&](int j) { return (void*)(ws + (size_t)(nck + j) * fb); };  // j = 1 .. k-1 used
    // lambda_t lives in slot t mod (k + 1): the k + 1 cotangents of a segment, the segment's
    // last one shared with the next segment's first
    auto lam = [&](int t) { return (void*)(ws + (size_t)(nck + k + t % (k + 1)) * fb); };
    SweepArgs a = args_of(h);
    cudaStream_t s = h->stream;
    double* gC[13] = {};
    for (int m = 0; m < nc; ++m) {
        gC[m] = static_cast<double*>(g_coef[m]);
        if (fill_value(gC[m], cnt, DT_F64, 0.0, s) != cudaSuccess) return STENCIL_ECUDA;
        ++h->launches;
    }
    for (int i = 0; i <= k; ++i) {  // zero halos: the transpose's "p is interior" condition
        if (fill_value(ws + (size_t)(nck + k + i) * fb, cnt, h->fdt, 0.0, s) != cudaSuccess) return STENCIL_ECUDA;
        ++h->launches;
    }
    if (copy_interior_zero_halo(h->L, h->fdt, lambda_T, lam(T), s) != cudaSuccess) return STENCIL_ECUDA;
    ++h->launches;
    // in-segment states inherit the Dirichlet halo of u_0
    for (int j = 1; j < k; ++j)
        if (cudaMemcpyAsync(state(j), ckpt(0), fb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return STENCIL_ECUDA;
    for (int c = nck - 1; c >= 0 && T > 0; --c) {
        const int t0 = c * k;
        const int t1 = (t0 + k < T) ? t0 + k : T;
        auto st = [&](int j) { return j == 0 ? ckpt(c) : state(j); };
        bool done = false;
        if (h->scheme == STENCIL_WAVEFRONT && h->ws && t1 - t0 > 1 && t1 - t0 <= 64) {
            // the segment's states recomputed by one temporally blocked pass whose time levels
            // each write their own state array (a pass the workspace cannot plan falls back to
            // one plain step per state; nothing is launched in that case)
            if (!h->status_armed) {
                if (cudaMemsetAsync(static_cast<int*>(h->ws) + PERSIST_WS_STATUS, 0, sizeof(int), s) != cudaSuccess)
                    return STENCIL_ECUDA;
                h->status_armed = true;
            }
            void* lv[64];
            const int nlev = t1 - t0;  // states t0 .. t1 - 1
            for (int j = 0; j < nlev; ++j) lv[j] = st(j);
            cudaError_t e = wave_run_levels(a, lv, nlev, h->wtune, h->ws, GRID_WORKSPACE_BYTES, h->ctl, s, &h->launches);
            if (e != cudaSuccess && e != cudaErrorInvalidValue) return STENCIL_ECUDA;
            done = e == cudaSuccess;
        }
        for (int j = 1; j < t1 - t0 && !done; ++j) {
            if (plain_step(a, st(j - 1), st(j), s) != cudaSuccess) return STENCIL_ECUDA;
            ++h->launches;
        }
        // the cotangents of the segment: with the wavefront schedule tuned, one temporally blocked
        // pass of transposed steps whose levels each write their own cotangent array; otherwise
        // one transposed step per launch
        bool lam_done = false;
        if (h->scheme == STENCIL_WAVEFRONT && h->ws && t1 - t0 <= 64) {
            void* lv[65];
            for (int i = 0; i <= t1 - t0; ++i) lv[i] = lam(t1 - i);
            cudaError_t e = wave_run_levels(a, lv, t1 - t0 + 1, h->wtune, h->ws, GRID_WORKSPACE_BYTES, h->ctl, s,
                                            &h->launches, true);
            if (e != cudaSuccess && e != cudaErrorInvalidValue) return STENCIL_ECUDA;
            lam_done = e == cudaSuccess;
        }
        for (int t = t1 - 1; t >= t0 && !lam_done; --t) {
            if (adjoint_step(a, lam(t + 1), lam(t), s) != cudaSuccess) return STENCIL_ECUDA;
            ++h->launches;
        }
        // then the coefficient gradients of all its steps in one pass (t = t1 - 1 down to t0)
        const void* lams[64];
        const void* us[64];
        int n = 0;
        for (int t = t1 - 1; t >= t0; --t, ++n) {
            if (n == 64) {
                if (adjoint_grads(a, lams, us, n, gC, s) != cudaSuccess) return STENCIL_ECUDA;
                h->launches += (n + 15) / 16;
                n = 0;
            }
            lams[n] = lam(t + 1);
            us[n] = st(t - t0);
        }
        if (adjoint_grads(a, lams, us, n, gC, s) != cudaSuccess) return STENCIL_ECUDA;
        h->launches += (n + 15) / 16;
    }
    if (cudaMemcpyAsync(g_u0, lam(0), fb, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return STENCIL_ECUDA;
    return STENCIL_OK;
}

size_t stencil_blocked_smem_bytes(stencil_t h, const stencil_tuning* tuning) {
    if (!h || !tuning) return 0;
    BlockedTune t{tuning->dw, tuning->nf, tuning->warps, tuning->xtile};
    return blocked_smem_bytes(args_of(h), t);
}

int stencil_launch_count(stencil_t h, long long* out) {
    if (!h || !out) return STENCIL_EINVAL;
    *out = h->launches;
    return STENCIL_OK;
}

int stencil_tile_copy_passes(stencil_t h, long long* out) {
    if (!h || !out) return STENCIL_EINVAL;
    *out = h->tile_passes;
    return STENCIL_OK;
}

int stencil_copy(void* dst, const void* src, size_t bytes, int ctas, void* cuda_stream) {
    if (!dst || !src || ctas < 1 || ctas > 1024) return STENCIL_EINVAL;
    void* d = device_view(dst);
    const void* s = device_view(src);
    if (!d || !s) return STENCIL_EINVAL;
    if ((((uintptr_t)d | (uintptr_t)s | bytes) & 15u) != 0) return STENCIL_EINVAL;
    if (dense_copy(d, s, bytes, ctas, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) return STENCIL_ECUDA;
    return STENCIL_OK;
}

// ------------------------------------------------------------------ batch

struct stencil_batch {
    std::vector<stencil_t> grids;
    std::vector<int> T;
    BlockedTune tn;
    BatchLaunch bl;
    bool bound = false;
    cudaStream_t stream = nullptr;
    long long launches = 0;
};

static void batch_grids(const stencil_batch* b, std::vector<BatchGrid>& g) {
    g.resize(b->grids.size());
    for (size_t q = 0; q < b->grids.size(); ++q) {
        const stencil_grid* h = b->grids[q];
        g[q].a = args_of(h);
        g[q].field[0] = h->field[0];
        g[q].field[1] = h->field[1];
        g[q].parity = h->parity;
        g[q].T = b->T[q];
    }
}

int stencil_batch_create(stencil_batch_t* out, const stencil_t* grids, const int* T, int n,
                         const stencil_tuning* tuning) {
    if (!out || !grids || !T || n < 1 || !tuning) return STENCIL_EINVAL;
    *out = nullptr;
    for (int q = 0; q < n; ++q) {
        if (!grids[q] || T[q] < 0) return STENCIL_EINVAL;
        if (!grids[q]->bound) return STENCIL_EUNBOUND;
    }
    stencil_batch* b = new (std::nothrow) stencil_batch();
    if (!b) return STENCIL_EINVAL;
    b->grids.assign(grids, grids + n);
    b->T.assign(T, T + n);
    b->tn = BlockedTune{tuning->dw, tuning->nf, tuning->warps, 0};
    std::vector<BatchGrid> g;
    batch_grids(b, g);
    cudaError_t e = batch_plan(g.data(), n, b->tn, &b->bl);
    if (e != cudaSuccess) {
        delete b;
        return STENCIL_EINVAL;
    }
    *out = b;
    return STENCIL_OK;
}

size_t stencil_batch_workspace_bytes(stencil_batch_t b) { return b ? b->bl.bytes : 0; }

int stencil_batch_item_count(stencil_batch_t b) { return b ? b->bl.nitems : STENCIL_EINVAL; }

int stencil_batch_bind(stencil_batch_t b, void* workspace, void* cuda_stream) {
    if (!b || !workspace || !aligned16(workspace)) return STENCIL_EINVAL;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap) != cudaSuccess) return STENCIL_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return STENCIL_EINVAL;  // the upload waits for the stream
    std::vector<BatchGrid> g;
    batch_grids(b, g);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    if (batch_upload(g.data(), (int)g.size(), b->tn, &b->bl, workspace, b->stream) != cudaSuccess)
        return STENCIL_ECUDA;
    b->bound = true;
    return STENCIL_OK;
}

int stencil_batch_launch(stencil_batch_t b, void* cuda_stream) {
    if (!b) return STENCIL_EINVAL;
    if (!b->bound) return STENCIL_EUNBOUND;
    if (batch_launch(b->bl, static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) return STENCIL_ECUDA;
    b->launches += 2;  // counter reset + persistent kernel
    for (size_t q = 0; q < b->grids.size(); ++q) b->grids[q]->parity = (b->grids[q]->parity + b->T[q]) & 1;
    return STENCIL_OK;
}

int stencil_batch_launch_count(stencil_batch_t b, long long* out) {
    if (!b || !out) return STENCIL_EINVAL;
    *out = b->launches;
    return STENCIL_OK;
}

int stencil_batch_status(stencil_batch_t b, int* status) {
    if (!b || !status) return STENCIL_EINVAL;
    if (!b->bound) return STENCIL_EUNBOUND;
    int v = 0;
    if (cudaMemcpy(&v, b->bl.ws + b->bl.off_counters + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return STENCIL_ECUDA;
    *status = v == 0 ? STENCIL_OK : STENCIL_ETIMEOUT;
    return STENCIL_OK;
}

int stencil_batch_sync_parity(stencil_batch_t b) {
    if (!b) return STENCIL_EINVAL;
    if (!b->bound) return STENCIL_EUNBOUND;
    std::vector<int> par(b->grids.size());
    if (cudaMemcpy(par.data(), b->bl.ws + b->bl.off_parity, sizeof(int) * par.size(), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return STENCIL_ECUDA;
    for (size_t q = 0; q < par.size(); ++q) b->grids[q]->parity = par[q] & 1;
    return STENCIL_OK;
}

int stencil_batch_set_wait_limit(stencil_batch_t b, unsigned spins) {
    if (!b || spins == 0) return STENCIL_EINVAL;
    b->bl.spin_limit = spins;
    return STENCIL_OK;
}

int stencil_batch_inject_stall(stencil_batch_t b, int item) {
    if (!b || item < 0 || item >= b->bl.nitems) return STENCIL_EINVAL;
    if (!b->bound) return STENCIL_EUNBOUND;
    b->bl.items[item].dep[2] = b->bl.nitems;  // the extra completion flag, which no tile ever sets
    if (batch_reupload_items(&b->bl, b->stream) != cudaSuccess) return STENCIL_ECUDA;
    return STENCIL_OK;
}

int stencil_batch_destroy(stencil_batch_t b) {
    if (!b) return STENCIL_EINVAL;
    delete b;
    return STENCIL_OK;
}

int stencil_set_stream(stencil_t h, void* cuda_stream) {
    if (!h) return STENCIL_EINVAL;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return STENCIL_OK;
}

// The persistent schedule's status word (synchronous): STENCIL_OK or STENCIL_ETIMEOUT.
static int read_status(stencil_t h) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return STENCIL_ECUDA;
    if (!h->bound || !h->ws || !h->status_armed) return STENCIL_OK;
    int v = 0;
    if (cudaMemcpyAsync(&v, static_cast<int*>(h->ws) + PERSIST_WS_STATUS, sizeof(int), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
        return STENCIL_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return STENCIL_ECUDA;
    return v == 0 ? STENCIL_OK : STENCIL_ETIMEOUT;
}

int stencil_sync(stencil_t h) {
    if (!h) return STENCIL_EINVAL;
    return read_status(h);
}

int stencil_status(stencil_t h) {
    if (!h) return STENCIL_EINVAL;
    return read_status(h);
}

int stencil_set_wait_limit(stencil_t h, unsigned spins) {
    if (!h || spins == 0) return STENCIL_EINVAL;
    h->ctl.spin_limit = spins;
    return STENCIL_OK;
}

int stencil_inject_stall(stencil_t h, int tile) {
    if (!h || tile < -1) return STENCIL_EINVAL;
    h->ctl.stall_item = tile;
    return STENCIL_OK;
}

const char* stencil_strerror(int status) {
    switch (status) {
        case STENCIL_OK: return "ok";
        case STENCIL_EINVAL: return "invalid argument";
        case STENCIL_ENOSMEM: return "blocked tuning exceeds the shared-memory limit";
        case STENCIL_ETIMEOUT: return "device-side wait timed out";
        case STENCIL_ECUDA: return "CUDA runtime error";
        case STENCIL_EUNBOUND: return "arrays not bound";
        case STENCIL_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

int stencil_destroy(stencil_t h) {
    if (!h) return STENCIL_EINVAL;
    delete h;
    return STENCIL_OK;
}

}  // extern "C"
