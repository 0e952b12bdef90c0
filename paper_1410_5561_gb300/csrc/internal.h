// Internal interface between the C-ABI layer (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "common.cuh"

struct stencil_grid;  // the C ABI's grid handle (api.cu)

namespace stg {

enum DType { DT_F32 = 0, DT_F64 = 1, DT_BF16 = 2 };

inline int dtype_bytes(int dt) { return dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2); }
inline int kind_radius(int kind) { return kind == K25V ? 4 : 1; }
inline int kind_ncoef(int kind) { return kind == K7C ? 0 : (kind == K7V ? 7 : 13); }

// Everything a sweep kernel needs to know about one grid.
struct SweepArgs {
    int kind;              // K7C / K7V / K25V
    int fdt;               // field dtype: DT_F32 or DT_F64
    int cdt;               // coefficient dtype: DT_F32, DT_F64 or DT_BF16
    Layout L;
    const void* coef[13];  // padded coefficient arrays (device)
    double c0, c1;         // Listing 1 scalars (7-point constant)
    double halo;           // Dirichlet value of every halo cell
    int plain_prefetch;    // plain sweep: planes each thread copies ahead into shared memory (0 or 2)
};

// Blocked-sweep tunables (D_w, N_F, warps per CTA, x-tile width).
struct BlockedTune {
    int dw;       // diamond width in y (multiple of 2R)
    int nf;       // frontlines: z-planes per level per wavefront step
    int warps;    // warps per CTA
    int xtile;    // x columns owned by one CTA (multiple of the vector width)
};

// One plain step: dst(interior) = A src.
cudaError_t plain_step(const SweepArgs& a, const void* src, void* dst, cudaStream_t s);

// Fill n elements of dtype dt at p with value v.
cudaError_t fill_value(void* p, size_t n, int dt, double v, cudaStream_t s);
// bytes (a multiple of 16, both pointers 16-byte aligned) from src to dst by `ctas` CTAs of
// 1024 threads; either side may be page-locked host memory.
cudaError_t dense_copy(void* dst, const void* src, size_t bytes, int ctas, cudaStream_t s);
// Dense interior rows <-> padded layout (src/dst device or device-mapped host pointers).
cudaError_t copy_rows(const Layout& L, int eb, const void* src, void* dst, bool to_padded, cudaStream_t s);

// Temporally blocked run of T steps from parity p0 (array (p0 + t) & 1 holds u_t).
// Returns cudaErrorInvalidValue for an infeasible tuning, after checking it on the host.
cudaError_t blocked_run(const SweepArgs& a, void* const field[2], int p0, int T,
                        const BlockedTune& tune, cudaStream_t s, long long* launches);

// One transposed step of the adjoint's cotangent recursion: lam_out = A^T lam_in over the interior.
cudaError_t adjoint_step(const SweepArgs& a, const void* lam_in, void* lam_out, cudaStream_t s);

// Coefficient gradients of n steps in one pass per group of up to 16 steps:
// gC[m] += lam[g] * (field value multiplying C_m in the step whose state is u[g]),
// g = 0 .. n-1 in that order (lam[g] = lambda_{t+1} for the state u[g] = u_t).
cudaError_t adjoint_grads(const SweepArgs& a, const void* const* lam, const void* const* u, int n, double* const* gC,
                          cudaStream_t s);

// dst = src on the interior, 0 on every other cell (FP32 / FP64).
cudaError_t copy_interior_zero_halo(const Layout& L, int dt, const void* src, void* dst, cudaStream_t s);

// Controls of a persistent single-grid launch.
struct PersistCtl {
    unsigned spin_limit;  // bound on the spin iterations of one dependency wait
    int stall_item;       // test hook: tile that also waits on a flag no tile sets (-1: none)
};
// Words (ints) of a grid workspace used by the persistent schedule: the status word
// (sticky: set to 1 when a dependency wait gives up), a flag no tile ever sets, then
// one completion counter per tile.
constexpr int PERSIST_WS_STATUS = 0, PERSIST_WS_NEVER = 1, PERSIST_WS_DONE = 2;

// Blocked run of T steps by one persistent launch whose clusters walk the
// dependency-ordered tile list (derived on the device from a row table passed as a
// kernel parameter; ws holds only the status word and the counters).
// cudaErrorNotReady: the plan for T steps does not fit one launch.
cudaError_t blocked_run_persistent(const SweepArgs& a, void* const field[2], int p0, int T, const BlockedTune& tune,
                                   void* ws, size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s,
                                   long long* launches);

// Workspace a grid handle asks for: the persistent schedules' status word and
// completion counters.
constexpr size_t GRID_WORKSPACE_BYTES = size_t(16) << 20;

// Wavefront schedule through L2 (wavefront.cu): h time levels per pass, z chunks of
// zc planes, xy tiles of 32 vectors by `by` rows (one CTA), level l trailing level
// l-1 by `lag` chunks.
struct WaveTune {
    int h, zc, by, lag;
    int cp;  // 0; 2: each thread copies its loads two planes ahead into shared memory;
             // 4: tensor copies of whole tiles into shared memory (25-point, FP32 field)
};
// Workspace words (ints) of the wavefront schedule: the status word (shared with the
// persistent blocked schedule), a flag no unit sets, the unit counter, then one
// completion flag per unit.
constexpr int WAVE_WS_STATUS = 0, WAVE_WS_NEVER = 1, WAVE_WS_HEAD = 2, WAVE_WS_FLAGS = 3;
// Workspace bytes one pass of h levels needs (0 if the tuning is malformed for the grid).
size_t wave_workspace_bytes(const SweepArgs& a, const WaveTune& tn);
// One pass whose time level l reads levels[l] and writes levels[l + 1] (nlev - 1 levels,
// at most 64), so that every intermediate state is kept. With transposed, each level is the
// adjoint's transposed step (levels[l + 1] = A^T levels[l]; variable-coefficient stencils).
cudaError_t wave_run_levels(const SweepArgs& a, void* const* levels, int nlev, const WaveTune& tn, void* ws,
                            size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s, long long* launches,
                            bool transposed = false);
// T steps in passes of tn.h levels, one launch per pass.
cudaError_t wave_run(const SweepArgs& a, void* const field[2], int p0, int T, const WaveTune& tn, void* ws,
                     size_t ws_bytes, const PersistCtl& ctl, cudaStream_t s, long long* launches,
                     long long* tile_passes = nullptr);
// One forward pass of the 25-point stencil (FP32 field) whose operands are staged in shared
// memory by tensor copies (wave_tma.cu); levels[l] -> levels[l + 1], h levels alternating between
// two arrays. cudaErrorNotReady when the grid, tuning or device does not allow it (the caller
// then runs the column-walk form).
cudaError_t wave_tma_pass(const SweepArgs& a, void* const* levels, int h, const WaveTune& tn, int* ws,
                          const PersistCtl& ctl, cudaStream_t st, long long* launches);

// Shared-memory bytes the blocked kernel needs for a tuning (0 if infeasible).
size_t blocked_smem_bytes(const SweepArgs& a, const BlockedTune& tune);

// ---- persistent batch of grids (blocked schedule, one launch)
struct BatchItem {
    int g, k, b;   // grid, diamond row, diamond
    int dep[3];    // items this one waits for (-1: none)
};

struct BatchGrid {
    SweepArgs a;
    void* field[2];
    int parity;  // array holding the grid's current time level
    int T;       // steps to advance
};

struct BatchLaunch {
    int kind, fdt, cdt, K, nf, threads, ngrids, nitems;
    size_t smem, bytes, counter_bytes;
    size_t off_grids, off_items, off_ntiles, off_parity, off_counters;
    unsigned spin_limit = 1u << 24;
    char* ws = nullptr;
    std::vector<BatchItem> items;
    std::vector<int> ntiles;
};

cudaError_t batch_plan(const BatchGrid* g, int n, const BlockedTune& tn, BatchLaunch* bl);
cudaError_t batch_upload(const BatchGrid* g, int n, const BlockedTune& tn, BatchLaunch* bl, void* ws, cudaStream_t s);
cudaError_t batch_reupload_items(BatchLaunch* bl, cudaStream_t s);
cudaError_t batch_launch(const BatchLaunch& bl, cudaStream_t s);

// Read access to a bound grid handle for batch planning (STENCIL_EUNBOUND if unbound),
// and the parity update after a batch launch.
int grid_batch_view(const stencil_grid* h, SweepArgs* a, void** f0, void** f1, int* parity);
void grid_set_parity(stencil_grid* h, int parity);

}  // namespace stg
