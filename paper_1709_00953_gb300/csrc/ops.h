// Launchers of the Siddon operators (ops.cu), used by the C ABI and the solver.
#pragma once
#include <cuda_runtime.h>

#include "common.h"

namespace csgd {

constexpr int kHistCols = 5;

// Items passed by value to the stand-alone operators (kernel parameter space).
constexpr int kMaxInlineItems = 900;

struct InlineItems {
    StepDesc step;
    int32_t n;
    int32_t pad;
    WorkItem items[kMaxInlineItems];
};

// Backprojection decomposition: the tile is cut along its last axis into `nsb`
// sub-boxes that fit in shared memory; `C` CTAs (one cluster) share the rays of
// one (slot, sub-box) and reduce their partial sub-boxes through distributed
// shared memory.
struct BPPlan {
    int nsb;
    int C;
    int smem_bytes;
};
BPPlan plan_backprojection(const DevGeom& G, const DevTile& tile, int nslots, int sm_count);

// ---- stand-alone operators (inline items, one slot) -------------------------
// out[ray] = (accumulate ? out[ray] : 0) + h * sum A x over the items' rays.
cudaError_t launch_project_inline(const DevGeom& G, const InlineItems& it, const float* x,
                                  float* out, int accumulate, cudaStream_t s);
// g[v] = (accumulate ? g[v] : 0) + h * sum A^T r, v in tile it.step.j (row-major volume).
cudaError_t launch_backproject_inline(const DevGeom& G, const DevTile& tile,
                                      const InlineItems& it, const float* r, float* g,
                                      int accumulate, int sm_count, cudaStream_t s);

// ---- solver operators (device item / step arrays, several slots) -----------
struct SolverBuffers {
    // state
    float* x;        // tile-major volume
    float* xh;       // candidate sums (tile-major)
    int32_t* cnt;    // per tile
    const float* y;
    float* r;
    float* z;        // z store on the per (view, tile) shadow rectangles
    float* d;        // pending residual change (epoch sync), or null
    // scratch
    float* p;        // A x_J per ray
    float* q;        // A g_J per ray
    float* g;        // g_J per slot, tile-local [slot][max_tile_voxels]
    double* gg_part; // [slot][nsb * C]
    double* qq_part; // [slot][max_fwd_blocks]
    unsigned int* counters;  // [slot]
    double* mu;      // [slot]
    double* hist;    // [step][kHistCols] = beta, gg, qq, mu, nnz
    unsigned long long* nnz;       // non-zeros visited since the last reset
    unsigned long long* nnz_slot;  // [slot] non-zeros of the current batch
    int64_t g_stride;
    int max_fwd_blocks;
    int max_slots;
    int64_t hist_cap;
};

struct BatchLaunch {
    int first;       // first step descriptor of the batch
    int nslots;      // steps in the batch (all on tile j)
    int j;
    int64_t max_rays;
    int sync_epoch;
};

// ev (optional, 4 events): recorded before the backprojection, after it, after
// the forward products and after the epilogue.
cudaError_t launch_batch(const DevGeom& G, const DevTile& tile, const WorkItem* items,
                         const StepDesc* steps, const BatchLaunch& b, const SolverBuffers& sb,
                         int sm_count, cudaStream_t s, cudaEvent_t* ev = nullptr);
cudaError_t launch_epoch_close(const DevGeom& G, const SolverBuffers& sb, int64_t n_rays,
                               int64_t max_tile_voxels, int sync_epoch, cudaStream_t s);
cudaError_t launch_tile_to_rowmajor(const DevGeom& G, const float* xt, float* out,
                                    int64_t max_tile_voxels, cudaStream_t s);
cudaError_t launch_sq_residual(const float* y, const float* ax, int64_t n, double* out,
                               cudaStream_t s);

}  // namespace csgd
