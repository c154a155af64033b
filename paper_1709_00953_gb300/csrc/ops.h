// Launchers of the Siddon operators (ops.cu), used by the C ABI and the solver.
#pragma once
#include <cuda_runtime.h>

#include "../../include/csgd.h"
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

// Backprojection launch: `blocks` CTAs per slot, each owning a patch of kBPVox
// voxels of the tile (8 x 8 in 2D, 4 x 4 x 4 in 3D) with its views split among
// C thread groups of kBPVox threads.
constexpr int kFwdThreads = 128;  // threads of a dual-forward CTA (256 and 64 measured slower)
constexpr int kBPVox = 64;
constexpr int kBPMaxChunks = 8;  // view groups per CTA at most
constexpr int kBPScatter = -1;   // bp_groups value selecting the scatter backprojection
constexpr int kBPBrick = -2;     // bp_groups values -2, -3, -4 select the brick
constexpr int kBPBrickLast = -4; // backprojection with brick shape 0, 1, 2
inline int bp_patch(int dim, int axis) { return dim == 2 ? (axis < 2 ? 8 : 1) : 4; }
inline int bp_blocks(const DevTile& t, int dim) {
    int b = 1;
    for (int a = 0; a < 3; ++a) b *= (t.n[a] + bp_patch(dim, a) - 1) / bp_patch(dim, a);
    return b;
}
struct BPPlan {
    int blocks;  // CTAs per slot (one g^T g partial each)
    int C;       // view groups per CTA
};
BPPlan plan_backprojection(const DevGeom& G, const DevTile& tile, int nslots, int views,
                           int sm_count, int force_groups = 0);

// ---- stand-alone operators (inline items, one slot) -------------------------
// out[ray] = (accumulate ? out[ray] : 0) + h * sum A x over the items' rays.
cudaError_t launch_project_inline(const DevGeom& G, const InlineItems& it, const float* x,
                                  float* out, int accumulate, int sm_count, cudaStream_t s);
// threads per ray of the forward kernels for a launch over `rays` rays
int lanes_per_ray(int64_t rays, int sm_count);
// g[v] = (accumulate ? g[v] : 0) + h * sum A^T r, v in tile it.step.j (row-major volume).
// `table` must hold it.step.n_rays records (device scratch).
cudaError_t launch_backproject_inline(const DevGeom& G, const DevTile& tile,
                                      const InlineItems& it, const float* r, float* g,
                                      int accumulate, RayRec* table, int sm_count,
                                      cudaStream_t s);

// ---- backprojection without allocation (fixed ray table in global memory) --
constexpr int kNoAllocMaxRays = CSGD_NOALLOC_MAX_RAYS;
constexpr int kNoAllocMaxDevices = 64;
// Device address of the fixed ray table, looked up once per device (the current
// one) with cudaGetSymbolAddress.
cudaError_t noalloc_table_address(int device, RayRec** out);

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
    float* g;        // (x_J, g_J) pairs per slot, tile-local [slot][g_stride][2]
    float* gg_part;  // [slot][gg_stride]: g^T g per backprojection CTA (FP32)
    unsigned long long* acc;  // [slot][g_stride]: fixed-point g_J of the scatter
                              // backprojection (zero between batches)
    unsigned int* rmax;       // [slot]: bits of max |r| over the batch's rays (zero
                              // between batches)
    int gg_stride;
    RayRec* table;   // [slot][table_stride]: ray table of the batch
    int64_t table_stride;
    float* qq_part;  // [slot][qq_stride]: q^T q per forward CTA (FP32)
    int qq_stride;
    unsigned int* counters;  // [slot]
    double* mu;      // [slot]
    double* hist;    // [step][kHistCols] = beta, gg, qq, mu, nnz
    unsigned long long* nnz;       // non-zeros visited since the last reset
    unsigned long long* nnz_slot;  // [slot] non-zeros of the current batch
    int64_t g_stride;
    int max_fwd_blocks;   // per slot, at 4 lanes per ray
    int max_slots;
    int64_t hist_cap;
};

struct BatchLaunch {
    int first;       // first step descriptor of the batch
    int nslots;      // steps in the batch (all on tile j)
    int j;
    int64_t max_rays;        // rays of the largest step
    int w_begin, n_items;    // work items of the batch (contiguous)
    int64_t max_item_rays;   // rays of the largest work item
    int sync_epoch;
    int bp_groups = 0;       // view groups per backprojection CTA (0: occupancy model;
                             // kBPScatter: ray-driven scatter backprojection;
                             // kBPBrick: brick backprojection, no ray table)
    int fwd_lanes = 0;       // lanes per ray of the dual forward (0: by ray count)
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

// ---- batch executor: the kernels of many solves in one persistent launch ----
struct ExecPlan;
ExecPlan* exec_plan_new(int n_problems);
void exec_plan_free(ExecPlan* p);
// the kernels of one batch of problem `problem`'s solve (see launch_batch)
cudaError_t exec_plan_add_batch(ExecPlan* p, int problem, const DevGeom& G, const DevTile& tile,
                                const WorkItem* items, const StepDesc* steps, const BatchLaunch& b,
                                const SolverBuffers& sb, int sm_count);
// an epoch close (see launch_epoch_close) and the row-major copy of x
void exec_plan_add_close(ExecPlan* p, int problem, const DevGeom& G, const SolverBuffers& sb,
                         int64_t n_rays, int64_t max_tile_voxels, int sync_epoch);
void exec_plan_add_xout(ExecPlan* p, int problem, const DevGeom& G, const float* xt, float* out,
                        int64_t max_tile_voxels);
// interleave and upload; wait_ns bounds every wait; stall_last makes the last
// task of problem 0 wait for a unit that never completes (tests of the bound)
cudaError_t exec_plan_finalize(ExecPlan* p, int64_t wait_ns, int stall_last, int sm_count);
// counters cleared, then the persistent launch (capturable into a graph)
cudaError_t exec_plan_launch(ExecPlan* p, cudaStream_t s);
// 0, or 1 when a wait of the last launch ran out (synchronous)
cudaError_t exec_plan_status(ExecPlan* p, int* status);
void exec_plan_info(const ExecPlan* p, int* n_tasks, int64_t* n_units, int* grid);

}  // namespace csgd
