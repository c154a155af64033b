// The C ABI of include/csgd.h: handles, argument checks, device tables and the
// solver's host-side schedule (Alg. 2 / 3 / 4 around the Alg. 1 step).
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/csgd.h"
#include "host.h"
#include "ops.h"

using namespace csgd;

struct csgd_geometry {
    Geometry g;
};

struct csgd_partition {
    Partition p;
    std::mutex mu;
    bool on_device = false;
    int sm_count = 0;
    int64_t max_rays_per_block_tile = 0;  // max over (i, j) of rays of row block i in tile j
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? CSGD_ERR_OOM : CSGD_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define CSGD_CUDA(call, where)                       \
    do {                                             \
        cudaError_t _e = (call);                     \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

// Upload the partition's tables to the current device on first use.
int ensure_device(csgd_partition* P) {
    std::lock_guard<std::mutex> lk(P->mu);
    int dev = 0;
    CSGD_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (P->on_device) {
        if (dev != P->p.device)
            return fail(CSGD_ERR_INVALID_ARG, "partition tables live on another device");
        return CSGD_OK;
    }
    Partition& p = P->p;
    p.device = dev;
    CSGD_CUDA(cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, dev),
              "cudaDeviceGetAttribute");
    size_t bv = sizeof(DevView) * p.views_h.size();
    size_t bv64 = sizeof(DevView64) * p.views64_h.size();
    size_t bt = sizeof(DevVT) * p.vt_h.size();
    size_t bti = sizeof(DevTile) * p.tiles_h.size();
    cudaError_t e = cudaMalloc(&p.d_views, bv);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_views64, bv64);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_vt, bt);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_tiles, bti);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_views, p.views_h.data(), bv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p.d_views64, p.views64_h.data(), bv64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_vt, p.vt_h.data(), bt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_tiles, p.tiles_h.data(), bti, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        // leave the partition as it was: nothing on the device
        cudaFree(p.d_views);
        cudaFree(p.d_views64);
        cudaFree(p.d_vt);
        cudaFree(p.d_tiles);
        p.d_views = nullptr;
        p.d_views64 = nullptr;
        p.d_vt = nullptr;
        p.d_tiles = nullptr;
        return cuda_fail(e, "upload partition tables");
    }
    p.dg.views = p.d_views;
    p.dg.views64 = p.d_views64;
    p.dg.vt = p.d_vt;
    p.dg.tiles = p.d_tiles;
    P->on_device = true;
    return CSGD_OK;
}

int check_rows(const Partition& p, const int32_t* rows, int32_t n_rb) {
    if (n_rb < 1 || !rows) return fail(CSGD_ERR_INVALID_ARG, "need at least one row block");
    std::vector<char> seen(p.m, 0);
    for (int k = 0; k < n_rb; ++k) {
        if (rows[k] < 0 || rows[k] >= p.m) return fail(CSGD_ERR_INVALID_ARG, "row block out of range");
        if (seen[rows[k]]) return fail(CSGD_ERR_INVALID_ARG, "row blocks must be distinct");
        seen[rows[k]] = 1;
    }
    return CSGD_OK;
}

// Items of the stand-alone operators: every view of every row block, over the
// whole sub-rectangle (rays that miss the tile produce exact zeros) when
// `full_subrect`, else clipped to the tile's shadow rectangle.
void items_for_rows(const Partition& p, const int32_t* rows, int n_rb, int j, bool full_subrect,
                    std::vector<WorkItem>* out) {
    for (int r = 0; r < n_rb; ++r) {
        int su0, su1, sv0, sv1;
        p.subrect(rows[r], &su0, &su1, &sv0, &sv1);
        for (int v : p.views_of(rows[r])) {
            WorkItem w;
            w.view = v;
            w.slot = 0;
            if (full_subrect) {
                w.u0 = su0; w.u1 = su1; w.v0 = sv0; w.v1 = sv1;
            } else {
                const DevVT& e = p.vt(v, j);
                w.u0 = std::max(su0, e.u0); w.u1 = std::min(su1, e.u1);
                w.v0 = std::max(sv0, e.v0); w.v1 = std::min(sv1, e.v1);
                if (w.u1 <= w.u0 || w.v1 <= w.v0) continue;
            }
            w.ray_off = 0;
            out->push_back(w);
        }
    }
}

// Launch the stand-alone forward / backward operator over `items` in chunks
// that fit the kernel parameter space.
int run_inline(csgd_partition* P, const std::vector<WorkItem>& items, int j, bool forward,
               const float* in, float* out, int accumulate, cudaStream_t s) {
    const Partition& p = P->p;
    InlineItems* it = new (std::nothrow) InlineItems;
    if (!it) return fail(CSGD_ERR_OOM, "host allocation");
    size_t pos = 0;
    bool first = true;
    int rc = CSGD_OK;
    while (pos < items.size() || first) {
        size_t cnt = std::min(items.size() - pos, (size_t)kMaxInlineItems);
        memset(&it->step, 0, sizeof(it->step));
        it->step.j = j;
        it->step.w0 = 0;
        it->step.w1 = (int32_t)cnt;
        it->n = (int32_t)cnt;
        int64_t rays = 0;
        for (size_t k = 0; k < cnt; ++k) {
            it->items[k] = items[pos + k];
            it->items[k].ray_off = rays;
            rays += (int64_t)(it->items[k].u1 - it->items[k].u0) * (it->items[k].v1 - it->items[k].v0);
        }
        it->step.n_rays = rays;
        int acc = (first ? accumulate : 1);
        cudaError_t e;
        if (forward) {
            e = launch_project_inline(p.dg, *it, in, out, accumulate, P->sm_count, s);
        } else if (cnt == 0) {
            // no rays: g = 0 on the tile unless accumulating
            if (!acc) {
                InlineItems empty;
                memset(&empty.step, 0, sizeof(empty.step));
                empty.step.j = j;
                empty.n = 0;
                e = launch_backproject_inline(p.dg, p.tiles_h[j], empty, in, out, 0, nullptr,
                                              P->sm_count, s);
            } else {
                e = cudaSuccess;
            }
        } else {
            RayRec* table = nullptr;
            e = cudaMallocAsync((void**)&table, sizeof(RayRec) * (size_t)rays, s);
            if (e == cudaSuccess) {
                e = launch_backproject_inline(p.dg, p.tiles_h[j], *it, in, out, acc, table,
                                              P->sm_count, s);
                cudaError_t e2 = cudaFreeAsync(table, s);
                if (e == cudaSuccess) e = e2;
            }
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, forward ? "project kernel" : "backproject kernel");
            break;
        }
        pos += cnt;
        first = false;
        if (cnt == 0) break;
    }
    delete it;
    return rc;
}

}  // namespace

// ===========================================================================
// Solver
// ===========================================================================
struct QueuedStep {
    int j;
    std::vector<int> group;
    bool last_in_batch;
};

struct csgd_solver {
    csgd_partition* P = nullptr;
    csgd_solver_params prm{};
    SolverBuffers sb{};
    int64_t n_rays = 0, n_vox = 0;
    SplitMix64 rng{0};
    int64_t epoch = 0;       // epochs closed
    int64_t steps_done = 0;  // since the last reset
    std::deque<QueuedStep> queue;  // rest of the current epoch
    bool epoch_open = false;        // candidates accumulated since the last close
    int max_slots = 1;
    int last_group = 0;             // row blocks of the last planned step
    int bp_groups = 0;              // launch shapes (0: the library's models)
    int fwd_lanes = 0;
    int64_t max_rays_per_step = 0;
    // device arrays for the schedule of one solve call
    WorkItem* d_items = nullptr;
    int64_t items_cap = 0;
    StepDesc* d_steps = nullptr;
    int64_t steps_cap = 0;
    // temporaries for the residual norm
    float* d_xrow = nullptr;
    float* d_ax = nullptr;
    double* d_sq = nullptr;
    int64_t bytes = 0;
    std::vector<void*> allocs;
    // optional per-kernel timing with CUDA events
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec {
        int kind;
        int e0, e1;
    };
    std::vector<Rec> recs;
    size_t ev_used = 0;
};

namespace {

int dmalloc(csgd_solver* S, void** ptr, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(ptr, bytes == 0 ? 16 : bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return cuda_fail(e, what);
    }
    S->allocs.push_back(*ptr);
    S->bytes += (int64_t)bytes;
    return CSGD_OK;
}

void dfree(csgd_solver* S, void* ptr) {
    if (!ptr) return;
    auto it = std::find(S->allocs.begin(), S->allocs.end(), ptr);
    if (it != S->allocs.end()) S->allocs.erase(it);
    cudaFree(ptr);
}

int64_t max_rays_per_step(const Partition& p, int s) {
    // largest sum over one row block's views of its clipped shadow rectangles,
    // times the group size
    int64_t best = 0;
    for (int i = 0; i < p.m; ++i) {
        int su0, su1, sv0, sv1;
        p.subrect(i, &su0, &su1, &sv0, &sv1);
        for (int j = 0; j < p.n; ++j) {
            int64_t rays = 0;
            for (int v : p.views_of(i)) {
                const DevVT& e = p.vt(v, j);
                int u0 = std::max(su0, e.u0), u1 = std::min(su1, e.u1);
                int v0 = std::max(sv0, e.v0), v1 = std::min(sv1, e.v1);
                if (u1 > u0 && v1 > v0) rays += (int64_t)(u1 - u0) * (v1 - v0);
            }
            best = std::max(best, rays);
        }
    }
    return best * s;
}

int groups_per_column(const Partition& p, const csgd_solver_params& prm) {
    int s = std::max(1, prm.group_size);
    double v = ceil(prm.alpha * p.m / s - 1e-9);
    return std::max(1, std::min((int)v, p.m));
}

int validate_params(const Partition& p, const csgd_solver_params* prm) {
    if (!prm) return fail(CSGD_ERR_INVALID_ARG, "params is NULL");
    if (prm->sampling < 0 || prm->sampling > 3) return fail(CSGD_ERR_INVALID_ARG, "bad sampling");
    if (prm->sync < 0 || prm->sync > 1) return fail(CSGD_ERR_INVALID_ARG, "bad sync");
    if (prm->group_size < 1 || prm->group_size > p.m)
        return fail(CSGD_ERR_INVALID_ARG, "group size must be in [1, m]");
    if (!(prm->alpha > 0) || prm->alpha > 1.0 + 1e-12)
        return fail(CSGD_ERR_INVALID_ARG, "alpha must be in (0, 1]");
    if (!(prm->gamma > 0) || prm->gamma > 1.0 + 1e-12)
        return fail(CSGD_ERR_INVALID_ARG, "gamma must be in (0, 1]");
    if (!(prm->b >= 0) || !std::isfinite(prm->b)) return fail(CSGD_ERR_INVALID_ARG, "bad b");
    if (!(prm->theta_step >= 0)) return fail(CSGD_ERR_INVALID_ARG, "bad theta_step");
    return CSGD_OK;
}

int64_t bp_partials_per_slot(const csgd_partition* P) {
    // one g^T g partial per backprojection CTA of a slot (one voxel patch each)
    int64_t n = 1;
    for (const DevTile& t : P->p.tiles_h) n = std::max<int64_t>(n, bp_blocks(t, P->p.dg.dim));
    return n;
}

int solver_reset_device(csgd_solver* S, cudaStream_t s) {
    const SolverBuffers& b = S->sb;
    CSGD_CUDA(cudaMemcpyAsync(b.r, b.y, sizeof(float) * S->n_rays, cudaMemcpyDeviceToDevice, s),
              "r = y");
    CSGD_CUDA(cudaMemsetAsync(b.x, 0, sizeof(float) * S->n_vox, s), "x = 0");
    CSGD_CUDA(cudaMemsetAsync(b.xh, 0, sizeof(float) * S->n_vox, s), "xhat = 0");
    CSGD_CUDA(cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * S->P->p.n, s), "count = 0");
    CSGD_CUDA(cudaMemsetAsync(b.z, 0, sizeof(float) * std::max<int64_t>(1, S->P->p.z_floats), s),
              "z = 0");
    if (b.d) CSGD_CUDA(cudaMemsetAsync(b.d, 0, sizeof(float) * S->n_rays, s), "d = 0");
    CSGD_CUDA(cudaMemsetAsync(b.nnz, 0, sizeof(unsigned long long), s), "nnz = 0");
    CSGD_CUDA(cudaMemsetAsync(b.counters, 0, sizeof(unsigned) * b.max_slots, s), "counters");
    CSGD_CUDA(cudaMemsetAsync(b.nnz_slot, 0, sizeof(unsigned long long) * b.max_slots, s),
              "slot counters");
    CSGD_CUDA(cudaMemsetAsync(b.acc, 0, sizeof(unsigned long long) * b.max_slots * b.g_stride, s),
              "scatter accumulators");
    CSGD_CUDA(cudaMemsetAsync(b.rmax, 0, sizeof(unsigned) * b.max_slots, s), "max |r|");
    return CSGD_OK;
}

void solver_reset_host(csgd_solver* S) {
    S->rng = SplitMix64(S->prm.seed);
    S->epoch = 0;
    S->steps_done = 0;
    S->queue.clear();
    S->epoch_open = false;
}

int solver_reset_state(csgd_solver* S, cudaStream_t s) {
    int rc = solver_reset_device(S, s);
    if (rc) return rc;
    solver_reset_host(S);
    return CSGD_OK;
}

int ensure_history(csgd_solver* S, int64_t need, cudaStream_t s) {
    if (need <= S->sb.hist_cap) return CSGD_OK;
    int64_t cap = std::max<int64_t>(need, 2 * S->sb.hist_cap);
    double* nh = nullptr;
    int rc = dmalloc(S, (void**)&nh, sizeof(double) * kHistCols * cap, "cudaMalloc(history)");
    if (rc) return rc;
    if (S->sb.hist && S->sb.hist_cap > 0)
        CSGD_CUDA(cudaMemcpyAsync(nh, S->sb.hist, sizeof(double) * kHistCols * S->sb.hist_cap,
                                  cudaMemcpyDeviceToDevice, s), "history copy");
    CSGD_CUDA(cudaStreamSynchronize(s), "history sync");
    dfree(S, S->sb.hist);
    S->sb.hist = nh;
    S->sb.hist_cap = cap;
    return CSGD_OK;
}

int ensure_sched_capacity(csgd_solver* S, int64_t n_items, int64_t n_steps, cudaStream_t s) {
    if (n_items > S->items_cap || n_steps > S->steps_cap) {
        CSGD_CUDA(cudaStreamSynchronize(s), "schedule buffer sync");
    }
    if (n_items > S->items_cap) {
        dfree(S, S->d_items);
        S->d_items = nullptr;
        int64_t cap = std::max<int64_t>(n_items, 2 * S->items_cap);
        int rc = dmalloc(S, (void**)&S->d_items, sizeof(WorkItem) * cap, "cudaMalloc(items)");
        if (rc) return rc;
        S->items_cap = cap;
    }
    if (n_steps > S->steps_cap) {
        dfree(S, S->d_steps);
        S->d_steps = nullptr;
        int64_t cap = std::max<int64_t>(n_steps, 2 * S->steps_cap);
        int rc = dmalloc(S, (void**)&S->d_steps, sizeof(StepDesc) * cap, "cudaMalloc(steps)");
        if (rc) return rc;
        S->steps_cap = cap;
    }
    return CSGD_OK;
}

void fill_queue(csgd_solver* S) {
    const Partition& p = S->P->p;
    std::vector<ColumnBatch> ep = epoch_schedule(S->rng, p, S->prm, S->epoch);
    for (auto& cb : ep)
        for (size_t g = 0; g < cb.groups.size(); ++g)
            S->queue.push_back(QueuedStep{cb.j, cb.groups[g], g + 1 == cb.groups.size()});
}

struct Plan {
    std::vector<WorkItem> items;
    std::vector<StepDesc> steps;
    // sequence: batch (first, n) or epoch close (n == -1)
    struct Op {
        int first, n, j;
        int64_t max_rays;
    };
    std::vector<Op> ops;
};

double beta_of(const csgd_solver* S, int j, const std::vector<int>& group) {
    const Partition& p = S->P->p;
    double s = 0.0;
    for (int i : group) s += p.P[(size_t)i * p.n + j];
    return S->prm.b * s;
}

void plan_step(csgd_solver* S, Plan* pl, int j, const std::vector<int>& group, int slot) {
    const Partition& p = S->P->p;
    StepDesc sd;
    memset(&sd, 0, sizeof(sd));
    sd.j = j;
    sd.w0 = (int32_t)pl->items.size();
    int64_t rays = build_work_items(p, group.data(), (int)group.size(), j, slot, &pl->items);
    sd.w1 = (int32_t)pl->items.size();
    sd.n_rays = rays;
    double terms = 0.0;
    for (int32_t w = sd.w0; w < sd.w1; ++w) {
        const DevVT& e = p.vt(pl->items[w].view, j);
        const double tu = std::floor(std::min(2.0 * e.hw_u, 4096.0)) + 2.0;
        const double tv = p.g->dim == 3 ? std::floor(std::min(2.0 * e.hw_v, 4096.0)) + 2.0 : 1.0;
        terms += tu * tv;
    }
    sd.terms = (float)terms;
    sd.step = S->steps_done;
    sd.beta = beta_of(S, j, group);
    pl->steps.push_back(sd);
    S->steps_done++;
    S->last_group = (int)group.size();
}

int take_events(csgd_solver* S, int n, int* first) {
    while (S->ev_pool.size() < S->ev_used + n) {
        cudaEvent_t e;
        CSGD_CUDA(cudaEventCreate(&e), "cudaEventCreate");
        S->ev_pool.push_back(e);
    }
    *first = (int)S->ev_used;
    S->ev_used += n;
    return CSGD_OK;
}

// Device buffers for a plan: capacity, history and the upload of its items and
// step descriptors (stream-ordered).
int prepare_plan(csgd_solver* S, Plan& pl, cudaStream_t s) {
    if (pl.ops.empty()) return CSGD_OK;
    int rc = ensure_sched_capacity(S, (int64_t)pl.items.size(), (int64_t)pl.steps.size(), s);
    if (rc) return rc;
    rc = ensure_history(S, S->steps_done, s);
    if (rc) return rc;
    if (!pl.items.empty())
        CSGD_CUDA(cudaMemcpyAsync(S->d_items, pl.items.data(), sizeof(WorkItem) * pl.items.size(),
                                  cudaMemcpyHostToDevice, s), "upload items");
    if (!pl.steps.empty())
        CSGD_CUDA(cudaMemcpyAsync(S->d_steps, pl.steps.data(), sizeof(StepDesc) * pl.steps.size(),
                                  cudaMemcpyHostToDevice, s), "upload steps");
    return CSGD_OK;
}

// The kernel launches of a prepared plan (no allocation, no host sync:
// capturable into a CUDA graph).
int launch_plan(csgd_solver* S, Plan& pl, cudaStream_t s) {
    const Partition& p = S->P->p;
    for (const auto& op : pl.ops) {
        if (op.n < 0) {
            int e0 = 0;
            if (S->profiling) {
                if (take_events(S, 2, &e0)) return CSGD_ERR_CUDA;
                cudaEventRecord(S->ev_pool[e0], s);
            }
            CSGD_CUDA(launch_epoch_close(p.dg, S->sb, S->n_rays, p.max_tile_voxels,
                                         S->prm.sync == CSGD_SYNC_EPOCH, s), "epoch close");
            if (S->profiling) {
                cudaEventRecord(S->ev_pool[e0 + 1], s);
                S->recs.push_back({3, e0, e0 + 1});
            }
            continue;
        }
        BatchLaunch b;
        b.first = op.first;
        b.nslots = op.n;
        b.j = op.j;
        b.max_rays = op.max_rays;
        b.w_begin = pl.steps[op.first].w0;
        b.n_items = pl.steps[op.first + op.n - 1].w1 - b.w_begin;
        b.max_item_rays = 0;
        for (int w = b.w_begin; w < b.w_begin + b.n_items; ++w)
            b.max_item_rays = std::max<int64_t>(
                b.max_item_rays,
                (int64_t)(pl.items[w].u1 - pl.items[w].u0) * (pl.items[w].v1 - pl.items[w].v0));
        b.sync_epoch = S->prm.sync == CSGD_SYNC_EPOCH;
        b.bp_groups = S->bp_groups;
        b.fwd_lanes = S->fwd_lanes;
        cudaEvent_t evs[4];
        int e0 = 0;
        if (S->profiling) {
            if (take_events(S, 4, &e0)) return CSGD_ERR_CUDA;
            for (int k = 0; k < 4; ++k) evs[k] = S->ev_pool[e0 + k];
            S->recs.push_back({0, e0, e0 + 1});
            S->recs.push_back({1, e0 + 1, e0 + 2});
            S->recs.push_back({2, e0 + 2, e0 + 3});
        }
        CSGD_CUDA(launch_batch(p.dg, p.tiles_h[op.j], S->d_items, S->d_steps, b, S->sb,
                               S->P->sm_count, s, S->profiling ? evs : nullptr), "batch kernels");
    }
    return CSGD_OK;
}

int execute_plan(csgd_solver* S, Plan& pl, cudaStream_t s) {
    if (pl.ops.empty()) return CSGD_OK;
    int rc = prepare_plan(S, pl, s);
    if (rc) return rc;
    return launch_plan(S, pl, s);
}

// Append the next `n` scheduled steps (and the epoch closes they cross) to pl.
void plan_scheduled(csgd_solver* S, Plan* pl, int64_t n, bool close_at_end) {
    int64_t left = n;
    while (left > 0) {
        if (S->queue.empty()) {
            fill_queue(S);
            if (S->queue.empty()) break;
        }
        // one batch: consecutive steps of the same column block, up to max_slots
        int j = S->queue.front().j;
        Plan::Op op{(int)pl->steps.size(), 0, j, 0};
        while (left > 0 && !S->queue.empty() && op.n < S->max_slots) {
            QueuedStep qs = S->queue.front();
            if (qs.j != j) break;
            S->queue.pop_front();
            plan_step(S, pl, qs.j, qs.group, op.n);
            op.max_rays = std::max(op.max_rays, pl->steps.back().n_rays);
            op.n++;
            left--;
            S->epoch_open = true;
            if (qs.last_in_batch) break;
        }
        pl->ops.push_back(op);
        if (S->queue.empty() && S->epoch_open) {
            pl->ops.push_back(Plan::Op{0, -1, 0, 0});
            S->epoch++;
            S->epoch_open = false;
        }
    }
    if (close_at_end && S->epoch_open) {
        S->queue.clear();
        pl->ops.push_back(Plan::Op{0, -1, 0, 0});
        S->epoch++;
        S->epoch_open = false;
    }
}

}  // namespace

// ===========================================================================
// extern "C"
// ===========================================================================
extern "C" {

const char* csgd_last_error(void) { return g_err.c_str(); }

const char* csgd_version(void) { return "csgd-gb300 0.1 (sm_103a)"; }

int32_t csgd_geometry_create(const csgd_geometry_desc* desc, csgd_geometry** out) {
    if (!out) return fail(CSGD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    csgd_geometry* g = new (std::nothrow) csgd_geometry;
    if (!g) return fail(CSGD_ERR_OOM, "host allocation");
    std::string err;
    int rc = geometry_from_desc(desc, &g->g, &err);
    if (rc) {
        delete g;
        return fail(rc, err);
    }
    *out = g;
    return CSGD_OK;
}

int32_t csgd_geometry_destroy(csgd_geometry* geom) {
    delete geom;
    return CSGD_OK;
}

int32_t csgd_block_partition(const csgd_geometry* geom, const csgd_partition_desc* desc,
                             csgd_partition** out) {
    if (!out || !geom) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    csgd_partition* P = new (std::nothrow) csgd_partition;
    if (!P) return fail(CSGD_ERR_OOM, "host allocation");
    std::string err;
    int rc = partition_build(&geom->g, desc, &P->p, &err);
    if (rc) {
        delete P;
        return fail(rc, err);
    }
    *out = P;
    return CSGD_OK;
}

int32_t csgd_partition_destroy(csgd_partition* P) {
    if (!P) return CSGD_OK;
    if (P->on_device) {
        cudaFree(P->p.d_views);
        cudaFree(P->p.d_views64);
        cudaFree(P->p.d_vt);
        cudaFree(P->p.d_tiles);
    }
    delete P;
    return CSGD_OK;
}

int32_t csgd_partition_get_info(const csgd_partition* P, csgd_partition_info* info) {
    if (!P || !info) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    info->m = P->p.m;
    info->n = P->p.n;
    info->n_rays = P->p.g->n_rays();
    info->n_voxels = P->p.g->n_voxels();
    info->z_floats = P->p.z_floats;
    return CSGD_OK;
}

int32_t csgd_partition_probabilities(const csgd_partition* P, double* out) {
    if (!P || !out) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    memcpy(out, P->p.P.data(), sizeof(double) * P->p.P.size());
    return CSGD_OK;
}

int32_t csgd_project_block(const csgd_partition* Pc, const int32_t* row_blocks, int32_t n_rb,
                           int32_t j, const float* x, float* out, int32_t accumulate,
                           csgd_stream stream) {
    csgd_partition* P = const_cast<csgd_partition*>(Pc);
    if (!P || !x || !out) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    if (j < 0 || j >= P->p.n) return fail(CSGD_ERR_INVALID_ARG, "column block out of range");
    int rc = check_rows(P->p, row_blocks, n_rb);
    if (rc) return rc;
    rc = ensure_device(P);
    if (rc) return rc;
    std::vector<WorkItem> items;
    items_for_rows(P->p, row_blocks, n_rb, j, true, &items);
    return run_inline(P, items, j, true, x, out, accumulate, (cudaStream_t)stream);
}

int32_t csgd_backproject_block(const csgd_partition* Pc, const int32_t* row_blocks,
                               int32_t n_rb, int32_t j, const float* r, float* g,
                               int32_t accumulate, csgd_stream stream) {
    csgd_partition* P = const_cast<csgd_partition*>(Pc);
    if (!P || !r || !g) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    if (j < 0 || j >= P->p.n) return fail(CSGD_ERR_INVALID_ARG, "column block out of range");
    int rc = check_rows(P->p, row_blocks, n_rb);
    if (rc) return rc;
    rc = ensure_device(P);
    if (rc) return rc;
    std::vector<WorkItem> items;
    items_for_rows(P->p, row_blocks, n_rb, j, false, &items);
    return run_inline(P, items, j, false, r, g, accumulate, (cudaStream_t)stream);
}

int32_t csgd_backproject_block_noalloc(const csgd_partition* Pc, const int32_t* row_blocks,
                                       int32_t n_rb, int32_t j, const float* r, float* g,
                                       int32_t accumulate, csgd_stream stream) {
    // Same result as csgd_backproject_block, with the ray table in the fixed
    // array of ops.cu and every other piece of state on the stack: no host or
    // device allocation on success.
    csgd_partition* P = const_cast<csgd_partition*>(Pc);
    if (!P || !r || !g || !row_blocks) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    const Partition& p = P->p;
    if (j < 0 || j >= p.n) return fail(CSGD_ERR_INVALID_ARG, "column block out of range");
    if (n_rb < 1 || n_rb > p.m) return fail(CSGD_ERR_INVALID_ARG, "bad number of row blocks");
    unsigned char seen[65536 / 8];
    memset(seen, 0, sizeof(seen));
    for (int k = 0; k < n_rb; ++k) {
        int i = row_blocks[k];
        if (i < 0 || i >= p.m) return fail(CSGD_ERR_INVALID_ARG, "row block out of range");
        if (seen[i >> 3] & (1u << (i & 7))) return fail(CSGD_ERR_INVALID_ARG, "row blocks must be distinct");
        seen[i >> 3] |= (unsigned char)(1u << (i & 7));
    }
    if (!P->on_device)
        return fail(CSGD_ERR_STATE,
                    "partition tables are not on the device yet: make one ordinary device call "
                    "with this partition (e.g. csgd_project_block) before the allocation-free one");
    int dev = 0;
    CSGD_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p.device) return fail(CSGD_ERR_INVALID_ARG, "partition tables live on another device");
    // count the rays first: reject the call before launching anything
    int64_t total = 0;
    for (int r2 = 0; r2 < n_rb; ++r2) {
        int su0, su1, sv0, sv1;
        p.subrect(row_blocks[r2], &su0, &su1, &sv0, &sv1);
        for (int v : p.views_of(row_blocks[r2])) {
            const DevVT& e = p.vt(v, j);
            int u0 = std::max(su0, e.u0), u1 = std::min(su1, e.u1);
            int v0 = std::max(sv0, e.v0), v1 = std::min(sv1, e.v1);
            if (u1 > u0 && v1 > v0) total += (int64_t)(u1 - u0) * (v1 - v0);
        }
    }
    if (total > CSGD_NOALLOC_MAX_RAYS)
        return fail(CSGD_ERR_INVALID_ARG,
                    "the call covers " + std::to_string(total) + " rays, more than "
                    "CSGD_NOALLOC_MAX_RAYS = " + std::to_string(CSGD_NOALLOC_MAX_RAYS));
    RayRec* table = nullptr;
    CSGD_CUDA(noalloc_table_address(dev, &table), "cudaGetSymbolAddress(ray table)");
    cudaStream_t s = (cudaStream_t)stream;
    // Fill launches of at most kMaxInlineItems views on the stack, in the same
    // order as csgd_backproject_block; later launches accumulate.
    InlineItems it;
    int cnt = 0;
    int64_t rays = 0;
    bool first = true;
    auto flush = [&]() -> int {
        it.step.j = j;
        it.step.w0 = 0;
        it.step.w1 = cnt;
        it.step.n_rays = rays;
        it.step.step = 0;
        it.step.beta = 0.0;
        it.step.terms = 0.f;
        it.n = cnt;
        cudaError_t e = launch_backproject_inline(p.dg, p.tiles_h[j], it, r, g,
                                                  first ? accumulate : 1, table, P->sm_count, s);
        if (e != cudaSuccess) return cuda_fail(e, "backproject kernel");
        first = false;
        cnt = 0;
        rays = 0;
        return CSGD_OK;
    };
    for (int r2 = 0; r2 < n_rb; ++r2) {
        int su0, su1, sv0, sv1;
        p.subrect(row_blocks[r2], &su0, &su1, &sv0, &sv1);
        for (int v : p.views_of(row_blocks[r2])) {
            const DevVT& e = p.vt(v, j);
            int u0 = std::max(su0, e.u0), u1 = std::min(su1, e.u1);
            int v0 = std::max(sv0, e.v0), v1 = std::min(sv1, e.v1);
            if (u1 <= u0 || v1 <= v0) continue;
            WorkItem& w = it.items[cnt++];
            w.view = v;
            w.slot = 0;
            w.u0 = u0; w.u1 = u1; w.v0 = v0; w.v1 = v1;
            w.ray_off = rays;
            rays += (int64_t)(u1 - u0) * (v1 - v0);
            if (cnt == kMaxInlineItems) {
                int rc = flush();
                if (rc) return rc;
            }
        }
    }
    if (cnt > 0 || first) {
        int rc = flush();
        if (rc) return rc;
    }
    return CSGD_OK;
}

int32_t csgd_project_full(const csgd_partition* Pc, const float* x, float* out,
                          csgd_stream stream) {
    csgd_partition* P = const_cast<csgd_partition*>(Pc);
    if (!P || !x || !out) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    int rc = ensure_device(P);
    if (rc) return rc;
    const Partition& p = P->p;
    cudaStream_t s = (cudaStream_t)stream;
    CSGD_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * p.g->n_rays(), s), "memset");
    for (int j = 0; j < p.n; ++j) {
        std::vector<WorkItem> items;
        for (int v = 0; v < p.g->n_views; ++v) {
            const DevVT& e = p.vt(v, j);
            if (e.u1 <= e.u0 || e.v1 <= e.v0) continue;
            WorkItem w;
            w.view = v; w.slot = 0;
            w.u0 = e.u0; w.u1 = e.u1; w.v0 = e.v0; w.v1 = e.v1;
            w.ray_off = 0;
            items.push_back(w);
        }
        if (items.empty()) continue;
        rc = run_inline(P, items, j, true, x, out, 1, s);
        if (rc) return rc;
    }
    return CSGD_OK;
}

int32_t csgd_schedule_generate(const csgd_partition* P, const csgd_solver_params* params,
                               int32_t n_epochs, int32_t* out, int64_t capacity, int64_t* len) {
    if (!P || !len) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    int rc = validate_params(P->p, params);
    if (rc) return rc;
    SplitMix64 rng(params->seed);
    std::vector<int32_t> flat;
    for (int e = 0; e < n_epochs; ++e) {
        std::vector<ColumnBatch> ep = epoch_schedule(rng, P->p, *params, e);
        flat.push_back((int32_t)ep.size());
        for (auto& cb : ep) {
            flat.push_back(cb.j);
            flat.push_back((int32_t)cb.groups.size());
            for (auto& g : cb.groups) {
                flat.push_back((int32_t)g.size());
                for (int i : g) flat.push_back(i);
            }
        }
    }
    *len = (int64_t)flat.size();
    if (!out || capacity < (int64_t)flat.size())
        return fail(CSGD_ERR_INVALID_ARG, "schedule buffer too small");
    memcpy(out, flat.data(), sizeof(int32_t) * flat.size());
    return CSGD_OK;
}

static int64_t footprint(const csgd_partition* P, const csgd_solver_params* prm, int* max_slots,
                         int64_t* max_rays, int64_t* fwd_blocks, int64_t* n_gg) {
    const Partition& p = P->p;
    int64_t ny = p.g->n_rays(), nx = p.g->n_voxels();
    *max_slots = groups_per_column(p, *prm);
    *max_rays = max_rays_per_step(p, std::max(1, prm->group_size));
    *fwd_blocks = std::max<int64_t>(1, (*max_rays * 4 + kFwdThreads - 1) / kFwdThreads);
    *n_gg = bp_partials_per_slot(P);
    int64_t b = 0;
    b += 4 * (2 * nx);                           // x, xhat
    b += 4 * (int64_t)p.n;                       // counts
    b += 4 * (4 * ny);                           // y, r, p, q
    if (prm->sync == CSGD_SYNC_EPOCH) b += 4 * ny;  // pending residual change
    b += 4 * std::max<int64_t>(1, p.z_floats);   // z store
    b += 16 * (int64_t)(*max_slots) * p.max_tile_voxels;  // (x, g) pairs and scatter sums per slot
    b += (int64_t)sizeof(RayRec) * (*max_slots) * (*max_rays);  // ray tables
    b += 4 * (int64_t)(*max_slots) * (*n_gg + *fwd_blocks) + 24 * (int64_t)(*max_slots);  // partials, mu, counters, nnz, max |r|
    return b;
}

int32_t csgd_solver_footprint_bytes(const csgd_partition* P, const csgd_solver_params* params,
                                    int64_t* bytes) {
    if (!P || !bytes) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    int rc = validate_params(P->p, params);
    if (rc) return rc;
    int ms;
    int64_t mr, fb, ng;
    *bytes = footprint(P, params, &ms, &mr, &fb, &ng);
    return CSGD_OK;
}

int32_t csgd_solver_create(const csgd_partition* Pc, const csgd_solver_params* params,
                           const float* y, csgd_stream stream, csgd_solver** out) {
    csgd_partition* P = const_cast<csgd_partition*>(Pc);
    if (!P || !y || !out) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    int rc = validate_params(P->p, params);
    if (rc) return rc;
    rc = ensure_device(P);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    csgd_solver* S = new (std::nothrow) csgd_solver;
    if (!S) return fail(CSGD_ERR_OOM, "host allocation");
    S->P = P;
    S->prm = *params;
    S->n_rays = P->p.g->n_rays();
    S->n_vox = P->p.g->n_voxels();
    int64_t mr, fb, ng;
    footprint(P, params, &S->max_slots, &mr, &fb, &ng);
    S->max_rays_per_step = mr;
    SolverBuffers& b = S->sb;
    memset(&b, 0, sizeof(b));
    b.max_slots = S->max_slots;
    b.max_fwd_blocks = (int)fb;
    b.g_stride = P->p.max_tile_voxels;
    b.gg_stride = (int)ng;
    b.table_stride = std::max<int64_t>(1, mr);
    const Partition& p = P->p;
#define ALLOC(ptr, bytes, what)                                    \
    do {                                                           \
        rc = dmalloc(S, (void**)&(ptr), (bytes), what);            \
        if (rc) {                                                  \
            std::string m = g_err;                                 \
            csgd_solver_destroy(S);                                \
            return fail(rc, m);                                    \
        }                                                          \
    } while (0)
    ALLOC(b.x, sizeof(float) * S->n_vox, "cudaMalloc(x)");
    ALLOC(b.xh, sizeof(float) * S->n_vox, "cudaMalloc(xhat)");
    ALLOC(b.cnt, sizeof(int32_t) * p.n, "cudaMalloc(count)");
    float* yy = nullptr;
    ALLOC(yy, sizeof(float) * S->n_rays, "cudaMalloc(y)");
    b.y = yy;
    ALLOC(b.r, sizeof(float) * S->n_rays, "cudaMalloc(r)");
    ALLOC(b.z, sizeof(float) * std::max<int64_t>(1, p.z_floats), "cudaMalloc(z store)");
    if (params->sync == CSGD_SYNC_EPOCH) ALLOC(b.d, sizeof(float) * S->n_rays, "cudaMalloc(d)");
    ALLOC(b.p, sizeof(float) * S->n_rays, "cudaMalloc(p)");
    ALLOC(b.q, sizeof(float) * S->n_rays, "cudaMalloc(q)");
    ALLOC(b.g, 2 * sizeof(float) * b.max_slots * b.g_stride, "cudaMalloc(x, g pairs)");
    ALLOC(b.gg_part, sizeof(float) * b.max_slots * ng, "cudaMalloc(gg partials)");
    ALLOC(b.acc, sizeof(unsigned long long) * b.max_slots * b.g_stride,
          "cudaMalloc(scatter accumulators)");
    ALLOC(b.rmax, sizeof(unsigned) * b.max_slots, "cudaMalloc(max |r| per slot)");
    ALLOC(b.table, sizeof(RayRec) * b.max_slots * b.table_stride, "cudaMalloc(ray tables)");
    b.qq_stride = b.max_fwd_blocks;  // one q^T q partial per forward CTA
    ALLOC(b.qq_part, sizeof(float) * b.max_slots * b.qq_stride, "cudaMalloc(qq partials)");
    ALLOC(b.counters, sizeof(unsigned) * b.max_slots, "cudaMalloc(counters)");
    ALLOC(b.mu, sizeof(double) * b.max_slots, "cudaMalloc(mu)");
    ALLOC(b.nnz, sizeof(unsigned long long), "cudaMalloc(nnz)");
    ALLOC(b.nnz_slot, sizeof(unsigned long long) * b.max_slots, "cudaMalloc(nnz per slot)");
    ALLOC(S->d_sq, sizeof(double) * 256, "cudaMalloc(norm partials)");
#undef ALLOC
    cudaError_t e = cudaMemcpyAsync(yy, y, sizeof(float) * S->n_rays, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        csgd_solver_destroy(S);
        return cuda_fail(e, "copy y");
    }
    rc = solver_reset_state(S, s);
    if (rc == CSGD_OK) rc = ensure_history(S, 1024, s);
    if (rc == CSGD_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "solver init");
    }
    if (rc) {
        std::string m = g_err;
        csgd_solver_destroy(S);
        return fail(rc, m);
    }
    *out = S;
    return CSGD_OK;
}

int32_t csgd_solver_destroy(csgd_solver* S) {
    if (!S) return CSGD_OK;
    for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
    for (void* p : S->allocs) cudaFree(p);
    delete S;
    return CSGD_OK;
}

int32_t csgd_solver_reset(csgd_solver* S, const float* y, int32_t y_on_host, csgd_stream stream) {
    if (!S || !y) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CSGD_CUDA(cudaMemcpyAsync((void*)S->sb.y, y, sizeof(float) * S->n_rays,
                              y_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s),
              "copy y");
    return solver_reset_state(S, s);
}

int32_t csgd_solve_step(csgd_solver* S, const csgd_block_choice* choice, csgd_step_info* info,
                        csgd_stream stream) {
    if (!S) return fail(CSGD_ERR_INVALID_ARG, "NULL solver");
    cudaStream_t s = (cudaStream_t)stream;
    Plan pl;
    int64_t step_index = S->steps_done;
    int j = -1, nrows = 0;
    if (choice) {
        const Partition& p = S->P->p;
        if (choice->j < 0 || choice->j >= p.n)
            return fail(CSGD_ERR_INVALID_ARG, "column block out of range");
        int rc = check_rows(p, choice->row_blocks, choice->n_rows);
        if (rc) return rc;
        std::vector<int> grp(choice->row_blocks, choice->row_blocks + choice->n_rows);
        int64_t rays = 0;
        for (int i : grp) {
            std::vector<WorkItem> tmp;
            rays += build_work_items(p, &i, 1, choice->j, 0, &tmp);
        }
        if (rays > S->max_rays_per_step)
            return fail(CSGD_ERR_INVALID_ARG, "group larger than the solver was sized for");
        Plan::Op op{0, 1, choice->j, 0};
        plan_step(S, &pl, choice->j, grp, 0);
        op.max_rays = pl.steps.back().n_rays;
        pl.ops.push_back(op);
        S->epoch_open = true;
        j = choice->j;
        nrows = choice->n_rows;
    } else {
        plan_scheduled(S, &pl, 1, false);
        if (pl.steps.empty()) return fail(CSGD_ERR_STATE, "schedule has no steps");
        j = pl.steps[0].j;
    }
    int rc = execute_plan(S, pl, s);
    if (rc) return rc;
    if (info) {
        double h[kHistCols] = {0, 0, 0, 0, 0};
        CSGD_CUDA(cudaMemcpyAsync(h, S->sb.hist + kHistCols * step_index, sizeof(h),
                                  cudaMemcpyDeviceToHost, s), "read step");
        CSGD_CUDA(cudaStreamSynchronize(s), "step sync");
        info->step = step_index;
        info->j = j;
        info->n_rows = choice ? nrows : S->last_group;
        info->beta = h[0];
        info->gg = h[1];
        info->qq = h[2];
        info->mu = h[3];
    }
    return CSGD_OK;
}

int32_t csgd_solve(csgd_solver* S, int64_t n_steps, float* x_out, int32_t x_on_host,
                   csgd_report* report, int32_t compute_residual, csgd_stream stream) {
    if (!S || n_steps < 0) return fail(CSGD_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Partition& p = S->P->p;
    unsigned long long nnz0 = 0;
    if (report) {
        CSGD_CUDA(cudaMemcpyAsync(&nnz0, S->sb.nnz, sizeof(nnz0), cudaMemcpyDeviceToHost, s),
                  "read nnz");
        CSGD_CUDA(cudaStreamSynchronize(s), "sync");
    }
    int64_t steps0 = S->steps_done;
    Plan pl;
    plan_scheduled(S, &pl, n_steps, true);
    int rc = execute_plan(S, pl, s);
    if (rc) return rc;
    int64_t rays = 0, tile_voxels = 0;
    for (const StepDesc& sd : pl.steps) {
        const DevTile& t = p.tiles_h[sd.j];
        rays += sd.n_rays;
        tile_voxels += (int64_t)t.n[0] * t.n[1] * t.n[2];
    }
    if (x_out) {
        if (x_on_host) {
            if (!S->d_xrow) {
                rc = dmalloc(S, (void**)&S->d_xrow, sizeof(float) * S->n_vox, "cudaMalloc(x row)");
                if (rc) return rc;
            }
            CSGD_CUDA(launch_tile_to_rowmajor(p.dg, S->sb.x, S->d_xrow, p.max_tile_voxels, s),
                      "x layout");
            CSGD_CUDA(cudaMemcpyAsync(x_out, S->d_xrow, sizeof(float) * S->n_vox,
                                      cudaMemcpyDeviceToHost, s), "x to host");
        } else {
            CSGD_CUDA(launch_tile_to_rowmajor(p.dg, S->sb.x, x_out, p.max_tile_voxels, s),
                      "x layout");
        }
    }
    if (report) {
        memset(report, 0, sizeof(*report));
        if (compute_residual) {
            if (!S->d_xrow) {
                rc = dmalloc(S, (void**)&S->d_xrow, sizeof(float) * S->n_vox, "cudaMalloc(x row)");
                if (rc) return rc;
            }
            if (!S->d_ax) {
                rc = dmalloc(S, (void**)&S->d_ax, sizeof(float) * S->n_rays, "cudaMalloc(Ax)");
                if (rc) return rc;
            }
            CSGD_CUDA(launch_tile_to_rowmajor(p.dg, S->sb.x, S->d_xrow, p.max_tile_voxels, s),
                      "x layout");
            rc = csgd_project_full(S->P, S->d_xrow, S->d_ax, s);
            if (rc) return rc;
            CSGD_CUDA(launch_sq_residual(S->sb.y, S->d_ax, S->n_rays, S->d_sq, s), "norm");
            double part[256];
            CSGD_CUDA(cudaMemcpyAsync(part, S->d_sq, sizeof(part), cudaMemcpyDeviceToHost, s),
                      "read norm");
            CSGD_CUDA(cudaStreamSynchronize(s), "sync");
            double ss = 0.0;
            for (int k = 0; k < 256; ++k) ss += part[k];
            report->residual_norm = sqrt(ss);
        }
        unsigned long long nnz1 = 0;
        CSGD_CUDA(cudaMemcpyAsync(&nnz1, S->sb.nnz, sizeof(nnz1), cudaMemcpyDeviceToHost, s),
                  "read nnz");
        CSGD_CUDA(cudaStreamSynchronize(s), "sync");
        report->steps = S->steps_done - steps0;
        report->epochs = S->epoch;
        report->nnz = (int64_t)(nnz1 - nnz0);
        report->updates = 3.0 * (double)(nnz1 - nnz0);
        report->rays = rays;
        report->tile_voxels = tile_voxels;
    }
    return CSGD_OK;
}

int32_t csgd_solver_history(csgd_solver* S, csgd_step_info* out, int64_t capacity,
                            int64_t* count) {
    if (!S || !count) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    int64_t n = std::min<int64_t>(S->steps_done, S->sb.hist_cap);
    int64_t take = std::min<int64_t>(n, capacity);
    *count = take;
    if (take <= 0) return CSGD_OK;
    std::vector<double> h(kHistCols * take);
    int64_t start = n - take;
    CSGD_CUDA(cudaMemcpy(h.data(), S->sb.hist + kHistCols * start, sizeof(double) * kHistCols * take,
                         cudaMemcpyDeviceToHost), "read history");
    for (int64_t k = 0; k < take; ++k) {
        const double* row = &h[kHistCols * k];
        out[k].step = start + k;
        out[k].j = -1;
        out[k].n_rows = -1;
        out[k].beta = row[0];
        out[k].gg = row[1];
        out[k].qq = row[2];
        out[k].mu = row[3];
        out[k].nnz = (int64_t)row[4];
    }
    return CSGD_OK;
}

struct csgd_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int32_t csgd_solver_graph_create(csgd_solver* S, int64_t n_steps, float* x_out, int32_t x_on_host,
                                 csgd_graph** out) {
    if (!S || !out || n_steps < 0) return fail(CSGD_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    if (S->profiling) return fail(CSGD_ERR_STATE, "disable profiling before building a graph");
    const Partition& p = S->P->p;
    if (x_out && x_on_host) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, x_out) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return fail(CSGD_ERR_INVALID_ARG, "a graph can copy x only to pinned host memory");
        }
    }
    cudaStream_t cs = nullptr;
    CSGD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    // plan the whole run from a fresh schedule and upload it before capturing
    solver_reset_host(S);
    Plan pl;
    plan_scheduled(S, &pl, n_steps, true);
    int rc = prepare_plan(S, pl, cs);
    if (rc == CSGD_OK && x_out && x_on_host && !S->d_xrow)
        rc = dmalloc(S, (void**)&S->d_xrow, sizeof(float) * S->n_vox, "cudaMalloc(x row)");
    if (rc == CSGD_OK) {
        cudaError_t e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "upload sync");
    }
    cudaGraph_t graph = nullptr;
    if (rc == CSGD_OK) {
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "begin capture");
    }
    if (rc == CSGD_OK) {
        rc = solver_reset_device(S, cs);
        if (rc == CSGD_OK) rc = launch_plan(S, pl, cs);
        if (rc == CSGD_OK && x_out) {
            float* dst = x_on_host ? S->d_xrow : x_out;
            cudaError_t e = launch_tile_to_rowmajor(p.dg, S->sb.x, dst, p.max_tile_voxels, cs);
            if (e == cudaSuccess && x_on_host)
                e = cudaMemcpyAsync(x_out, S->d_xrow, sizeof(float) * S->n_vox,
                                    cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) rc = cuda_fail(e, "x output");
        }
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (rc == CSGD_OK && e != cudaSuccess) rc = cuda_fail(e, "end capture");
    }
    cudaStreamDestroy(cs);
    // the graph starts from the seed each time it runs; so does the host side
    solver_reset_host(S);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    csgd_graph* G = new (std::nothrow) csgd_graph;
    if (!G) {
        cudaGraphDestroy(graph);
        return fail(CSGD_ERR_OOM, "host allocation");
    }
    G->graph = graph;
    cudaError_t e = cudaGraphInstantiate(&G->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete G;
        return cuda_fail(e, "graph instantiate");
    }
    *out = G;
    return CSGD_OK;
}

int32_t csgd_graph_batch_create(csgd_graph* const* parts, int32_t n, csgd_graph** out) {
    if (!parts || n < 1 || !out) return fail(CSGD_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    cudaGraph_t g = nullptr;
    CSGD_CUDA(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    for (int k = 0; k < n; ++k) {
        if (!parts[k] || !parts[k]->graph) {
            cudaGraphDestroy(g);
            return fail(CSGD_ERR_INVALID_ARG, "NULL part");
        }
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, parts[k]->graph);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            return cuda_fail(e, "add child graph");
        }
    }
    csgd_graph* G = new (std::nothrow) csgd_graph;
    if (!G) {
        cudaGraphDestroy(g);
        return fail(CSGD_ERR_OOM, "host allocation");
    }
    G->graph = g;
    cudaError_t e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        delete G;
        return cuda_fail(e, "graph instantiate");
    }
    *out = G;
    return CSGD_OK;
}

struct csgd_batch {
    ExecPlan* plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    int device = 0;
};

int32_t csgd_batch_destroy(csgd_batch* B) {
    if (!B) return CSGD_OK;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->done) cudaEventDestroy(B->done);
    exec_plan_free(B->plan);
    delete B;
    return CSGD_OK;
}

int32_t csgd_batch_create(csgd_solver* const* solvers, const int64_t* n_steps, float* const* x_out,
                          int32_t n, const csgd_batch_params* params, csgd_batch** out) {
    if (!solvers || !n_steps || n < 1 || !out) return fail(CSGD_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    int dev = 0;
    CSGD_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    int dim = 0;
    for (int k = 0; k < n; ++k) {
        csgd_solver* S = solvers[k];
        if (!S || n_steps[k] < 0) return fail(CSGD_ERR_INVALID_ARG, "NULL solver or negative steps");
        if (S->profiling) return fail(CSGD_ERR_STATE, "disable profiling before building a batch");
        if (S->P->p.device != dev) return fail(CSGD_ERR_INVALID_ARG, "solvers on another device");
        if (dim && S->P->p.dg.dim != dim) return fail(CSGD_ERR_INVALID_ARG, "mixed 2D and 3D solvers");
        dim = S->P->p.dg.dim;
        for (int m = 0; m < k; ++m)
            if (solvers[m] == S) return fail(CSGD_ERR_INVALID_ARG, "a solver appears twice");
    }
    csgd_batch* B = new (std::nothrow) csgd_batch;
    if (!B) return fail(CSGD_ERR_OOM, "host allocation");
    B->device = dev;
    B->plan = exec_plan_new(n);
    if (!B->plan) {
        delete B;
        return fail(CSGD_ERR_OOM, "host allocation");
    }
    cudaStream_t cs = nullptr;
    int rc = CSGD_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate");
    // plan every solve from a fresh schedule, upload it, and turn its kernels
    // into executor tasks
    for (int k = 0; rc == CSGD_OK && k < n; ++k) {
        csgd_solver* S = solvers[k];
        const Partition& p = S->P->p;
        solver_reset_host(S);
        Plan pl;
        plan_scheduled(S, &pl, n_steps[k], true);
        rc = prepare_plan(S, pl, cs);
        for (const auto& op : pl.ops) {
            if (rc) break;
            if (op.n < 0) {
                exec_plan_add_close(B->plan, k, p.dg, S->sb, S->n_rays, p.max_tile_voxels,
                                    S->prm.sync == CSGD_SYNC_EPOCH);
                continue;
            }
            BatchLaunch b;
            b.first = op.first;
            b.nslots = op.n;
            b.j = op.j;
            b.max_rays = op.max_rays;
            b.w_begin = pl.steps[op.first].w0;
            b.n_items = pl.steps[op.first + op.n - 1].w1 - b.w_begin;
            b.max_item_rays = 0;
            for (int w = b.w_begin; w < b.w_begin + b.n_items; ++w)
                b.max_item_rays = std::max<int64_t>(
                    b.max_item_rays,
                    (int64_t)(pl.items[w].u1 - pl.items[w].u0) * (pl.items[w].v1 - pl.items[w].v0));
            b.sync_epoch = S->prm.sync == CSGD_SYNC_EPOCH;
            b.bp_groups = S->bp_groups;
            b.fwd_lanes = S->fwd_lanes;
            e = exec_plan_add_batch(B->plan, k, p.dg, p.tiles_h[op.j], S->d_items, S->d_steps, b, S->sb,
                                    S->P->sm_count);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch task");
        }
        if (rc == CSGD_OK && x_out && x_out[k])
            exec_plan_add_xout(B->plan, k, p.dg, S->sb.x, x_out[k], p.max_tile_voxels);
        solver_reset_host(S);  // every launch starts from the seed; so does the host side
    }
    if (rc == CSGD_OK) {
        const int64_t wait = params && params->wait_limit_ns > 0 ? params->wait_limit_ns
                                                                  : (int64_t)2000000000;
        e = exec_plan_finalize(B->plan, wait, params ? params->stall_last_task : 0,
                               solvers[0]->P->sm_count);
        if (e != cudaSuccess) rc = cuda_fail(e, "batch plan upload");
    }
    if (rc == CSGD_OK) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "upload sync");
    }
    // the graph: every solver's reset, then the persistent launch
    if (rc == CSGD_OK) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "begin capture");
        for (int k = 0; rc == CSGD_OK && k < n; ++k) rc = solver_reset_device(solvers[k], cs);
        if (rc == CSGD_OK) {
            e = exec_plan_launch(B->plan, cs);
            if (e != cudaSuccess) rc = cuda_fail(e, "executor launch");
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (rc == CSGD_OK && e != cudaSuccess) rc = cuda_fail(e, "end capture");
        B->graph = g;
    }
    if (cs) cudaStreamDestroy(cs);
    if (rc == CSGD_OK) {
        e = cudaGraphInstantiate(&B->exec, B->graph, 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming);
        if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
    }
    if (rc) {
        std::string m = g_err;
        csgd_batch_destroy(B);
        return fail(rc, m);
    }
    *out = B;
    return CSGD_OK;
}

int32_t csgd_batch_launch(csgd_batch* B, csgd_stream stream) {
    if (!B) return fail(CSGD_ERR_INVALID_ARG, "NULL batch");
    CSGD_CUDA(cudaGraphLaunch(B->exec, (cudaStream_t)stream), "batch launch");
    CSGD_CUDA(cudaEventRecord(B->done, (cudaStream_t)stream), "batch event");
    return CSGD_OK;
}

int32_t csgd_batch_status(csgd_batch* B) {
    if (!B) return fail(CSGD_ERR_INVALID_ARG, "NULL batch");
    CSGD_CUDA(cudaEventSynchronize(B->done), "batch sync");
    int st = 0;
    CSGD_CUDA(exec_plan_status(B->plan, &st), "batch status");
    if (st) return fail(CSGD_ERR_TIMEOUT, "a wait of the batch executor ran out of time");
    return CSGD_OK;
}

int32_t csgd_batch_info(csgd_batch* B, int32_t* n_tasks, int64_t* n_units, int32_t* grid) {
    if (!B || !n_tasks || !n_units || !grid) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    int nt = 0, gr = 0;
    int64_t nu = 0;
    exec_plan_info(B->plan, &nt, &nu, &gr);
    *n_tasks = nt;
    *n_units = nu;
    *grid = gr;
    return CSGD_OK;
}

int32_t csgd_graph_launch(csgd_graph* G, csgd_stream stream) {
    if (!G || !G->exec) return fail(CSGD_ERR_INVALID_ARG, "NULL graph");
    CSGD_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream), "cudaGraphLaunch");
    return CSGD_OK;
}

int32_t csgd_graph_destroy(csgd_graph* G) {
    if (!G) return CSGD_OK;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
    return CSGD_OK;
}

int32_t csgd_solver_profile(csgd_solver* S, int32_t enable) {
    if (!S) return fail(CSGD_ERR_INVALID_ARG, "NULL solver");
    S->profiling = enable != 0;
    return CSGD_OK;
}

int32_t csgd_solver_profile_read(csgd_solver* S, csgd_kernel_times* out, int32_t reset) {
    if (!S || !out) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof(*out));
    if (!S->recs.empty()) {
        CSGD_CUDA(cudaEventSynchronize(S->ev_pool[S->recs.back().e1]), "event sync");
    }
    for (const auto& r : S->recs) {
        float ms = 0.f;
        CSGD_CUDA(cudaEventElapsedTime(&ms, S->ev_pool[r.e0], S->ev_pool[r.e1]), "elapsed");
        out->launches[r.kind] += 1;
        out->ms[r.kind] += ms;
    }
    if (reset) {
        S->recs.clear();
        S->ev_used = 0;
    }
    return CSGD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// checkpoint and resume
// ---------------------------------------------------------------------------
namespace {

constexpr char kStateMagic[8] = {'C', 'S', 'G', 'D', 'S', 'T', 'A', 'T'};
constexpr int32_t kStateVersion = 1;

struct StateHeader {
    char magic[8];
    int32_t version;
    int32_t has_d;            // the pending refresh d of epoch sync follows r
    int64_t n_rays, n_vox, n_tiles, z_floats;
    int64_t hist_rows;        // history rows stored
    int64_t queue_len;        // queued steps of the current epoch
    int64_t queue_ints;       // int32 values of the queue section
    csgd_solver_params prm;   // must equal the restoring solver's
    uint64_t rng_state;
    int64_t epoch, steps_done;
    int32_t epoch_open, last_group;
    uint64_t nnz;             // non-zeros counted since the last reset
};

int64_t align8(int64_t n) { return (n + 7) & ~(int64_t)7; }

// Section sizes of a solver's state, in the order they are written.
struct StateLayout {
    int64_t queue_ints = 0, hist_rows = 0;
    int64_t off_queue = 0, off_y = 0, off_x = 0, off_xh = 0, off_r = 0, off_z = 0, off_d = 0,
            off_cnt = 0, off_hist = 0, total = 0;
};

StateLayout state_layout(const csgd_solver* S, int64_t queue_ints, int64_t hist_rows, bool has_d) {
    const Partition& p = S->P->p;
    StateLayout L;
    L.queue_ints = queue_ints;
    L.hist_rows = hist_rows;
    int64_t o = align8(sizeof(StateHeader));
    L.off_queue = o;
    o = align8(o + 4 * queue_ints);
    L.off_y = o;
    o = align8(o + 4 * S->n_rays);
    L.off_x = o;
    o = align8(o + 4 * S->n_vox);
    L.off_xh = o;
    o = align8(o + 4 * S->n_vox);
    L.off_r = o;
    o = align8(o + 4 * S->n_rays);
    L.off_z = o;
    o = align8(o + 4 * std::max<int64_t>(0, p.z_floats));
    L.off_d = o;
    o = align8(o + (has_d ? 4 * S->n_rays : 0));
    L.off_cnt = o;
    o = align8(o + 4 * (int64_t)p.n);
    L.off_hist = o;
    o = align8(o + 8 * kHistCols * hist_rows);
    L.total = o;
    return L;
}

int64_t queue_int_count(const csgd_solver* S) {
    int64_t n = 0;
    for (const QueuedStep& q : S->queue) n += 3 + (int64_t)q.group.size();
    return n;
}

bool same_params(const csgd_solver_params& a, const csgd_solver_params& b) {
    return a.sampling == b.sampling && a.sync == b.sync && a.group_size == b.group_size &&
           a.alpha == b.alpha && a.gamma == b.gamma && a.b == b.b &&
           a.theta_step == b.theta_step && a.seed == b.seed;
}

}  // namespace

int32_t csgd_solver_state_bytes(const csgd_solver* S, int64_t* bytes) {
    if (!S || !bytes) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    const int64_t rows = std::min<int64_t>(S->steps_done, S->sb.hist_cap);
    *bytes = state_layout(S, queue_int_count(S), rows, S->prm.sync == CSGD_SYNC_EPOCH).total;
    return CSGD_OK;
}

int32_t csgd_solver_get_state(csgd_solver* S, void* buf, int64_t capacity, csgd_stream stream) {
    if (!S || !buf) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Partition& p = S->P->p;
    const bool has_d = S->prm.sync == CSGD_SYNC_EPOCH;
    const int64_t rows = std::min<int64_t>(S->steps_done, S->sb.hist_cap);
    const StateLayout L = state_layout(S, queue_int_count(S), rows, has_d);
    if (capacity < L.total) return fail(CSGD_ERR_INVALID_ARG, "state buffer too small");
    char* out = (char*)buf;
    std::memset(out, 0, (size_t)L.total);
    StateHeader h{};
    std::memcpy(h.magic, kStateMagic, 8);
    h.version = kStateVersion;
    h.has_d = has_d ? 1 : 0;
    h.n_rays = S->n_rays;
    h.n_vox = S->n_vox;
    h.n_tiles = p.n;
    h.z_floats = p.z_floats;
    h.hist_rows = rows;
    h.queue_len = (int64_t)S->queue.size();
    h.queue_ints = L.queue_ints;
    h.prm = S->prm;
    h.rng_state = S->rng.state;
    h.epoch = S->epoch;
    h.steps_done = S->steps_done;
    h.epoch_open = S->epoch_open ? 1 : 0;
    h.last_group = S->last_group;
    unsigned long long nnz = 0;
    CSGD_CUDA(cudaMemcpyAsync(&nnz, S->sb.nnz, sizeof(nnz), cudaMemcpyDeviceToHost, s), "read nnz");
    int32_t* qi = (int32_t*)(out + L.off_queue);
    for (const QueuedStep& q : S->queue) {
        *qi++ = q.j;
        *qi++ = (int32_t)q.group.size();
        *qi++ = q.last_in_batch ? 1 : 0;
        for (int g : q.group) *qi++ = g;
    }
    auto d2h = [&](int64_t off, const void* src, int64_t bytes, const char* what) {
        if (bytes <= 0) return cudaSuccess;
        cudaError_t e = cudaMemcpyAsync(out + off, src, (size_t)bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) fail(CSGD_ERR_CUDA, what);
        return e;
    };
    if (d2h(L.off_y, S->sb.y, 4 * S->n_rays, "read y") != cudaSuccess ||
        d2h(L.off_x, S->sb.x, 4 * S->n_vox, "read x") != cudaSuccess ||
        d2h(L.off_xh, S->sb.xh, 4 * S->n_vox, "read x^") != cudaSuccess ||
        d2h(L.off_r, S->sb.r, 4 * S->n_rays, "read r") != cudaSuccess ||
        d2h(L.off_z, S->sb.z, 4 * p.z_floats, "read z") != cudaSuccess ||
        (has_d && d2h(L.off_d, S->sb.d, 4 * S->n_rays, "read d") != cudaSuccess) ||
        d2h(L.off_cnt, S->sb.cnt, 4 * (int64_t)p.n, "read counts") != cudaSuccess ||
        d2h(L.off_hist, S->sb.hist, 8 * kHistCols * rows, "read history") != cudaSuccess)
        return CSGD_ERR_CUDA;
    CSGD_CUDA(cudaStreamSynchronize(s), "state sync");
    h.nnz = nnz;
    std::memcpy(out, &h, sizeof(h));
    return CSGD_OK;
}

int32_t csgd_solver_set_state(csgd_solver* S, const void* buf, int64_t size, csgd_stream stream) {
    if (!S || !buf) return fail(CSGD_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Partition& p = S->P->p;
    if (size < (int64_t)sizeof(StateHeader)) return fail(CSGD_ERR_STATE, "not a solver state");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kStateMagic, 8) != 0 || h.version != kStateVersion)
        return fail(CSGD_ERR_STATE, "not a solver state of this version");
    const bool has_d = S->prm.sync == CSGD_SYNC_EPOCH;
    if (h.n_rays != S->n_rays || h.n_vox != S->n_vox || h.n_tiles != p.n ||
        h.z_floats != p.z_floats || (h.has_d != 0) != has_d)
        return fail(CSGD_ERR_STATE, "state of a solver with other sizes");
    if (!same_params(h.prm, S->prm)) return fail(CSGD_ERR_STATE, "state of a solver with other parameters");
    if (h.hist_rows < 0 || h.hist_rows > h.steps_done || h.queue_len < 0 || h.queue_ints < 3 * h.queue_len)
        return fail(CSGD_ERR_STATE, "corrupt state header");
    const StateLayout L = state_layout(S, h.queue_ints, h.hist_rows, has_d);
    if (size < L.total) return fail(CSGD_ERR_STATE, "truncated solver state");
    // the queued schedule, checked before anything is changed
    const char* in = (const char*)buf;
    const int32_t* qi = (const int32_t*)(in + L.off_queue);
    const int32_t* qe = qi + h.queue_ints;
    std::deque<QueuedStep> queue;
    for (int64_t k = 0; k < h.queue_len; ++k) {
        if (qe - qi < 3) return fail(CSGD_ERR_STATE, "corrupt schedule section");
        QueuedStep q;
        q.j = qi[0];
        const int32_t ng = qi[1];
        q.last_in_batch = qi[2] != 0;
        qi += 3;
        if (q.j < 0 || q.j >= p.n || ng < 0 || ng > p.m || qe - qi < ng)
            return fail(CSGD_ERR_STATE, "corrupt schedule section");
        for (int32_t g = 0; g < ng; ++g) {
            if (qi[g] < 0 || qi[g] >= p.m) return fail(CSGD_ERR_STATE, "corrupt schedule section");
            q.group.push_back(qi[g]);
        }
        qi += ng;
        queue.push_back(std::move(q));
    }
    int rc = ensure_history(S, std::max<int64_t>(h.hist_rows, 1), s);
    if (rc) return rc;
    auto h2d = [&](void* dst, int64_t off, int64_t bytes) {
        if (bytes <= 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, in + off, (size_t)bytes, cudaMemcpyHostToDevice, s);
    };
    const unsigned long long nnz = h.nnz;
    cudaError_t e = h2d((void*)S->sb.y, L.off_y, 4 * S->n_rays);
    if (e == cudaSuccess) e = h2d(S->sb.x, L.off_x, 4 * S->n_vox);
    if (e == cudaSuccess) e = h2d(S->sb.xh, L.off_xh, 4 * S->n_vox);
    if (e == cudaSuccess) e = h2d(S->sb.r, L.off_r, 4 * S->n_rays);
    if (e == cudaSuccess) e = h2d(S->sb.z, L.off_z, 4 * p.z_floats);
    if (e == cudaSuccess && has_d) e = h2d(S->sb.d, L.off_d, 4 * S->n_rays);
    if (e == cudaSuccess) e = h2d(S->sb.cnt, L.off_cnt, 4 * (int64_t)p.n);
    if (e == cudaSuccess) e = h2d(S->sb.hist, L.off_hist, 8 * kHistCols * h.hist_rows);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->sb.nnz, &nnz, sizeof(nnz), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "restore solver state");
    S->rng.state = h.rng_state;
    S->epoch = h.epoch;
    S->steps_done = h.steps_done;
    S->epoch_open = h.epoch_open != 0;
    S->last_group = h.last_group;
    S->queue = std::move(queue);
    return CSGD_OK;
}

// ---------------------------------------------------------------------------
// launch shapes and their autotuning
// ---------------------------------------------------------------------------
int32_t csgd_solver_set_launch(csgd_solver* S, int32_t bp_groups, int32_t fwd_lanes) {
    if (!S) return fail(CSGD_ERR_INVALID_ARG, "NULL solver");
    if (bp_groups < kBPBrickLast || bp_groups > kBPMaxChunks)
        return fail(CSGD_ERR_INVALID_ARG,
                    "view groups must be -4..-2 (bricks), -1 (scatter), 0 (model) or 1..8");
    if (fwd_lanes != 0 && fwd_lanes != 1 && fwd_lanes != 2 && fwd_lanes != 4)
        return fail(CSGD_ERR_INVALID_ARG, "lanes per ray must be 0 (model), 1, 2 or 4");
    S->bp_groups = bp_groups;
    S->fwd_lanes = fwd_lanes;
    return CSGD_OK;
}

namespace {
// Device time of the backprojection (kind 0), the dual forward (kind 1) or both
// (kind 2) over the first `steps` scheduled steps from a fresh state.
int trial_ms(csgd_solver* S, int64_t steps, int kind, cudaStream_t s, double* ms) {
    int rc = solver_reset_state(S, s);
    if (rc) return rc;
    rc = csgd_solver_profile(S, 1);
    if (rc) return rc;
    csgd_kernel_times t{};
    csgd_solver_profile_read(S, &t, 1);
    Plan pl;
    plan_scheduled(S, &pl, steps, false);
    rc = execute_plan(S, pl, s);
    if (rc == CSGD_OK) rc = csgd_solver_profile_read(S, &t, 1);
    csgd_solver_profile(S, 0);
    if (rc) return rc;
    *ms = kind == 2 ? t.ms[0] + t.ms[1] : t.ms[kind];
    return CSGD_OK;
}
}  // namespace

int32_t csgd_solver_autotune(csgd_solver* S, int64_t trial_steps, int32_t* bp_groups,
                             int32_t* fwd_lanes, csgd_stream stream) {
    if (!S || trial_steps <= 0) return fail(CSGD_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    double ms = 0.0;
    S->bp_groups = 0;
    S->fwd_lanes = 0;
    int rc = trial_ms(S, trial_steps, 0, s, &ms);  // warm-up (module loading, caches)
    int best_c = 0;
    double best = 0.0;
    // the gather with 1..8 view groups per CTA, then the scatter, then the bricks
    const int n_shapes = kBPMaxChunks + 1 + (kBPBrick - kBPBrickLast + 1);
    for (int c = 1; rc == CSGD_OK && c <= n_shapes; ++c) {
        S->bp_groups = c <= kBPMaxChunks ? c
                     : (c == kBPMaxChunks + 1 ? kBPScatter : kBPBrick - (c - kBPMaxChunks - 2));
        rc = trial_ms(S, trial_steps, 0, s, &ms);
        if (rc == CSGD_OK && (best_c == 0 || ms < best)) {
            best = ms;
            best_c = S->bp_groups;
        }
    }
    S->bp_groups = best_c;
    // lanes per ray: the dual forward's, which the scatter shares
    const int kind = best_c == kBPScatter ? 2 : 1;
    // (the brick backprojection has no lanes; its forward sets its own lines up)
    int best_l = 0;
    for (int l = 1; rc == CSGD_OK && l <= 4; l *= 2) {
        S->fwd_lanes = l;
        rc = trial_ms(S, trial_steps, kind, s, &ms);
        if (rc == CSGD_OK && (best_l == 0 || ms < best)) {  // l = 1 starts the comparison
            best = ms;
            best_l = l;
        }
    }
    if (rc != CSGD_OK) {
        S->bp_groups = S->fwd_lanes = 0;
        solver_reset_state(S, s);
        return rc;
    }
    S->fwd_lanes = best_l;
    rc = solver_reset_state(S, s);
    if (rc) return rc;
    CSGD_CUDA(cudaStreamSynchronize(s), "autotune sync");
    if (bp_groups) *bp_groups = S->bp_groups;
    if (fwd_lanes) *fwd_lanes = S->fwd_lanes;
    return CSGD_OK;
}
