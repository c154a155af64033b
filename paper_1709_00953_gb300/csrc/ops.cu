// Siddon block operators and the solver's per-batch kernels (sm_103a).
//
//   k_forward      z_I = A_I^J x_J (one vector) or, in the solver, p = A x_J and
//                  q = A g_J in one traversal with ||q||^2 in FP64 and the step
//                  length mu computed by the last CTA (Alg. 1 lines 2-3).
//   k_backproject  g_J = (A_I^J)^T r_I (Eq. 'direction'): ray-driven traversal of a
//                  shared-memory sub-box of the tile, partial sums reduced across
//                  the CTAs of a thread-block cluster through distributed shared
//                  memory, g^T g in FP64.  No global atomics.
//   k_epilogue     z_I^j = p + mu q, r -= z_new - z_old (the refresh of Alg. 2-4
//                  applied incrementally), x^_J += x_J + mu g_J.
//   k_average      x_J = x^_J / count_J at the end of an epoch.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>

#include "device.cuh"
#include "ops.h"

namespace cg = cooperative_groups;

namespace csgd {

namespace {

constexpr int kFwdThreads = 256;
constexpr int kBPThreads = 256;
constexpr int kEpiThreads = 256;
constexpr int kMaxSubboxFloats = 16384;  // 64 KB of shared memory per CTA

__device__ __forceinline__ Box tile_box(const DevTile& t, int dim, int base, int s1, int s2) {
    Box b;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = a < dim ? -0.5f * (float)t.n[a] : -0.5f;
        b.n[a] = a < dim ? t.n[a] : 1;
    }
    b.stride[0] = 1;
    b.stride[1] = s1;
    b.stride[2] = s2;
    b.base = base;
    return b;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
struct FwdSolverArgs {
    DevGeom G;
    const WorkItem* items;
    const StepDesc* steps;
    int first;
    int sync_epoch;
    int n_gg;  // g^T g partials per slot written by the backprojection
    SolverBuffers sb;
};

template <int DIM>
__device__ __forceinline__ void forward_single(const DevGeom& G, const WorkItem* items,
                                               const StepDesc& sd, const float* x, float* out,
                                               int accumulate) {
    const DevTile t = G.tiles[sd.j];
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= sd.n_rays) return;
    int w = find_item(items, sd.w0, sd.w1, k);
    const WorkItem it = items[w];
    int64_t within = k - it.ray_off;
    int wu = it.u1 - it.u0;
    int ku = it.u0 + (int)(within % wu);
    int kv = it.v0 + (int)(within / wu);
    const DevView V = G.views[it.view];
    const DevVT E = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
    float q[3], d[3];
    ray_setup(G, V, E, ku, kv, q, d);
    int base = (t.lo[2] * G.ny + t.lo[1]) * G.nx + t.lo[0];
    Box b = tile_box(t, DIM, base, G.nx, G.nx * G.ny);
    Kahan acc;
    traverse<DIM>(q, d, b, [&](int idx, float len) { acc.add(len * __ldg(x + idx)); });
    int64_t ray = ray_index(G, it.view, ku, kv);
    float v = G.h * (acc.s - acc.c);
    out[ray] = accumulate ? out[ray] + v : v;
}

template <int DIM>
__global__ void __launch_bounds__(kFwdThreads) k_project_inline(
    const DevGeom G, const __grid_constant__ InlineItems it, const float* __restrict__ x,
    float* __restrict__ out, int accumulate) {
    forward_single<DIM>(G, it.items, it.step, x, out, accumulate);
}

template <int DIM>
__global__ void __launch_bounds__(kFwdThreads) k_forward_dual(const FwdSolverArgs a) {
    __shared__ double sh[kFwdThreads / 32];
    __shared__ int last;
    const DevGeom& G = a.G;
    const int slot = blockIdx.y;
    const StepDesc sd = a.steps[a.first + slot];
    const DevTile t = G.tiles[sd.j];
    const float* __restrict__ xj = a.sb.x + t.voff;
    const float* __restrict__ gj = a.sb.g + (int64_t)slot * a.sb.g_stride;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double qq = 0.0;
    long long nz = 0;
    if (k < sd.n_rays) {
        int w = find_item(a.items, sd.w0, sd.w1, k);
        const WorkItem it = a.items[w];
        int64_t within = k - it.ray_off;
        int wu = it.u1 - it.u0;
        int ku = it.u0 + (int)(within % wu);
        int kv = it.v0 + (int)(within / wu);
        const DevView V = G.views[it.view];
        const DevVT E = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
        float q[3], d[3];
        ray_setup(G, V, E, ku, kv, q, d);
        Box b = tile_box(t, DIM, 0, t.n[0], t.n[0] * t.n[1]);
        Kahan ax, ag;
        nz = traverse<DIM>(q, d, b, [&](int idx, float len) {
            ax.add(len * __ldg(xj + idx));
            ag.add(len * __ldg(gj + idx));
        });
        int64_t ray = ray_index(G, it.view, ku, kv);
        float pv = G.h * (ax.s - ax.c);
        float qv = G.h * (ag.s - ag.c);
        a.sb.p[ray] = pv;
        a.sb.q[ray] = qv;
        qq = (double)qv * (double)qv;
    }
    double bq = block_sum(qq, sh);
    __syncthreads();
    double bn = block_sum((double)nz, sh);
    if (threadIdx.x == 0) {
        a.sb.qq_part[(int64_t)slot * a.sb.max_fwd_blocks + blockIdx.x] = bq;
        atomicAdd(a.sb.nnz, (unsigned long long)bn);
        atomicAdd(a.sb.nnz_slot + slot, (unsigned long long)bn);
        __threadfence();
        unsigned prev = atomicAdd(a.sb.counters + slot, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        // fixed-order sums: deterministic
        double qs = 0.0;
        for (int bb = 0; bb < (int)gridDim.x; ++bb)
            qs += __ldcg(a.sb.qq_part + (int64_t)slot * a.sb.max_fwd_blocks + bb);
        const int ngg = a.n_gg;
        double gs = 0.0;
        for (int bb = 0; bb < ngg; ++bb) gs += __ldcg(a.sb.gg_part + (int64_t)slot * ngg + bb);
        double mu = qs > 0.0 ? sd.beta * gs / qs : 0.0;
        a.sb.mu[slot] = mu;
        unsigned long long nzs = atomicExch(a.sb.nnz_slot + slot, 0ull);
        if (sd.step >= 0 && sd.step < a.sb.hist_cap) {
            double* hrow = a.sb.hist + kHistCols * sd.step;
            hrow[0] = sd.beta;
            hrow[1] = gs;
            hrow[2] = qs;
            hrow[3] = mu;
            hrow[4] = (double)nzs;
        }
        a.sb.counters[slot] = 0u;
    }
}

// ---------------------------------------------------------------------------
// backprojection
// ---------------------------------------------------------------------------
struct BPArgs {
    DevGeom G;
    int first;
    int nsb;
    const float* r;
    float* gout;       // tile-local scratch (mode 0) or row-major volume (mode 1)
    int mode;
    int accumulate;
    int64_t slot_stride;
    double* gg_part;   // [slot][nsb * C] or null
};

template <int DIM>
__device__ __forceinline__ void backproject_body(const BPArgs& a, const WorkItem* items,
                                                 const StepDesc& sd, float* acc) {
    cg::cluster_group cluster = cg::this_cluster();
    const DevGeom& G = a.G;
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int slot = blockIdx.z;
    const int sb = blockIdx.y;
    const DevTile t = G.tiles[sd.j];
    // sub-box: cut along the last axis
    const int ax = DIM - 1;
    const int W = t.n[ax];
    const int s0 = (int)(((int64_t)sb * W) / a.nsb);
    const int s1 = (int)(((int64_t)(sb + 1) * W) / a.nsb);
    Box b;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        b.lo[c] = c < DIM ? -0.5f * (float)t.n[c] : -0.5f;
        b.n[c] = c < DIM ? t.n[c] : 1;
    }
    b.lo[ax] += (float)s0;
    b.n[ax] = s1 - s0;
    b.stride[0] = 1;
    b.stride[1] = b.n[0];
    b.stride[2] = b.n[0] * b.n[1];
    b.base = 0;
    const int nvox = b.n[0] * b.n[1] * b.n[2];
    for (int v = threadIdx.x; v < nvox; v += blockDim.x) acc[v] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float* __restrict__ r = a.r;
    for (int w = sd.w0 + rank; w < sd.w1; w += C) {
        const WorkItem it = items[w];
        const DevView V = G.views[it.view];
        const DevVT E = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
        // bins whose lines can meet this sub-box: project its corners (lanes 0..7)
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        if (lane < (1 << DIM)) {
            float P[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float off = c < DIM ? (((lane >> c) & 1) ? b.lo[c] + (float)b.n[c] : b.lo[c]) : 0.f;
                P[c] = t.T[c] + off;
            }
            float wu, wv;
            detector_coord(G, V, P, &wu, &wv);
            umin = umax = wu;
            vmin = vmax = wv;
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
            umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        }
        umin = __shfl_sync(0xffffffffu, umin, 0);
        umax = __shfl_sync(0xffffffffu, umax, 0);
        vmin = __shfl_sync(0xffffffffu, vmin, 0);
        vmax = __shfl_sync(0xffffffffu, vmax, 0);
        int u0 = max(it.u0, (int)ceilf(umin - 0.5f) - 1);
        int u1 = min(it.u1, (int)floorf(umax - 0.5f) + 2);
        int v0 = it.v0, v1 = it.v1;
        if (DIM == 3) {
            v0 = max(it.v0, (int)ceilf(vmin - 0.5f) - 1);
            v1 = min(it.v1, (int)floorf(vmax - 0.5f) + 2);
        }
        if (u1 <= u0 || v1 <= v0) continue;
        const int wu = u1 - u0;
        const int nr = wu * (v1 - v0);
        for (int k = threadIdx.x; k < nr; k += blockDim.x) {
            int ku = u0 + k % wu;
            int kv = v0 + k / wu;
            float rv = __ldg(r + ray_index(G, it.view, ku, kv));
            if (rv == 0.f) continue;
            float q[3], d[3];
            ray_setup(G, V, E, ku, kv, q, d);
            traverse<DIM>(q, d, b, [&](int idx, float len) {
                if (len > 0.f) atomicAdd(acc + idx, len * rv);
            });
        }
    }
    cluster.sync();
    // each CTA of the cluster reduces one slice of the sub-box over all ranks
    const int v_lo = (int)(((int64_t)rank * nvox) / C);
    const int v_hi = (int)(((int64_t)(rank + 1) * nvox) / C);
    double gg = 0.0;
    for (int v = v_lo + threadIdx.x; v < v_hi; v += blockDim.x) {
        float s = 0.f;
        for (int rr = 0; rr < C; ++rr) s += cluster.map_shared_rank(acc, rr)[v];
        s *= G.h;
        int x0 = v % b.n[0];
        int rest = v / b.n[0];
        int x1 = rest % b.n[1];
        int x2 = rest / b.n[1];
        if (ax == 1) x1 += s0; else x2 += s0;
        if (a.mode == 0) {
            int64_t li = ((int64_t)x2 * t.n[1] + x1) * t.n[0] + x0;
            a.gout[(int64_t)slot * a.slot_stride + li] = s;
        } else {
            int64_t gi = ((int64_t)(t.lo[2] + x2) * G.ny + (t.lo[1] + x1)) * G.nx + t.lo[0] + x0;
            a.gout[gi] = a.accumulate ? a.gout[gi] + s : s;
        }
        gg += (double)s * (double)s;
    }
    if (a.gg_part) {
        __shared__ double sh[kBPThreads / 32];
        double bg = block_sum(gg, sh);
        if (threadIdx.x == 0)
            a.gg_part[((int64_t)slot * a.nsb + sb) * C + rank] = bg;
    }
    cluster.sync();
}

template <int DIM>
__global__ void __launch_bounds__(kBPThreads) k_backproject_inline(
    const BPArgs a, const __grid_constant__ InlineItems it) {
    extern __shared__ float acc[];
    backproject_body<DIM>(a, it.items, it.step, acc);
}

template <int DIM>
__global__ void __launch_bounds__(kBPThreads) k_backproject_solver(
    const BPArgs a, const WorkItem* __restrict__ items, const StepDesc* __restrict__ steps) {
    extern __shared__ float acc[];
    const StepDesc sd = steps[a.first + blockIdx.z];
    backproject_body<DIM>(a, items, sd, acc);
}

// ---------------------------------------------------------------------------
// epilogue, averaging, conversions
// ---------------------------------------------------------------------------
struct EpiArgs {
    DevGeom G;
    const WorkItem* items;
    const StepDesc* steps;
    int first;
    int nslots;
    int j;
    int sync_epoch;
    SolverBuffers sb;
};

__global__ void __launch_bounds__(kEpiThreads) k_epilogue(const EpiArgs a) {
    const DevGeom& G = a.G;
    if ((int)blockIdx.y < a.nslots) {
        const int slot = blockIdx.y;
        const StepDesc sd = a.steps[a.first + slot];
        const float mu = (float)a.sb.mu[slot];
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < sd.n_rays;
             k += (int64_t)gridDim.x * blockDim.x) {
            int w = find_item(a.items, sd.w0, sd.w1, k);
            const WorkItem it = a.items[w];
            int64_t within = k - it.ray_off;
            int wu = it.u1 - it.u0;
            int ku = it.u0 + (int)(within % wu);
            int kv = it.v0 + (int)(within / wu);
            const DevVT& E = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
            int64_t zi = E.zoff + (int64_t)(kv - E.v0) * (E.u1 - E.u0) + (ku - E.u0);
            int64_t ray = ray_index(G, it.view, ku, kv);
            float zn = fmaf(mu, a.sb.q[ray], a.sb.p[ray]);
            float zo = a.sb.z[zi];
            a.sb.z[zi] = zn;
            if (a.sync_epoch) a.sb.d[ray] += zn - zo;
            else a.sb.r[ray] -= zn - zo;
        }
    } else {
        const DevTile t = G.tiles[a.j];
        const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
        float* xh = a.sb.xh + t.voff;
        const float* x = a.sb.x + t.voff;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
             v += (int64_t)gridDim.x * blockDim.x) {
            float xv = x[v];
            float s = xh[v];
            for (int sl = 0; sl < a.nslots; ++sl)
                s += fmaf((float)a.sb.mu[sl], a.sb.g[(int64_t)sl * a.sb.g_stride + v], xv);
            xh[v] = s;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sb.cnt[a.j] += a.nslots;
    }
}

__global__ void k_average(const DevGeom G, float* x, float* xh, const int32_t* cnt) {
    const int j = blockIdx.y;
    const DevTile t = G.tiles[j];
    const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
    const int c = cnt[j];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (c > 0) x[t.voff + v] = xh[t.voff + v] / (float)c;
        xh[t.voff + v] = 0.f;
    }
}

__global__ void k_apply_pending(float* r, float* d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float dv = d[i];
        if (dv != 0.f) {
            r[i] -= dv;
            d[i] = 0.f;
        }
    }
}

__global__ void k_tile_to_rowmajor(const DevGeom G, const float* xt, float* out) {
    const int j = blockIdx.y;
    const DevTile t = G.tiles[j];
    const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)gridDim.x * blockDim.x) {
        int x0 = (int)(v % t.n[0]);
        int64_t rest = v / t.n[0];
        int x1 = (int)(rest % t.n[1]);
        int x2 = (int)(rest / t.n[1]);
        int64_t gi = ((int64_t)(t.lo[2] + x2) * G.ny + t.lo[1] + x1) * G.nx + t.lo[0] + x0;
        out[gi] = xt[t.voff + v];
    }
}

__global__ void k_sq_residual(const float* y, const float* ax, int64_t n, double* out) {
    __shared__ double sh[8];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double e = (double)y[i] - (double)ax[i];
        s += e * e;
    }
    double b = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = b;
}

template <class K>
void set_smem(K kernel, int bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
BPPlan plan_backprojection(const DevGeom& G, const DevTile& tile, int nslots, int sm_count) {
    BPPlan p;
    const int ax = G.dim - 1;
    const int64_t nv = (int64_t)tile.n[0] * tile.n[1] * tile.n[2];
    const int64_t slab = nv / tile.n[ax];  // voxels per unit thickness along ax
    int nsb = (int)((nv + kMaxSubboxFloats - 1) / kMaxSubboxFloats);
    p.C = 8;
    // enough CTAs for about two waves, but sub-boxes of at least 4096 voxels
    int64_t want = (int64_t)2 * sm_count;
    while ((int64_t)nsb * p.C * nslots < want && nv / (nsb + 1) >= 4096 && nsb < tile.n[ax])
        ++nsb;
    if (nsb > tile.n[ax]) nsb = tile.n[ax];
    p.nsb = nsb;
    int64_t thick = (tile.n[ax] + nsb - 1) / nsb;
    p.smem_bytes = (int)(thick * slab * sizeof(float));
    return p;
}

static cudaError_t launch_bp_common(const DevGeom& G, const BPPlan& plan, int nslots,
                                    cudaStream_t s, const BPArgs& a, const InlineItems* inl,
                                    const WorkItem* items, const StepDesc* steps) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.C, plan.nsb, nslots);
    cfg.blockDim = dim3(kBPThreads);
    cfg.dynamicSmemBytes = plan.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (inl) {
        if (G.dim == 2) {
            set_smem(k_backproject_inline<2>, plan.smem_bytes);
            return cudaLaunchKernelEx(&cfg, k_backproject_inline<2>, a, *inl);
        }
        set_smem(k_backproject_inline<3>, plan.smem_bytes);
        return cudaLaunchKernelEx(&cfg, k_backproject_inline<3>, a, *inl);
    }
    if (G.dim == 2) {
        set_smem(k_backproject_solver<2>, plan.smem_bytes);
        return cudaLaunchKernelEx(&cfg, k_backproject_solver<2>, a, items, steps);
    }
    set_smem(k_backproject_solver<3>, plan.smem_bytes);
    return cudaLaunchKernelEx(&cfg, k_backproject_solver<3>, a, items, steps);
}

cudaError_t launch_project_inline(const DevGeom& G, const InlineItems& it, const float* x,
                                  float* out, int accumulate, cudaStream_t s) {
    if (it.step.n_rays <= 0) return cudaSuccess;
    dim3 grid((unsigned)((it.step.n_rays + kFwdThreads - 1) / kFwdThreads));
    if (G.dim == 2)
        k_project_inline<2><<<grid, kFwdThreads, 0, s>>>(G, it, x, out, accumulate);
    else
        k_project_inline<3><<<grid, kFwdThreads, 0, s>>>(G, it, x, out, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_backproject_inline(const DevGeom& G, const DevTile& tile,
                                      const InlineItems& it, const float* r, float* g,
                                      int accumulate, int sm_count, cudaStream_t s) {
    BPPlan plan = plan_backprojection(G, tile, 1, sm_count);
    BPArgs a;
    a.G = G;
    a.first = 0;
    a.nsb = plan.nsb;
    a.r = r;
    a.gout = g;
    a.mode = 1;
    a.accumulate = accumulate;
    a.slot_stride = 0;
    a.gg_part = nullptr;
    cudaError_t e = launch_bp_common(G, plan, 1, s, a, &it, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_batch(const DevGeom& G, const DevTile& tile, const WorkItem* items,
                         const StepDesc* steps, const BatchLaunch& b, const SolverBuffers& sb,
                         int sm_count, cudaStream_t s, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], s);
    BPPlan plan = plan_backprojection(G, tile, b.nslots, sm_count);
    // 1. g_J = (A_I^J)^T r_I per slot
    BPArgs a;
    a.G = G;
    a.first = b.first;
    a.nsb = plan.nsb;
    a.r = sb.r;
    a.gout = sb.g;
    a.mode = 0;
    a.accumulate = 0;
    a.slot_stride = sb.g_stride;
    a.gg_part = sb.gg_part;
    cudaError_t e = launch_bp_common(G, plan, b.nslots, s, a, nullptr, items, steps);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    // 2. p = A x_J, q = A g_J, ||q||^2, mu
    FwdSolverArgs f;
    f.G = G;
    f.items = items;
    f.steps = steps;
    f.first = b.first;
    f.sync_epoch = b.sync_epoch;
    f.n_gg = plan.nsb * plan.C;
    f.sb = sb;
    int64_t nb = (b.max_rays + kFwdThreads - 1) / kFwdThreads;
    if (nb < 1) nb = 1;
    if (nb > sb.max_fwd_blocks) return cudaErrorInvalidValue;
    dim3 grid((unsigned)nb, b.nslots);
    if (G.dim == 2) k_forward_dual<2><<<grid, kFwdThreads, 0, s>>>(f);
    else k_forward_dual<3><<<grid, kFwdThreads, 0, s>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[2], s);
    // 3. z, r and x^ updates
    EpiArgs ea;
    ea.G = G;
    ea.items = items;
    ea.steps = steps;
    ea.first = b.first;
    ea.nslots = b.nslots;
    ea.j = b.j;
    ea.sync_epoch = b.sync_epoch;
    ea.sb = sb;
    int64_t eb = (b.max_rays + kEpiThreads - 1) / kEpiThreads;
    eb = std::max<int64_t>(1, std::min<int64_t>(eb, 4 * sm_count));
    k_epilogue<<<dim3((unsigned)eb, b.nslots + 1), kEpiThreads, 0, s>>>(ea);
    e = cudaGetLastError();
    if (ev) cudaEventRecord(ev[3], s);
    return e;
}

cudaError_t launch_epoch_close(const DevGeom& G, const SolverBuffers& sb, int64_t n_rays,
                               int64_t max_tile_voxels, int sync_epoch, cudaStream_t s) {
    if (sync_epoch) {
        int64_t nb = std::min<int64_t>((n_rays + 255) / 256, 4096);
        k_apply_pending<<<(unsigned)std::max<int64_t>(nb, 1), 256, 0, s>>>(sb.r, sb.d, n_rays);
    }
    int64_t nb = std::min<int64_t>((max_tile_voxels + 255) / 256, 1024);
    k_average<<<dim3((unsigned)std::max<int64_t>(nb, 1), G.n_tiles), 256, 0, s>>>(G, sb.x, sb.xh,
                                                                                  sb.cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(sb.cnt, 0, sizeof(int32_t) * G.n_tiles, s);
}

cudaError_t launch_tile_to_rowmajor(const DevGeom& G, const float* xt, float* out,
                                    int64_t max_tile_voxels, cudaStream_t s) {
    int64_t nb = std::min<int64_t>((max_tile_voxels + 255) / 256, 1024);
    k_tile_to_rowmajor<<<dim3((unsigned)std::max<int64_t>(nb, 1), G.n_tiles), 256, 0, s>>>(G, xt,
                                                                                          out);
    return cudaGetLastError();
}

cudaError_t launch_sq_residual(const float* y, const float* ax, int64_t n, double* out,
                               cudaStream_t s) {
    k_sq_residual<<<256, 256, 0, s>>>(y, ax, n, out);
    return cudaGetLastError();
}

}  // namespace csgd
