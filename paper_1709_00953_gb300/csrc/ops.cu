// Siddon block operators and the solver's per-batch kernels (sm_103a).
//
//   k_project_inline  z_I = A_I^J x_J for the stand-alone operator: ray-driven
//                     incremental walk, 1-4 lanes per ray.
//   k_ray_table_*     per launch, the line (tile-centred point q, 1/d) and the
//                     residual r of every ray of every slot, set up once (and
//                     max |r| per slot for the scatter).
//   k_backproject_*   g_J = (A_I^J)^T r_I (Eq. 'direction'): voxel-driven gather
//                     over the ray table (each voxel sums len * r over the bins
//                     of its shadow), the partial sums of a CTA's view groups
//                     added in shared memory in a fixed order, g^T g per CTA.
//                     No atomics.
//   k_backproject_scatter + k_scatter_convert
//                     the same g_J ray-driven: every ray walks the tile and adds
//                     len * r to 32-bit fixed-point sums with integer atomics
//                     (exact, order-independent), then one pass converts them.
//   k_forward_dual    p = A x_J and q = A g_J in one walk per ray, ||q||^2 per
//                     CTA, the step length mu computed by the last CTA of each
//                     slot (Alg. 1, Eq. 'step').
//   k_epilogue        z_I^j = p + mu q, r -= z_new - z_old (the refresh of
//                     Alg. 2-4 applied incrementally), x^_J += x_J + mu g_J.
//   k_average         x_J = x^_J / count_J at the end of an epoch
//                     (k_apply_pending first under epoch sync).
// The kernels of the solver's batch sequence are launched with programmatic
// stream serialization (see pdl_wait in device.cuh).
#include <cuda_runtime.h>

#include <string.h>

#include <algorithm>
#include <new>
#include <vector>
#include <mutex>
#include <utility>

#include "device.cuh"
#include "ops.h"

namespace csgd {

namespace {

constexpr int kFwdBatch = 4;  // crossings per batch of gathers in the dual forward
constexpr int kMaxBlock = 256;  // most threads of any CTA of the solver's kernels

// Index of a thread block in its grid as the kernel bodies see it: blockIdx and
// gridDim for an ordinary launch; for the batch executor (one persistent
// launch running many kernels' blocks) the block of the unit it runs.
struct VBlock {
    unsigned x, y, z;     // block index
    unsigned gx, gy, gz;  // grid size
};
__device__ __forceinline__ VBlock hw_block() {
    return VBlock{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// Load of data an earlier kernel of the stream wrote: through the read-only
// cache in an ordinary launch (written before the kernel started); a plain
// load inside the executor, where the writer may be another block of the same
// launch (ordered by the executor's acquire, which the read-only path is not).
template <bool EX, class T>
__device__ __forceinline__ T ldro(const T* p) {
    if constexpr (EX) return *p;
    else return __ldg(p);
}
constexpr int kBPMaxThreads = kBPVox * kBPMaxChunks;
constexpr int kEpiThreads = 256;

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

// Line of bin (ku, kv) of view `view` in tile-centred coordinates: q and 1/d.
template <int DIM>
__device__ __forceinline__ void table_ray(const DevGeom& G, int view, const DevView& V,
                                          const DevVT& E, const DevTile& tile, int ku, int kv,
                                          float q[3], float inv[3]) {
    float d[3];
    ray_setup(G, V, E, ku, kv, q, d);
    reciprocal(d, inv);
    // a line parallel to the planes of axis ax (d exactly 0 there, in FP32 as
    // in FP64: a view at a multiple of 90 degrees) is put on the exact line's
    // side of its nearest voxel face, one ulp above a face it lies on
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax)
        if (isinf(inv[ax])) q[ax] = parallel_coord(G, view, ku, kv, tile, ax);
    // a line that only touches the tile (see exact_chord) gets no support in it
    const Box b = tile_box(tile, DIM, 0, tile.n[0], tile.n[0] * tile.n[1]);
    float tin, tout;
    bool sliver;
    if (clip_sliver<DIM>(q, inv, b, &tin, &tout, &sliver) && sliver &&
        exact_chord(G, view, ku, kv, tile) <= kTouchChord)
        q[0] = kNoSupport;
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

// Rays of one slot are split among L consecutive lanes by parameter range: every
// lane walks 1/L of the ray's chord through the tile and the L partial sums are
// combined with warp shuffles, so that short chains of dependent gathers keep
// more warps in flight.
template <int L>
__device__ __forceinline__ float lane_sum(float v) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int DIM, int L>
__device__ __forceinline__ void forward_single(const DevGeom& G, const WorkItem* items,
                                               const StepDesc& sd, const float* x, float* out,
                                               int accumulate) {
    const DevTile t = G.tiles[sd.j];
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t k = gid / L;
    const int sub = (int)(gid % L);
    const bool active = k < sd.n_rays;
    float part = 0.f;
    int64_t ray = 0;
    if (active) {
        int w = find_item(items, sd.w0, sd.w1, k);
        const WorkItem it = items[w];
        int64_t within = k - it.ray_off;
        int wu = it.u1 - it.u0;
        int ku = it.u0 + (int)(within % wu);
        int kv = it.v0 + (int)(within / wu);
        const DevView V = G.views[it.view];
        const DevVT E = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
        float q[3], inv[3];
        table_ray<DIM>(G, it.view, V, E, t, ku, kv, q, inv);  // the solver's line set-up
        int base = (t.lo[2] * G.ny + t.lo[1]) * G.nx + t.lo[0];
        Box b = tile_box(t, DIM, base, G.nx, G.nx * G.ny);
        float tin, tout;
        if (clip<DIM>(q, inv, b, &tin, &tout)) {
            float dt = (tout - tin) * (1.0f / L);
            float t0 = sub == 0 ? tin : fmaf((float)sub, dt, tin);
            float t1 = sub == L - 1 ? tout : fmaf((float)(sub + 1), dt, tin);
            Kahan acc;
            float plen = 0.f, pxv = 0.f;  // gather consumed one crossing later
            walk<DIM>(q, inv, b, t0, t1, [&](int idx, float len) {
                const float xv = __ldg(x + idx);
                acc.add(plen * pxv);
                plen = len;
                pxv = xv;
            });
            acc.add(plen * pxv);
            part = acc.s - acc.c;
        }
        ray = ray_index(G, it.view, ku, kv);
    }
    float v = G.h * lane_sum<L>(part);
    if (active && sub == 0) out[ray] = accumulate ? out[ray] + v : v;
}

template <int DIM, int L>
__global__ void __launch_bounds__(kFwdThreads) k_project_inline(
    const DevGeom G, const __grid_constant__ InlineItems it, const float* __restrict__ x,
    float* __restrict__ out, int accumulate) {
    forward_single<DIM, L>(G, it.items, it.step, x, out, accumulate);
}

// p = A x_J and q = A g_J for every ray of a slot in one walk (z = p + mu q by
// linearity), with ||q||^2.  Rays come from the batch's ray table (set up once
// for the backprojection), split over L lanes by parameter range.  Each CTA
// writes its partial sum of squares (FP32); the last CTA of the slot to finish
// adds them in a fixed order (exactly as FP32 pairs, then in FP64) and computes
// mu = beta g^T g / q^T q (no grid barrier).
template <int DIM, int L, bool TABLE, bool EX>
__device__ __forceinline__ void forward_dual_body(const FwdSolverArgs& a, const VBlock& vb) {
    pdl_trigger();
    const DevGeom& G = a.G;
    const int slot = vb.y;
    const StepDesc sd = a.steps[a.first + slot];
    const DevTile t = G.tiles[sd.j];
    const int nvox = t.n[0] * t.n[1] * t.n[2];
    const int lane = threadIdx.x & 31;
    int64_t gid = (int64_t)vb.x * blockDim.x + threadIdx.x;
    int64_t k = gid / L;
    const int sub = (int)(gid % L);
    const bool active = k < sd.n_rays;
    float pp = 0.f, qp = 0.f;
    int ray = 0;
    float q[3], inv[3];
    if constexpr (!TABLE) {
        // the line set up here, before the wait (it depends on the geometry
        // only), as the brick backprojection sets it up
        if (active) {
            const int w = find_item(a.items, sd.w0, sd.w1, k);
            const WorkItem it = a.items[w];
            const int within = (int)(k - it.ray_off);
            const int wu = it.u1 - it.u0;
            const int ku = it.u0 + within % wu, kv = it.v0 + within / wu;
            table_ray<DIM>(G, it.view, G.views[it.view], G.vt[(int64_t)it.view * G.n_tiles + sd.j],
                           t, ku, kv, q, inv);
            ray = (int)ray_index(G, it.view, ku, kv);
        }
    }
    pdl_wait();
    // (x_J, g_J) interleaved per voxel by the backprojection: one 8-byte gather per voxel
    const float2* __restrict__ xg = reinterpret_cast<const float2*>(a.sb.g) + (int64_t)slot * a.sb.g_stride;
    if (active) {
        if constexpr (TABLE) {
            const RayRec* rp = a.sb.table + (int64_t)slot * a.sb.table_stride + k;
            const float4 ra = *reinterpret_cast<const float4*>(rp->a);
            const float4 rb = *reinterpret_cast<const float4*>(rp->b);
            ray = __float_as_int(rb.w);
            q[0] = ra.x;
            q[1] = ra.y;
            q[2] = rb.y;
            inv[0] = ra.z;
            inv[1] = ra.w;
            inv[2] = rb.z;
        }
        Box b = tile_box(t, DIM, 0, t.n[0], t.n[0] * t.n[1]);
        float tin, tout;
        if (clip<DIM>(q, inv, b, &tin, &tout)) {
            float dt = (tout - tin) * (1.0f / L);
            float t0 = sub == 0 ? tin : fmaf((float)sub, dt, tin);
            float t1 = sub == L - 1 ? tout : fmaf((float)(sub + 1), dt, tin);
            // crossings in batches of kFwdBatch: the batch's (x, g) gathers are
            // all in flight before any is used.  A batch's terms are added as a
            // pairwise tree and the batch sum once into the lane's running sum:
            // for n terms the rounding error is at most (n / 4 + 3) u sum |term|
            // (u = 2^-24), below 1e-5 sum |term| while n < 650 (a lane meets at
            // most n_x + n_y (+ n_z) voxels of its tile: any 2D tile up to 320
            // voxels a side, any 3D tile up to 216).
            float sx = 0.f, sy = 0.f;
            auto batch = [&](const int (&id)[kFwdBatch], const float (&ln)[kFwdBatch]) {
                float2 e[kFwdBatch];
#pragma unroll
                for (int u = 0; u < kFwdBatch; ++u)
                    e[u] = ln[u] > 0.f && (unsigned)id[u] < (unsigned)nvox
                               ? ldro<EX>(xg + id[u]) : make_float2(0.f, 0.f);
                float px[kFwdBatch], py[kFwdBatch];
#pragma unroll
                for (int u = 0; u < kFwdBatch; ++u) {
                    px[u] = ln[u] * e[u].x;
                    py[u] = ln[u] * e[u].y;
                }
#pragma unroll
                for (int w = 1; w < kFwdBatch; w *= 2) {
#pragma unroll
                    for (int u = 0; u + w < kFwdBatch; u += 2 * w) {
                        px[u] += px[u + w];
                        py[u] += py[u + w];
                    }
                }
                sx += px[0];
                sy += py[0];
            };
            if constexpr (DIM == 2) walk2_batched<kFwdBatch>(q, inv, b, t0, t1, batch);
            else walk3_batched<kFwdBatch>(q, inv, b, t0, t1, batch);
            pp = sx;
            qp = sy;
        }
    }
    float pv = G.h * lane_sum<L>(pp);
    float qv = G.h * lane_sum<L>(qp);
    float qq = 0.f;
    if (active && sub == 0) {
        a.sb.p[ray] = pv;
        a.sb.q[ray] = qv;
        qq = qv * qv;
    }
    // per-CTA partials in FP32 (the squares, a warp tree, then the warps in
    // order: within 9 u of the CTA's exact sum of squares), then the last CTA
    // of the slot to finish adds the partials in a fixed order
    __shared__ double s_q[kMaxBlock / 32];
    __shared__ float s_qf[kMaxBlock / 32];
    __shared__ unsigned s_last;
    const float wq = warp_sum_f(qq);
    if (lane == 0) s_qf[threadIdx.x >> 5] = wq;
    __syncthreads();
    if (threadIdx.x == 0) {
        float cq = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) cq += s_qf[w];
        a.sb.qq_part[(int64_t)slot * a.sb.qq_stride + vb.x] = cq;
        __threadfence();
        const unsigned prev = atomicAdd(a.sb.counters + slot, 1u);
        s_last = prev == vb.gx - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // thread t adds partials t, t + blockDim.x, ... in order, error-free in
    // FP32 pairs; then a fixed FP64 tree over the threads
    TwoSumF tq, tg;
    for (int w = threadIdx.x; w < (int)vb.gx; w += blockDim.x)
        tq.add(__ldcg(a.sb.qq_part + (int64_t)slot * a.sb.qq_stride + w));
    for (int w = threadIdx.x; w < a.n_gg; w += blockDim.x)
        tg.add(__ldcg(a.sb.gg_part + (int64_t)slot * a.sb.gg_stride + w));
    const double qs = block_sum(tq.value(), s_q);
    const double gs = block_sum(tg.value(), s_q);
    if (threadIdx.x == 0) {
        // the exact line search (Eq. 'step'); mu = 0 when A g = 0
        double mu = qs > 0.0 ? sd.beta * gs / qs : 0.0;
        a.sb.mu[slot] = mu;
        // non-zeros of the step, counted by the backprojection
        unsigned long long nzs = atomicExch(a.sb.nnz_slot + slot, 0ull);
        atomicAdd(a.sb.nnz, nzs);
        if (sd.step >= 0 && sd.step < a.sb.hist_cap) {
            double* hrow = a.sb.hist + kHistCols * sd.step;
            hrow[0] = sd.beta;
            hrow[1] = gs;
            hrow[2] = qs;
            hrow[3] = mu;
            hrow[4] = (double)nzs;
        }
        a.sb.counters[slot] = 0u;
        if (a.sb.rmax) a.sb.rmax[slot] = 0u;  // read by the backprojection only
    }
}

template <int DIM, int L, bool TABLE>
__global__ void __maxnreg__(64) k_forward_dual(const FwdSolverArgs a) {
    forward_dual_body<DIM, L, TABLE, false>(a, hw_block());
}

// ---------------------------------------------------------------------------
// backprojection
// ---------------------------------------------------------------------------
// Ray table of a launch: every ray of every slot, set up once.  One CTA row per
// work item (view), so a thread knows its ray without searching.
struct TableArgs {
    DevGeom G;
    int j;               // tile of the launch
    int w_begin;         // first work item of the launch
    const float* r;
    RayRec* table;       // [slot][ray slot]
    int64_t slot_stride;
    unsigned* rmax;      // [slot] max |r| bits (k_slot_rmax)
};

// The first kTablePre rays of a thread are set up before waiting for the
// previous kernel (they need only the geometry); the residual is read and the
// records written after it.
constexpr int kTablePre = 4;

template <int DIM, bool EX>
__device__ __forceinline__ void ray_table_item(const TableArgs& a, const WorkItem& it,
                                               const VBlock& vb) {
    const DevGeom& G = a.G;
    const DevView V = G.views[it.view];
    const DevVT E = G.vt[(int64_t)it.view * G.n_tiles + a.j];
    const DevTile& tile = G.tiles[a.j];
    const int wu = it.u1 - it.u0;
    const int nr = wu * (it.v1 - it.v0);
    RayRec* dst = a.table + (int64_t)it.slot * a.slot_stride + it.ray_off;
    const int k0 = vb.y * blockDim.x + threadIdx.x;
    const int stride = vb.gy * blockDim.x;
    float pq[kTablePre][3], pi[kTablePre][3];
#pragma unroll
    for (int p = 0; p < kTablePre; ++p) {
        const int k = k0 + p * stride;
        if (k < nr)
            table_ray<DIM>(G, it.view, V, E, tile, it.u0 + k % wu, it.v0 + k / wu, pq[p], pi[p]);
    }
    pdl_wait();  // r and the table buffer belong to earlier kernels until here
#pragma unroll
    for (int p = 0; p < kTablePre; ++p) {
        const int k = k0 + p * stride;
        if (k < nr) {
            const int64_t ray = ray_index(G, it.view, it.u0 + k % wu, it.v0 + k / wu);
            const float rv = ldro<EX>(a.r + ray);
            *reinterpret_cast<float4*>(dst[k].a) = make_float4(pq[p][0], pq[p][1], pi[p][0], pi[p][1]);
            *reinterpret_cast<float4*>(dst[k].b) =
                make_float4(rv, pq[p][2], pi[p][2], __int_as_float((int)ray));
        }
    }
    for (int k = k0 + kTablePre * stride; k < nr; k += stride) {
        const int ku = it.u0 + k % wu;
        const int kv = it.v0 + k / wu;
        float q[3], inv[3];
        table_ray<DIM>(G, it.view, V, E, tile, ku, kv, q, inv);
        const int64_t ray = ray_index(G, it.view, ku, kv);
        const float rv = ldro<EX>(a.r + ray);
        *reinterpret_cast<float4*>(dst[k].a) = make_float4(q[0], q[1], inv[0], inv[1]);
        *reinterpret_cast<float4*>(dst[k].b) =
            make_float4(rv, q[2], inv[2], __int_as_float((int)ray));
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_ray_table_inline(const TableArgs a,
                                                          const __grid_constant__ InlineItems it) {
    ray_table_item<DIM, false>(a, it.items[blockIdx.x], hw_block());
}

template <int DIM, bool EX>
__device__ __forceinline__ void ray_table_body(const TableArgs& a, const WorkItem* items,
                                               const VBlock& vb) {
    pdl_trigger();
    const WorkItem it = items[a.w_begin + vb.x];
    ray_table_item<DIM, EX>(a, it, vb);
}

template <int DIM>
__global__ void __launch_bounds__(256) k_ray_table_solver(const TableArgs a,
                                                          const WorkItem* __restrict__ items) {
    ray_table_body<DIM, false>(a, items, hw_block());
}

// max |r| per slot over the rays of the batch's work items (the scatter's
// fixed-point scale when it sets its lines up itself): one CTA row per item.
__device__ __forceinline__ void slot_rmax_body(const TableArgs& a, const WorkItem* items,
                                               const VBlock& vb) {
    pdl_trigger();
    const WorkItem it = items[a.w_begin + vb.x];
    const DevGeom& G = a.G;
    const int wu = it.u1 - it.u0;
    const int nr = wu * (it.v1 - it.v0);
    pdl_wait();  // r belongs to earlier kernels until here
    float rm = 0.f;
    for (int k = vb.y * blockDim.x + threadIdx.x; k < nr; k += vb.gy * blockDim.x)
        rm = fmaxf(rm, fabsf(a.r[ray_index(G, it.view, it.u0 + k % wu, it.v0 + k / wu)]));
    // non-negative floats order like their bit patterns; the warps' maxima
    // meet in shared memory, so that the slot's word takes one atomic per CTA
    // (a slot's thousands of CTA rows would otherwise queue on one address)
    __shared__ unsigned s_m[kMaxBlock / 32];
    const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(rm));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_m[w]);
        if (m) atomicMax(a.rmax + it.slot, m);
    }
}

__global__ void __launch_bounds__(256) k_slot_rmax(const TableArgs a,
                                                   const WorkItem* __restrict__ items) {
    slot_rmax_body(a, items, hw_block());
}

struct BPArgs {
    DevGeom G;
    int first;
    const RayRec* table;   // [slot][ray slot]
    int64_t table_stride;
    const float* xt;       // mode 0: tile-major x, copied next to g
    float* gout;           // mode 0: (x_J, g_J) pairs per slot, tile-local; mode 1:
                           // row-major volume
    int mode;
    int accumulate;
    int64_t slot_stride;
    float* gg_part;        // [slot][voxel blocks] or null
    int gg_stride;
    unsigned long long* nnz_slot;  // [slot] non-zeros of the step, or null
};

// g_J = (A_I^J)^T r_I, voxel-driven: a thread owns one voxel of the tile and,
// for every view of its chunk, sums len * r over the rays whose bins lie within
// the voxel's shadow.  The length is the voxel's slab clip of the ray, t =
// (plane - q) / d on each face, i.e. the very crossings the forward walk
// evaluates, so forward and adjoint use the same lengths.  The ray table never
// holds a ray parallel to an axis whose q lies exactly on a face of that axis
// (see ray_table_item), so no crossing is 0 * inf and the clip needs no special
// case: a parallel ray's crossings are +-inf, which constrain nothing when q is
// inside the slab and empty the interval when it is outside.

// bins added on each side of a voxel's shadow window: covers the FP32 rounding
// of the window's centre, gradient and half-width
constexpr float kShadowMargin = 0.02f;
constexpr int kViewBatch = 96;
constexpr int kBPViewsPerPass = 2;  // 2D gather: views whose candidate loads are in flight together

// Per-view data of a 2D backprojection CTA, staged in shared memory: the bin
// coordinate of its 8 x 8 voxel patch, linearised about the patch centre Pc.
// For a voxel at Pc + d the candidate window is [w + g . d - h, w + g . d + h],
// where h covers the voxel's own shadow anywhere in the patch and the error of
// the linearisation (see stage_view).
struct alignas(16) ViewCtx2 {
    float w, g0, g1, h;  // bin coordinate of Pc minus 1/2, its gradient, half-width
    int u0, u1;          // bins of the work item
    int rbase;           // table position of bin 0 of the item
    int pad;
};

// Per-view data of a 3D backprojection CTA: the detector coordinates of its
// voxel patch, linearised about the patch centre Pc.  For a voxel at Pc + d the
// candidate window is [w + g . d - h, w + g . d + h] on each detector axis, where
// h covers the voxel's own shadow anywhere in the patch and the error of the
// linearisation (see stage_view).
struct alignas(16) ViewCtx3 {
    float wu, gu0, gu1, gu2;  // bin coordinate of Pc minus 1/2, and its gradient
    float wv, gv0, gv1, gv2;
    float hu, hv;             // window half-widths (bins)
    int u0, u1, v0, v1;       // bins of the work item
    int rbase;                // table position of bin (0, v0) of the item
    int pad[3];
};

template <int DIM>
struct ViewCtxOf { using type = ViewCtx3; };
template <>
struct ViewCtxOf<2> { using type = ViewCtx2; };

// 2D detector coordinate of a point P: parallel beam w = (P . e_u) / pitch,
// curved fan w = atan2(L, D) / pitch (the angle of r = P - S in the frame
// (d_c, e_u)), flat fan w = k L / D with k = sdd / pitch, L = r . e_u, D = r . d_c
// (e_u = (d_c1, -d_c0) in 2D).  Over the voxel centres of an 8 x 8 patch,
// |P - Pc| <= R = sqrt(2) 3.5; with Hm a bound of the Hessian's norm there
//   |w(P) - w(Pc) - g . (P - Pc)| <= Hm R^2 / 2,
//   the first-order half-width 0.5 sum_k |dw/dP_k| of a voxel is at most its
//   value at Pc plus 0.5 sqrt(2) Hm R,
//   and a voxel's shadow is within its first-order half-width times
//   (1 + 1.5 / depth) and within Hm / 4 (half diagonal^2 = 1/2) of it.
// Hm: 0 (parallel: w is linear); 1 / (pitch rho_min^2) for the angle (the
// Hessian of atan2 has norm 1 / |r|^2), rho_min = |r(Pc)| - R; k (2 / Dmin^2)
// (1 + (|L| + R) / Dmin) for the flat detector, Dmin = D(Pc) - R.
__device__ __forceinline__ void stage_view(const DevGeom& G, const DevTile&, const WorkItem& it,
                                           ViewCtx2* c, const float* Pc) {
    const DevView& V = G.views[it.view];
    const float R = 4.9497475f;  // sqrt(2) * 3.5
    const float wbase = fmaf(0.5f, (float)G.nu, -0.5f);
    const float dc0 = V.dc[0], dc1 = V.dc[1], e0 = dc1, e1 = -dc0;
    if (G.kind == PARALLEL_2D) {
        c->w = fmaf(Pc[0] * e0 + Pc[1] * e1, G.inv_pu, wbase);
        c->g0 = e0 * G.inv_pu;
        c->g1 = e1 * G.inv_pu;
        c->h = fmaf(0.5f * (fabsf(e0) + fabsf(e1)), G.inv_pu, kShadowMargin);
    } else {
        const float r0 = Pc[0] - V.S[0], r1 = Pc[1] - V.S[1];
        const float D = r0 * dc0 + r1 * dc1;
        const float L = r0 * e0 + r1 * e1;
        const float Dmin = D - R;
        if (Dmin > 1.0f) {
            float Hm;
            if (G.kind == FAN_2D_CURVED) {
                const float rho2 = D * D + L * L;
                const float rmin = sqrtf(rho2) - R;
                c->w = fmaf(atan2f(L, D), G.inv_pu, wbase);
                c->g0 = (D * e0 - L * dc0) / rho2 * G.inv_pu;
                c->g1 = (D * e1 - L * dc1) / rho2 * G.inv_pu;
                Hm = G.inv_pu / (rmin * rmin);
            } else {
                const float k = V.sdd * G.inv_pu, iD = 1.0f / D;
                c->w = fmaf(k * L, iD, wbase);
                c->g0 = k * (e0 * D - L * dc0) * iD * iD;
                c->g1 = k * (e1 * D - L * dc1) * iD * iD;
                Hm = k * 2.0f / (Dmin * Dmin) * (1.0f + (fabsf(L) + R) / Dmin);
            }
            const float h1 = 0.5f * (fabsf(c->g0) + fabsf(c->g1)) + 0.70710678f * Hm * R;
            c->h = h1 * (1.0f + 1.5f / Dmin) + 0.25f * Hm + 0.5f * Hm * R * R + kShadowMargin;
        } else {
            // the patch reaches the source: every bin of the item is a candidate
            c->w = c->g0 = c->g1 = 0.f;
            c->h = 1e30f;
        }
    }
    c->u0 = it.u0;
    c->u1 = it.u1;
    c->rbase = (int)it.ray_off - it.u0;
    c->pad = 0;
}

// Flat detector (cone beam, custom poses): w(P) = k L / D with D = r . d_c,
// L = r . e (e = e_u or e_v), r = P - S, k = sdd / pitch.  Its gradient is
// k (e D - L d_c) / D^2 and the norm of its Hessian is at most
// k (2 / D^2) (1 + |L| / D).  Over the voxel centres of a 4 x 4 x 4 patch,
// |P - Pc| <= rho = sqrt(3) 1.5, D >= Dmin = D(Pc) - rho and |L| / D <= T =
// (|L(Pc)| + rho) / Dmin, so with Hm = k (2 / Dmin^2) (1 + T):
//   |w(P) - w(Pc) - g . (P - Pc)| <= Hm rho^2 / 2,
//   the first-order half-width 0.5 sum_k |dw/dP_k| at P is at most its value
//   at Pc plus 0.5 sqrt(3) Hm rho,
//   and the second-order widening over a voxel (half diagonal^2 = 3/4) is at
//   most Hm 3/8.
// The window half-width adds these to the first-order half-width and the
// margin; any rounding here only widens or shifts the window by far less than
// the margin.
__device__ __forceinline__ void stage_flat_axis(float k, const float r[3], const float dc[3],
                                                const float e[3], float D, float Dmin, float rho,
                                                float wbase, float* w, float g[3], float* h) {
    const float L = r[0] * e[0] + r[1] * e[1] + r[2] * e[2];
    const float iD = 1.0f / D;
    *w = fmaf(k * L, iD, wbase);
    float h1 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g[a] = k * (e[a] * D - L * dc[a]) * iD * iD;
        h1 += fabsf(g[a]);
    }
    const float T = (fabsf(L) + rho) / Dmin;
    const float Hm = k * 2.0f / (Dmin * Dmin) * (1.0f + T);
    *h = 0.5f * h1 + 0.8660254f * Hm * rho + 0.5f * Hm * rho * rho + 0.375f * Hm + kShadowMargin;
}

__device__ __forceinline__ void stage_view(const DevGeom& G, const DevTile&, const WorkItem& it,
                                           ViewCtx3* c, const float Pc[3]) {
    const DevView& V = G.views[it.view];
    const float rho = 2.5980762f;  // sqrt(3) * 1.5
    float r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) r[a] = Pc[a] - V.S[a];
    const float D = r[0] * V.dc[0] + r[1] * V.dc[1] + r[2] * V.dc[2];
    const float Dmin = D - rho;
    float g[3];
    if (Dmin > 1.0f) {
        stage_flat_axis(V.sdd * G.inv_pu, r, V.dc, V.eu, D, Dmin, rho, fmaf(0.5f, (float)G.nu, -0.5f),
                        &c->wu, g, &c->hu);
        c->gu0 = g[0];
        c->gu1 = g[1];
        c->gu2 = g[2];
        stage_flat_axis(V.sdd * G.inv_pv, r, V.dc, V.ev, D, Dmin, rho, fmaf(0.5f, (float)G.nv, -0.5f),
                        &c->wv, g, &c->hv);
        c->gv0 = g[0];
        c->gv1 = g[1];
        c->gv2 = g[2];
    } else {
        // the patch reaches the source's plane: every bin of the item is a candidate
        c->wu = c->wv = 0.f;
        c->gu0 = c->gu1 = c->gu2 = c->gv0 = c->gv1 = c->gv2 = 0.f;
        c->hu = c->hv = 1e30f;
    }
    c->u0 = it.u0;
    c->u1 = it.u1;
    c->v0 = it.v0;
    c->v1 = it.v1;
    c->rbase = (int)it.ray_off - it.u0;
}

// Length of the unit voxel [lo, hi) on the line of a 2D table record.
__device__ __forceinline__ float slab2(const float4 a, const float lo[3], const float hi[3]) {
    const float ta0 = (lo[0] - a.x) * a.z, tb0 = (hi[0] - a.x) * a.z;
    const float ta1 = (lo[1] - a.y) * a.w, tb1 = (hi[1] - a.y) * a.w;
    const float tin = fmaxf(fminf(ta0, tb0), fminf(ta1, tb1));
    const float tout = fminf(fmaxf(ta0, tb0), fmaxf(ta1, tb1));
    return fmaxf(tout - tin, 0.f);
}

__device__ __forceinline__ float slab3(const float4 a, const float4 b, const float lo[3],
                                       const float hi[3]) {
    const float ta0 = (lo[0] - a.x) * a.z, tb0 = (hi[0] - a.x) * a.z;
    const float ta1 = (lo[1] - a.y) * a.w, tb1 = (hi[1] - a.y) * a.w;
    const float ta2 = (lo[2] - b.y) * b.z, tb2 = (hi[2] - b.y) * b.z;
    const float tin = fmaxf(fmaxf(fminf(ta0, tb0), fminf(ta1, tb1)), fminf(ta2, tb2));
    const float tout = fminf(fminf(fmaxf(ta0, tb0), fmaxf(ta1, tb1)), fmaxf(ta2, tb2));
    return fmaxf(tout - tin, 0.f);
}

__device__ __forceinline__ float4 rec_a(const RayRec* p) {
    return *reinterpret_cast<const float4*>(p->a);
}
__device__ __forceinline__ float4 rec_b(const RayRec* p) {
    return *reinterpret_cast<const float4*>(p->b);
}

// Candidate bins of one voxel in one view (2D), with the records of the first
// two already requested.
struct Cand2 {
    float4 a0, a1;
    float rA, rB;
    int ku0, ku1;
    const RayRec* row;
};

__device__ __forceinline__ Cand2 view_cands(const ViewCtx2& c, float dx, float dy,
                                            const RayRec* __restrict__ tab) {
    const float wu = fmaf(c.g1, dy, fmaf(c.g0, dx, c.w));
    const float hu = c.h;
    Cand2 k;
    k.ku0 = max(c.u0, __float2int_ru(fmaxf(wu - hu, -1e9f)));
    k.ku1 = min(c.u1 - 1, __float2int_rd(fminf(wu + hu, 1e9f)));
    k.row = tab + c.rbase;
    // The first two candidates without branches (most voxels have one or two,
    // and lanes of a warp differ): both records are loaded from bins clamped
    // into the item and the residual of a bin outside the window is zeroed.
    const int kA = min(k.ku0, c.u1 - 1);
    const int kB = min(kA + 1, c.u1 - 1);
    k.a0 = rec_a(k.row + kA);
    k.a1 = rec_a(k.row + kB);
    const float rA = k.row[kA].b[0], rB = k.row[kB].b[0];
    k.rA = k.ku0 <= k.ku1 ? rA : 0.f;
    k.rB = k.ku0 < k.ku1 ? rB : 0.f;
    return k;
}

// sum over the candidate bins of len * r for one voxel (2D); nz counts the
// candidates with a positive length (the non-zeros A_iv of the block)
__device__ __forceinline__ float cand_sum(const Cand2& k, const float lo[3], const float hi[3],
                                          int& nz) {
    const float lA = slab2(k.a0, lo, hi), lB = slab2(k.a1, lo, hi);
    nz += (lA > 0.f && k.ku0 <= k.ku1) + (lB > 0.f && k.ku0 < k.ku1);
    float s = fmaf(lA, k.rA, 0.f);
    s = fmaf(lB, k.rB, s);
    for (int ku = k.ku0 + 2; ku <= k.ku1; ++ku) {
        const float l = slab2(rec_a(k.row + ku), lo, hi);
        nz += l > 0.f;
        s = fmaf(l, k.row[ku].b[0], s);
    }
    return s;
}

// sum over the view's candidate bins of len * r for one voxel (3D), d = P - Pc;
// nz counts the candidates with a positive length
__device__ __forceinline__ float view_sum(const DevGeom&, const ViewCtx3& c, const float d[3],
                                          const float lo[3], const float hi[3],
                                          const RayRec* __restrict__ tab, int& nz) {
    const float wu = fmaf(c.gu2, d[2], fmaf(c.gu1, d[1], fmaf(c.gu0, d[0], c.wu)));
    const float wv = fmaf(c.gv2, d[2], fmaf(c.gv1, d[1], fmaf(c.gv0, d[0], c.wv)));
    const int ku0 = max(c.u0, __float2int_ru(fmaxf(wu - c.hu, -1e9f)));
    const int ku1 = min(c.u1 - 1, __float2int_rd(fminf(wu + c.hu, 1e9f)));
    const int kv0 = max(c.v0, __float2int_ru(fmaxf(wv - c.hv, -1e9f)));
    const int kv1 = min(c.v1 - 1, __float2int_rd(fminf(wv + c.hv, 1e9f)));
    const int wdt = c.u1 - c.u0;
    const RayRec* base = tab + c.rbase - c.v0 * wdt;  // + kv * wdt + ku
    // the first 2 x 2 candidates without branches (bins clamped into the item,
    // residuals outside the window zeroed), the rest in loops (rare)
    const int kA = min(ku0, c.u1 - 1), kB = min(kA + 1, c.u1 - 1);
    const int vA = min(kv0, c.v1 - 1), vB = min(vA + 1, c.v1 - 1);
    const bool uA = ku0 <= ku1, uB = ku0 < ku1, wA = kv0 <= kv1, wB = kv0 < kv1;
    const RayRec* p00 = base + vA * wdt + kA;
    const RayRec* p01 = base + vA * wdt + kB;
    const RayRec* p10 = base + vB * wdt + kA;
    const RayRec* p11 = base + vB * wdt + kB;
    const float4 a00 = rec_a(p00), b00 = rec_b(p00), a01 = rec_a(p01), b01 = rec_b(p01);
    const float4 a10 = rec_a(p10), b10 = rec_b(p10), a11 = rec_a(p11), b11 = rec_b(p11);
    const float l00 = slab3(a00, b00, lo, hi), l01 = slab3(a01, b01, lo, hi);
    const float l10 = slab3(a10, b10, lo, hi), l11 = slab3(a11, b11, lo, hi);
    nz += (l00 > 0.f && uA && wA) + (l01 > 0.f && uB && wA) + (l10 > 0.f && uA && wB) +
          (l11 > 0.f && uB && wB);
    float s = fmaf(l00, uA && wA ? b00.x : 0.f, 0.f);
    s = fmaf(l01, uB && wA ? b01.x : 0.f, s);
    s = fmaf(l10, uA && wB ? b10.x : 0.f, s);
    s = fmaf(l11, uB && wB ? b11.x : 0.f, s);
    if (ku1 - ku0 >= 2 || kv1 - kv0 >= 2) {  // candidates beyond the 2 x 2 block
        for (int kv = kv0; kv <= kv1; ++kv) {
            const RayRec* row = base + kv * wdt;
            for (int ku = (kv < kv0 + 2 ? ku0 + 2 : ku0); ku <= ku1; ++ku) {
                const RayRec* rp = row + ku;
                const float4 b = rec_b(rp);
                const float l = slab3(rec_a(rp), b, lo, hi);
                nz += l > 0.f;
                s = fmaf(l, b.x, s);
            }
        }
    }
    return s;
}

// A backprojection CTA owns a patch of kBPVox voxels of the tile and splits the
// views of its slot among C = blockDim.x / kBPVox thread groups (view i goes to group
// i mod C); the C partial sums of a voxel are added in shared memory in group
// order.  C is chosen per launch so that the grid fills whole waves.
template <int DIM>
__device__ __forceinline__ void backproject_body(const BPArgs& a, const WorkItem* items,
                                                 const StepDesc& sd, int slot, unsigned patch) {
    using Ctx = typename ViewCtxOf<DIM>::type;
    __shared__ float part[kBPMaxThreads];
    __shared__ Ctx vs[kViewBatch];
    const DevGeom& G = a.G;
    const int C = (int)blockDim.x / kBPVox;
    const int chunk = (int)threadIdx.x / kBPVox;
    const int lv = (int)threadIdx.x % kBPVox;
    const DevTile t = G.tiles[sd.j];
    // the CTA's patch of the tile (patches tile it in x-fastest order) and this
    // thread's voxel in it: a compact patch shares candidate rays among its voxels
    constexpr int P0 = DIM == 2 ? 8 : 4, P1 = DIM == 2 ? 8 : 4;
    const int nb0 = (t.n[0] + P0 - 1) / P0, nb1 = (t.n[1] + P1 - 1) / P1;
    const int b0 = patch % nb0, b12 = patch / nb0;
    const int x0 = b0 * P0 + lv % P0;
    const int x1 = (b12 % nb1) * P1 + (lv / P0) % P1;
    const int x2 = DIM == 3 ? (b12 / nb1) * 4 + lv / (P0 * P1) : 0;
    const bool valid = x0 < t.n[0] && x1 < t.n[1] && x2 < t.n[2];
    const int v = (x2 * t.n[1] + x1) * t.n[0] + x0;  // tile-local voxel index
    // patch centre (grid-centred voxel units) and this voxel's offset from it
    const float Pc[3] = {-0.5f * (float)t.n[0] + (float)(b0 * P0) + 0.5f * P0 + t.T[0],
                         -0.5f * (float)t.n[1] + (float)((b12 % nb1) * P1) + 0.5f * P1 + t.T[1],
                         DIM == 3 ? -0.5f * (float)t.n[2] + (float)((b12 / nb1) * 4) + 2.0f + t.T[2]
                                  : 0.f};
    const float dP[3] = {(float)(lv % P0) - 0.5f * (P0 - 1), (float)((lv / P0) % P1) - 0.5f * (P1 - 1),
                         DIM == 3 ? (float)(lv / (P0 * P1)) - 1.5f : 0.f};
    // voxel box [lo, hi) in tile-centred coordinates, centre P
    float lo[3], hi[3], P[3];
    lo[0] = -0.5f * (float)t.n[0] + (float)x0;
    lo[1] = -0.5f * (float)t.n[1] + (float)x1;
    lo[2] = DIM == 3 ? -0.5f * (float)t.n[2] + (float)x2 : -0.5f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        hi[c] = lo[c] + 1.0f;
        P[c] = c < DIM ? t.T[c] + lo[c] + 0.5f : 0.f;
    }
    const RayRec* __restrict__ tab = a.table + (int64_t)slot * a.table_stride;
    const int n_items = sd.w1 - sd.w0;
    Kahan acc;
    int nz = 0;  // candidates of this voxel with a positive length
    for (int base = 0; base < n_items; base += kViewBatch) {
        const int nb = min(kViewBatch, n_items - base);
        __syncthreads();
        for (int k = threadIdx.x; k < nb; k += blockDim.x)
            stage_view(G, t, items[sd.w0 + base + k], &vs[k], Pc);
        __syncthreads();
        if (base == 0) pdl_wait();  // the ray table is the previous kernel's
        if (!valid) continue;
        if constexpr (DIM == 2) {
            // kBPViewsPerPass views per pass: the records of all of them are
            // requested before any length is computed
            constexpr int V = kBPViewsPerPass;
            int i = chunk;
            for (; i + (V - 1) * C < nb; i += V * C) {
                Cand2 k[V];
#pragma unroll
                for (int u = 0; u < V; ++u) k[u] = view_cands(vs[i + u * C], dP[0], dP[1], tab);
#pragma unroll
                for (int u = 0; u < V; ++u) acc.add(cand_sum(k[u], lo, hi, nz));
            }
            for (; i < nb; i += C)
                acc.add(cand_sum(view_cands(vs[i], dP[0], dP[1], tab), lo, hi, nz));
        } else {
            for (int i = chunk; i < nb; i += C) acc.add(view_sum(G, vs[i], dP, lo, hi, tab, nz));
        }
    }
    if (n_items <= 0) pdl_wait();
    part[threadIdx.x] = acc.s - acc.c;
    __syncthreads();
    float gg = 0.f;
    if (chunk == 0 && valid) {
        float s = 0.f;
        for (int c = 0; c < C; ++c) s += part[c * kBPVox + lv];
        s *= G.h;
        if (a.mode == 0) {
            reinterpret_cast<float2*>(a.gout)[(int64_t)slot * a.slot_stride + v] =
                make_float2(a.xt[t.voff + v], s);
        } else {
            int64_t gi = ((int64_t)(t.lo[2] + x2) * G.ny + (t.lo[1] + x1)) * G.nx + t.lo[0] + x0;
            a.gout[gi] = a.accumulate ? a.gout[gi] + s : s;
        }
        gg = s * s;
    }
    // The CTA's g^T g partial in FP32 (a warp tree, then the warps in order:
    // within 13 u of its exact value); and nnz(A_I^J) of the
    // step: each (voxel, ray) pair is clipped by exactly one thread, with the
    // lengths the forward walk uses.
    __shared__ float s_gg[kBPMaxThreads / 32];
    __shared__ unsigned s_nz[kBPMaxThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (a.gg_part) {
        const float wg = warp_sum_f(gg);
        if (lane == 0) s_gg[w] = wg;
    }
    if (a.nnz_slot) {
        const unsigned wn = __reduce_add_sync(0xffffffffu, (unsigned)nz);
        if (lane == 0) s_nz[w] = wn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)(blockDim.x >> 5);
        if (a.gg_part) {
            float cg = 0.f;
            for (int k = 0; k < nw; ++k) cg += s_gg[k];
            a.gg_part[(int64_t)slot * a.gg_stride + patch] = cg;
        }
        if (a.nnz_slot) {
            unsigned long long cn = 0;
            for (int k = 0; k < nw; ++k) cn += s_nz[k];
            if (cn) atomicAdd(a.nnz_slot + slot, cn);
        }
    }
}

template <int DIM>
__global__ void __maxnreg__(64) k_backproject_inline(
    const BPArgs a, const __grid_constant__ InlineItems it) {
    backproject_body<DIM>(a, it.items, it.step, 0, blockIdx.x);
}

template <int DIM>
__device__ __forceinline__ void backproject_solver_body(const BPArgs& a, const WorkItem* items,
                                                        const StepDesc* steps, const VBlock& vb) {
    pdl_trigger();
    const StepDesc sd = steps[a.first + vb.z];
    backproject_body<DIM>(a, items, sd, vb.z, vb.x);
}

template <int DIM>
__global__ void __maxnreg__(64) k_backproject_solver(
    const BPArgs a, const WorkItem* __restrict__ items, const StepDesc* __restrict__ steps) {
    backproject_solver_body<DIM>(a, items, steps, hw_block());
}

// ---------------------------------------------------------------------------
// Ray-driven backprojection (scatter).  Every ray of a slot walks the tile as
// in the dual forward (same crossings, so the same lengths) and adds len * r_i
// to a 32-bit fixed-point accumulator of its voxel with an integer atomic: the
// sum of the slot's FP32 products len * r_i is then exact (below the fixed
// point's resolution) and independent of the order of the additions, so the
// result is deterministic.  A conversion pass turns the accumulator into the
// (x_J, g_J) pairs and the g^T g partials and clears it.  Which of the two
// backprojections is faster depends on the geometry: the gather evaluates
// every candidate line of a voxel's window, the scatter only the crossings.
// ---------------------------------------------------------------------------
struct ScatterArgs {
    DevGeom G;
    const WorkItem* items;
    const StepDesc* steps;
    int first;
    float lane_factor;  // 2 when the lanes of a line may split its segment in a voxel
    SolverBuffers sb;
};

// Fixed-point exponent S of a slot (term = round(2^S * len * r)): a line
// crosses a unit voxel over at most sqrt(3) < 2, so a term is below
// 2 max|r| 2^S, and a voxel receives at most `terms` of them (twice that when
// the lanes of a line can split its segment in a voxel), so with
// terms 2 max|r| < 2^e and S = 30 - e every sum stays below 2^30 and fits the
// 32-bit accumulator.  The resolution, 2^-S, is about 2 terms max|r| 2^-30:
// far below FP32 rounding of the sum for the tens to hundreds of terms a
// step's views put into one voxel.
__device__ __forceinline__ int scatter_shift(unsigned rmax_bits, float terms) {
    const float bound = __uint_as_float(rmax_bits) * 2.0f * fmaxf(1.0f, terms);
    int e = 0;
    frexpf(bound, &e);  // bound < 2^e (e = 0 for bound = 0)
    return min(100, max(-100, 30 - e));
}

// 2^k as a float, k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

template <int DIM, int L>
__device__ __forceinline__ void scatter_body(const ScatterArgs& a, const VBlock& vb) {
    pdl_trigger();
    const DevGeom& G = a.G;
    const int slot = vb.y;
    const StepDesc sd = a.steps[a.first + slot];
    const DevTile t = G.tiles[sd.j];
    const int nvox = t.n[0] * t.n[1] * t.n[2];
    const int64_t gid = (int64_t)vb.x * blockDim.x + threadIdx.x;
    const int64_t k = gid / L;
    const int sub = (int)(gid % L);
    const bool active = k < sd.n_rays;
    float q[3], inv[3];
    int ray = 0;
    // the line set up here, before the wait (geometry only), as the dual
    // forward sets it up
    if (active) {
        const int w = find_item(a.items, sd.w0, sd.w1, k);
        const WorkItem it = a.items[w];
        const int within = (int)(k - it.ray_off);
        const int wu = it.u1 - it.u0;
        const int ku = it.u0 + within % wu, kv = it.v0 + within / wu;
        table_ray<DIM>(G, it.view, G.views[it.view], G.vt[(int64_t)it.view * G.n_tiles + sd.j],
                       t, ku, kv, q, inv);
        ray = (int)ray_index(G, it.view, ku, kv);
    }
    pdl_wait();  // r and the slot's max |r| come from earlier kernels
    int* __restrict__ acc = reinterpret_cast<int*>(a.sb.acc) + (int64_t)slot * a.sb.g_stride;
    const float sc = pow2f(scatter_shift(a.sb.rmax[slot], sd.terms * a.lane_factor));
    int nz = 0;
    int first_id = -1, last_id = -1;  // voxels of the lane's first and last non-zero
    if (active) {
        const float rs = __ldcg(a.sb.r + ray) * sc;  // (len * r) * 2^S rounds as len * (r * 2^S)
        Box b = tile_box(t, DIM, 0, t.n[0], t.n[0] * t.n[1]);
        float tin, tout;
        if (clip<DIM>(q, inv, b, &tin, &tout)) {
            const float dt = (tout - tin) * (1.0f / L);
            const float t0 = sub == 0 ? tin : fmaf((float)sub, dt, tin);
            const float t1 = sub == L - 1 ? tout : fmaf((float)(sub + 1), dt, tin);
            auto batch = [&](const int (&id)[kFwdBatch], const float (&ln)[kFwdBatch]) {
#pragma unroll
                for (int u = 0; u < kFwdBatch; ++u) {
                    if (ln[u] > 0.f) {
                        ++nz;
                        first_id = first_id < 0 ? id[u] : first_id;
                        last_id = id[u];
                        const int term = __float2int_rn(ln[u] * rs);
                        if (term && (unsigned)id[u] < (unsigned)nvox) atomicAdd(acc + id[u], term);
                    }
                }
            };
            if constexpr (DIM == 2) walk2_batched<kFwdBatch>(q, inv, b, t0, t1, batch);
            else walk3_batched<kFwdBatch>(q, inv, b, t0, t1, batch);
        }
    }
    if constexpr (L > 1) {
        // a lane boundary inside a voxel splits its segment between two lanes:
        // count that non-zero once (the L lanes of a ray are consecutive lanes
        // of one warp; a boundary on a voxel face leaves two different voxels)
        const int prev_last = __shfl_up_sync(0xffffffffu, last_id, 1);
        if (sub > 0 && first_id >= 0 && first_id == prev_last) --nz;
    }
    if (a.sb.nnz_slot) {
        __shared__ unsigned s_nz[kMaxBlock / 32];
        const unsigned wn = __reduce_add_sync(0xffffffffu, (unsigned)nz);
        if ((threadIdx.x & 31) == 0) s_nz[threadIdx.x >> 5] = wn;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long cn = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) cn += s_nz[w];
            if (cn) atomicAdd(a.sb.nnz_slot + slot, cn);
        }
    }
}

template <int DIM, int L>
__global__ void __maxnreg__(64) k_backproject_scatter(const ScatterArgs a) {
    scatter_body<DIM, L>(a, hw_block());
}

constexpr int kConvThreads = 256;
constexpr int kConvPerThread = 4;  // voxels per thread, kConvThreads apart

// CTAs of the conversion pass for a tile of tv voxels (one g^T g partial each)
static inline int conv_blocks(int64_t tv) {
    const int64_t per = (int64_t)kConvThreads * kConvPerThread;
    return (int)std::max<int64_t>(1, (tv + per - 1) / per);
}

// g_J = h 2^-S acc (one rounding from the exact fixed-point sum), the pairs
// (x_J, g_J) for the dual forward, a g^T g partial per CTA (FP32 as in the
// gather), and acc cleared for the next batch.
__device__ __forceinline__ void scatter_convert_body(const ScatterArgs& a, const VBlock& vb) {
    pdl_trigger();
    const DevGeom& G = a.G;
    const int slot = vb.y;
    const StepDesc sd = a.steps[a.first + slot];
    const DevTile t = G.tiles[sd.j];
    const int nvox = t.n[0] * t.n[1] * t.n[2];
    pdl_wait();
    // the same exponent as the scatter's (same bound, same lane factor)
    const float isc = pow2f(-scatter_shift(a.sb.rmax[slot], sd.terms * a.lane_factor));
    int* acc = reinterpret_cast<int*>(a.sb.acc) + (int64_t)slot * a.sb.g_stride;
    float2* gout = reinterpret_cast<float2*>(a.sb.g) + (int64_t)slot * a.sb.g_stride;
    const float* xt = a.sb.x + t.voff;
    float gg = 0.f;
    // kConvPerThread voxels a thread, their loads issued together
    const int span = blockDim.x * kConvPerThread;
    for (int v0 = vb.x * span + threadIdx.x; v0 < nvox; v0 += vb.gx * span) {
        int s[kConvPerThread];
        float xv[kConvPerThread];
#pragma unroll
        for (int k = 0; k < kConvPerThread; ++k) {
            const int v = v0 + k * blockDim.x;
            s[k] = 0;
            xv[k] = 0.f;
            if (v < nvox) {
                s[k] = __ldcg(acc + v);  // summed by L2 atomics
                xv[k] = xt[v];
            }
        }
#pragma unroll
        for (int k = 0; k < kConvPerThread; ++k) {
            const int v = v0 + k * blockDim.x;
            if (v < nvox) {
                acc[v] = 0;
                const float g = (float)s[k] * isc * G.h;
                gout[v] = make_float2(xv[k], g);
                gg = fmaf(g, g, gg);
            }
        }
    }
    __shared__ float s_gg[kMaxBlock / 32];
    const float wg = warp_sum_f(gg);
    if ((threadIdx.x & 31) == 0) s_gg[threadIdx.x >> 5] = wg;
    __syncthreads();
    if (threadIdx.x == 0) {
        float cg = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) cg += s_gg[w];
        a.sb.gg_part[(int64_t)slot * a.sb.gg_stride + vb.x] = cg;
    }
}

__global__ void __launch_bounds__(kConvThreads) k_scatter_convert(const ScatterArgs a) {
    scatter_convert_body(a, hw_block());
}

// ---------------------------------------------------------------------------
// Backprojection by bricks.  A CTA owns one brick of the tile (16^3 voxels in
// 3D, 32^2 in 2D) for one slot and sums len * r over the slot's lines that
// cross it, in shared memory.  For every view of the slot it takes the bins of
// the work item whose centre lines can cross the brick (the bounding rectangle
// of the projections of the brick's corners, i.e. of its shadow), sets each
// line up exactly as the dual forward does (table_ray: the same q and 1/d, the
// same treatment of lines that only touch the tile), clips it to the brick and
// walks it there.  Plane crossings are the forward's, so every (line, voxel)
// length is the forward's, and each such pair lies in exactly one brick.
// Terms round(2^S len r) go to 32-bit fixed-point sums with shared-memory
// integer atomics: the sums are exact and do not depend on the order of the
// additions, so the result is deterministic.  S is chosen per CTA from the
// largest |r| it reads and a bound on the lines one voxel can receive (per
// view, the bins within hw_u, hw_v of the voxel's centre), so that no sum can
// overflow.  No ray table, no global atomics, no conversion pass.
// ---------------------------------------------------------------------------
// Brick shapes, by dimension and shape index SH (the autotuner picks one):
// 3D 16 x 16 x {16, 8, 4}; 2D {32, 16, 8} squared.  Thinner bricks give more
// CTAs per slot and smaller windows, at more line set-ups per line.
template <int DIM, int SH>
struct BrickShape {
    static constexpr int n0 = 16, n1 = 16, n2 = SH == 0 ? 16 : (SH == 1 ? 8 : 4);
};
template <int SH>
struct BrickShape<2, SH> {
    static constexpr int n0 = SH == 0 ? 32 : (SH == 1 ? 16 : 8), n1 = n0, n2 = 1;
};
constexpr int kBrickThreads = 256;
constexpr int kBrickViews = 64;  // views staged in shared memory at a time

struct BrickView {
    int u0, nu;   // bins [u0, u0 + nu) x [v0, v0 + nv) of the item that can cross the brick
    int v0, nv;
    int start;    // (view, bin) pairs of the staged views before this one
    int view;
    int terms;    // bound on this view's lines through one voxel
    int pad;
};

struct BrickArgs {
    DevGeom G;
    const WorkItem* items;
    const StepDesc* steps;
    int first;
    const float* r;
    SolverBuffers sb;
};

template <int DIM, int SH>
inline int brick_count_of(const DevTile& t) {
    using BS = BrickShape<DIM, SH>;
    return ((t.n[0] + BS::n0 - 1) / BS::n0) * ((t.n[1] + BS::n1 - 1) / BS::n1) *
           ((t.n[2] + BS::n2 - 1) / BS::n2);
}
inline int brick_count(const DevTile& t, int dim, int sh) {
    if (dim == 2) return sh == 0 ? brick_count_of<2, 0>(t) : (sh == 1 ? brick_count_of<2, 1>(t)
                                                                        : brick_count_of<2, 2>(t));
    return sh == 0 ? brick_count_of<3, 0>(t) : (sh == 1 ? brick_count_of<3, 1>(t)
                                                         : brick_count_of<3, 2>(t));
}

// Detector coordinates (bin index units: bin k's centre at w = k) of a point P
// (grid-centred voxel units) in view V; false if P is not in front of the source.
__device__ __forceinline__ bool det_coord(const DevGeom& G, const DevView& V, const float P[3],
                                          float* wu, float* wv) {
    const float bu = fmaf(0.5f, (float)G.nu, -0.5f), bv = fmaf(0.5f, (float)G.nv, -0.5f);
    if (G.kind == PARALLEL_2D) {
        *wu = fmaf(P[0] * V.eu[0] + P[1] * V.eu[1], G.inv_pu, bu);
        *wv = 0.f;
        return true;
    }
    float r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) r[a] = P[a] - V.S[a];
    const float D = r[0] * V.dc[0] + r[1] * V.dc[1] + r[2] * V.dc[2];
    if (!(D > 1e-3f)) return false;
    const float Lu = r[0] * V.eu[0] + r[1] * V.eu[1] + r[2] * V.eu[2];
    if (G.kind == FAN_2D_CURVED) {
        *wu = fmaf(atan2f(Lu, D), G.inv_pu, bu);
        *wv = 0.f;
        return true;
    }
    const float iD = V.sdd / D;
    *wu = fmaf(Lu * iD, G.inv_pu, bu);
    const float Lv = r[0] * V.ev[0] + r[1] * V.ev[1] + r[2] * V.ev[2];
    *wv = G.dim == 3 ? fmaf(Lv * iD, G.inv_pv, bv) : 0.f;
    return true;
}

// Window of the item's bins whose centre lines can cross the brick [blo, bhi)
// (grid-centred voxel units): the bounding rectangle of its corners' detector
// coordinates, widened by kShadowMargin for rounding.
template <int DIM>
__device__ __forceinline__ void brick_window(const DevGeom& G, const DevView& V, const WorkItem& it,
                                             const float blo[3], const float bhi[3],
                                             BrickView* bv) {
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    bool all = false;
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? 8 : 4); ++c) {
        const float P[3] = {(c & 1) ? bhi[0] : blo[0], (c & 2) ? bhi[1] : blo[1],
                            DIM == 3 ? ((c & 4) ? bhi[2] : blo[2]) : 0.f};
        float wu, wv;
        if (!det_coord(G, V, P, &wu, &wv)) all = true;
        umin = fminf(umin, wu);
        umax = fmaxf(umax, wu);
        vmin = fminf(vmin, wv);
        vmax = fmaxf(vmax, wv);
    }
    int u0 = it.u0, u1 = it.u1, v0 = it.v0, v1 = it.v1;
    if (!all) {
        u0 = max(u0, __float2int_ru(fmaxf(umin - kShadowMargin, -1e9f)));
        u1 = min(u1, __float2int_rd(fminf(umax + kShadowMargin, 1e9f)) + 1);
        if (DIM == 3) {
            v0 = max(v0, __float2int_ru(fmaxf(vmin - kShadowMargin, -1e9f)));
            v1 = min(v1, __float2int_rd(fminf(vmax + kShadowMargin, 1e9f)) + 1);
        }
    }
    bv->u0 = u0;
    bv->nu = max(0, u1 - u0);
    bv->v0 = v0;
    bv->nv = max(0, v1 - v0);
}

template <int DIM, int SH>
__global__ void __launch_bounds__(kBrickThreads, 4) k_backproject_brick(const BrickArgs a) {
    using BS = BrickShape<DIM, SH>;
    constexpr int kVox = BS::n0 * BS::n1 * BS::n2;
    __shared__ int acc[kVox];
    __shared__ BrickView sv[kBrickViews];
    __shared__ DevView sview[kBrickViews];
    __shared__ DevVT svt[kBrickViews];
    __shared__ float s_red[kBrickThreads / 32];
    __shared__ unsigned s_nz[kBrickThreads / 32];
    __shared__ float s_terms;  // bound on the terms one voxel receives (all views)
    __shared__ int s_total;
    pdl_trigger();
    const DevGeom& G = a.G;
    const int slot = blockIdx.y;
    const StepDesc sd = a.steps[a.first + slot];
    const DevTile t = G.tiles[sd.j];
    // this CTA's brick: voxels [b_lo, b_lo + bn) of the tile
    const int nb0 = (t.n[0] + BS::n0 - 1) / BS::n0, nb1 = (t.n[1] + BS::n1 - 1) / BS::n1;
    const int bidx[3] = {(int)blockIdx.x % nb0, ((int)blockIdx.x / nb0) % nb1,
                         (int)blockIdx.x / (nb0 * nb1)};
    const int b_lo[3] = {bidx[0] * BS::n0, bidx[1] * BS::n1, bidx[2] * BS::n2};
    const int bn[3] = {min(BS::n0, t.n[0] - b_lo[0]), min(BS::n1, t.n[1] - b_lo[1]),
                       DIM == 3 ? min(BS::n2, t.n[2] - b_lo[2]) : 1};
    Box bb;
    float blo[3], bhi[3];  // grid-centred
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        bb.lo[c] = c < DIM ? -0.5f * (float)t.n[c] + (float)b_lo[c] : -0.5f;
        bb.n[c] = bn[c];
        blo[c] = c < DIM ? t.T[c] + bb.lo[c] : 0.f;
        bhi[c] = c < DIM ? blo[c] + (float)bn[c] : 0.f;
    }
    bb.stride[0] = 1;
    bb.stride[1] = bn[0];
    bb.stride[2] = bn[0] * bn[1];
    bb.base = 0;
    const int nvox = bn[0] * bn[1] * bn[2];
    for (int v = threadIdx.x; v < kVox; v += blockDim.x) acc[v] = 0;
    const int n_items = sd.w1 - sd.w0;
    // stage views [base, base + nb): windows, frames and constants, prefix counts
    auto stage = [&](int base, int nb) {
        __syncthreads();
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const WorkItem it = a.items[sd.w0 + base + k];
            sview[k] = G.views[it.view];
            svt[k] = G.vt[(int64_t)it.view * G.n_tiles + sd.j];
            brick_window<DIM>(G, sview[k], it, blo, bhi, &sv[k]);
            sv[k].view = it.view;
            const int tu = (int)fminf(2.0f * svt[k].hw_u, 4096.f) + 2;
            const int tv = DIM == 3 ? (int)fminf(2.0f * svt[k].hw_v, 4096.f) + 2 : 1;
            sv[k].terms = tu * tv;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            float terms = 0.f;
            for (int k = 0; k < nb; ++k) {
                sv[k].start = run;
                run += sv[k].nu * sv[k].nv;
                terms += (float)sv[k].terms;
            }
            s_total = run;
            s_terms += terms;
        }
        __syncthreads();
    };
    if (threadIdx.x == 0) s_terms = 0.f;
    // pass 1: the largest |r| of the CTA's lines
    float rm = 0.f;
    for (int base = 0; base < n_items; base += kBrickViews) {
        const int nb = min(kBrickViews, n_items - base);
        stage(base, nb);
        if (base == 0) pdl_wait();  // r is the previous kernels'
        int vi = 0;
        for (int k = threadIdx.x; k < s_total; k += blockDim.x) {
            while (vi + 1 < nb && k >= sv[vi + 1].start) ++vi;
            const BrickView& w = sv[vi];
            const int kk = k - w.start;
            const int ku = w.u0 + kk % w.nu, kv = w.v0 + kk / w.nu;
            rm = fmaxf(rm, fabsf(__ldg(a.r + ray_index(G, w.view, ku, kv))));
        }
    }
    if (n_items <= 0) pdl_wait();
    {
        const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(rm));
        if ((threadIdx.x & 31) == 0) s_nz[threadIdx.x >> 5] = wm;
    }
    __syncthreads();
    unsigned mbits = 0;
    for (int w = 0; w < kBrickThreads / 32; ++w) mbits = max(mbits, s_nz[w]);
    // every voxel receives at most s_terms terms, each below 2 max|r| 2^S (a unit
    // voxel's chord is at most sqrt(3)), so sums stay below 2^30 when
    // s_terms 2 max|r| < 2^(30 - S)
    const float bound = __uint_as_float(mbits) * 2.0f * fmaxf(1.f, s_terms);
    int e = 0;
    frexpf(bound, &e);  // bound < 2^e
    const int S = min(100, max(-100, 30 - e));
    const float sc = pow2f(S);
    // pass 2: walk every line through the brick
    int nz = 0;
    for (int base = 0; base < n_items; base += kBrickViews) {
        const int nb = min(kBrickViews, n_items - base);
        if (n_items > kBrickViews) stage(base, nb);
        int vi = 0;
        for (int k = threadIdx.x; k < s_total; k += blockDim.x) {
            while (vi + 1 < nb && k >= sv[vi + 1].start) ++vi;
            const BrickView& w = sv[vi];
            const int kk = k - w.start;
            const int ku = w.u0 + kk % w.nu, kv = w.v0 + kk / w.nu;
            const float rs = __ldg(a.r + ray_index(G, w.view, ku, kv)) * sc;
            float q[3], inv[3];
            table_ray<DIM>(G, w.view, sview[vi], svt[vi], t, ku, kv, q, inv);
            float tin, tout;
            if (!clip<DIM>(q, inv, bb, &tin, &tout)) continue;
            auto add = [&](const int (&id)[kFwdBatch], const float (&ln)[kFwdBatch]) {
#pragma unroll
                for (int u = 0; u < kFwdBatch; ++u) {
                    if (ln[u] > 0.f && (unsigned)id[u] < (unsigned)nvox) {
                        ++nz;  // every non-zero of the block counts, whatever r is
                        const int term = __float2int_rn(ln[u] * rs);
                        if (term) atomicAdd(acc + id[u], term);
                    }
                }
            };
            if constexpr (DIM == 2) walk2_batched<kFwdBatch>(q, inv, bb, tin, tout, add);
            else walk3_batched<kFwdBatch>(q, inv, bb, tin, tout, add);
        }
    }
    __syncthreads();
    // g_J = h 2^-S sum, written as (x_J, g_J) pairs; g^T g and nnz per CTA
    const float isc = pow2f(-S) * G.h;
    float2* gout = reinterpret_cast<float2*>(a.sb.g) + (int64_t)slot * a.sb.g_stride;
    const float* xt = a.sb.x + t.voff;
    float gg = 0.f;
    for (int v = threadIdx.x; v < nvox; v += blockDim.x) {
        const int x0 = v % bn[0], x1 = (v / bn[0]) % bn[1], x2 = v / (bn[0] * bn[1]);
        const int vt = ((b_lo[2] + x2) * t.n[1] + (b_lo[1] + x1)) * t.n[0] + b_lo[0] + x0;
        const float gv = (float)acc[v] * isc;
        gout[vt] = make_float2(xt[vt], gv);
        gg = fmaf(gv, gv, gg);
    }
    const float wg = warp_sum_f(gg);
    const unsigned wn = __reduce_add_sync(0xffffffffu, (unsigned)nz);
    __syncthreads();  // s_nz is reused
    if ((threadIdx.x & 31) == 0) {
        s_red[threadIdx.x >> 5] = wg;
        s_nz[threadIdx.x >> 5] = wn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float cg = 0.f;
        unsigned long long cn = 0;
        for (int w = 0; w < kBrickThreads / 32; ++w) {
            cg += s_red[w];
            cn += s_nz[w];
        }
        a.sb.gg_part[(int64_t)slot * a.sb.gg_stride + blockIdx.x] = cg;
        if (a.sb.nnz_slot && cn) atomicAdd(a.sb.nnz_slot + slot, cn);
    }
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
    int w_begin;     // first work item of the batch
    int n_items;     // work items of the batch (CTA rows 0 .. n_items-1)
    int sync_epoch;
    SolverBuffers sb;
};

// CTAs 0 .. n_items-1 (x) update z and r on one work item's rays each; the
// remaining CTAs add the batch's candidates into x^ of the tile.
constexpr int kEpiMu = 32;

__device__ __forceinline__ void epilogue_body(const EpiArgs& a, const VBlock& vb) {
    pdl_trigger();
    const DevGeom& G = a.G;
    if ((int)vb.x < a.n_items) {
        // the item and its (view, tile) constants are fixed for the solve: read
        // them before waiting for the dual forward
        const WorkItem it = a.items[a.w_begin + vb.x];
        const DevVT& E = G.vt[(int64_t)it.view * G.n_tiles + a.j];
        const int ew = E.u1 - E.u0;
        const int64_t zbase = E.zoff - (int64_t)E.v0 * ew - E.u0;
        const int wu = it.u1 - it.u0;
        const int nr = wu * (it.v1 - it.v0);
        pdl_wait();
        const float mu = (float)a.sb.mu[it.slot];
        for (int k = vb.y * blockDim.x + threadIdx.x; k < nr; k += vb.gy * blockDim.x) {
            const int ku = it.u0 + k % wu;
            const int kv = it.v0 + k / wu;
            const int64_t zi = zbase + (int64_t)kv * ew + ku;
            const int64_t ray = ray_index(G, it.view, ku, kv);
            // every load before any store: the arrays are distinct, so all four
            // requests are in flight together
            float* rd = a.sync_epoch ? a.sb.d : a.sb.r;
            const float pv = __ldcg(a.sb.p + ray), qv = __ldcg(a.sb.q + ray);
            const float zo = __ldcg(a.sb.z + zi), rv = __ldcg(rd + ray);
            const float zn = fmaf(mu, qv, pv);
            a.sb.z[zi] = zn;
            rd[ray] = a.sync_epoch ? rv + (zn - zo) : rv - (zn - zo);
        }
    } else {
        const DevTile t = G.tiles[a.j];
        const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
        pdl_wait();
        float* xh = a.sb.xh + t.voff;
        const float* x = a.sb.x + t.voff;
        const int64_t nthreads = (int64_t)(vb.gx - a.n_items) * vb.gy * blockDim.x;
        int64_t v0 = ((int64_t)(vb.x - a.n_items) * vb.gy + vb.y) * blockDim.x +
                     threadIdx.x;
        // the step lengths of the first kEpiMu slots converted once per CTA,
        // not once per voxel
        __shared__ float s_mu[kEpiMu];
        const int nm = min(a.nslots, kEpiMu);
        if ((int)threadIdx.x < nm) s_mu[threadIdx.x] = (float)a.sb.mu[threadIdx.x];
        __syncthreads();
        for (int64_t v = v0; v < nv; v += nthreads) {
            float xv = x[v];
            float s = xh[v];
            for (int sl = 0; sl < nm; ++sl)
                s += fmaf(s_mu[sl], a.sb.g[2 * ((int64_t)sl * a.sb.g_stride + v) + 1], xv);
            for (int sl = nm; sl < a.nslots; ++sl)
                s += fmaf((float)a.sb.mu[sl], a.sb.g[2 * ((int64_t)sl * a.sb.g_stride + v) + 1], xv);
            xh[v] = s;
        }
        if (vb.x == a.n_items && vb.y == 0 && threadIdx.x == 0)
            a.sb.cnt[a.j] += a.nslots;
    }
}

__global__ void __launch_bounds__(kEpiThreads) k_epilogue(const EpiArgs a) {
    epilogue_body(a, hw_block());
}

// x_J = x^_J / count_J and x^_J = 0 for every tile (grid.y = tile), 16-byte
// accesses over the aligned body of each tile's range.
__device__ __forceinline__ void average_body(const DevGeom& G, float* x, float* xh,
                                             const int32_t* cnt, const VBlock& vb) {
    pdl_trigger();
    pdl_wait();
    const int j = vb.y;
    const DevTile t = G.tiles[j];
    const int64_t a0 = t.voff, a1 = t.voff + (int64_t)t.n[0] * t.n[1] * t.n[2];
    const int64_t b0 = min(a1, (a0 + 3) & ~(int64_t)3), b1 = max(b0, a1 & ~(int64_t)3);
    const int c = cnt[j];
    const int64_t tid = (int64_t)vb.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)vb.gx * blockDim.x;
    auto one = [&](int64_t v) {
        if (c > 0) x[v] = xh[v] / (float)c;
        xh[v] = 0.f;
    };
    if (tid < b0 - a0) one(a0 + tid);
    if (tid < a1 - b1) one(b1 + tid);
    float4* x4 = reinterpret_cast<float4*>(x + b0);
    float4* h4 = reinterpret_cast<float4*>(xh + b0);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // four 16-byte groups a thread, nth apart, their loads issued together
    const int64_t n4 = (b1 - b0) / 4;
    for (int64_t k0 = tid; k0 < n4; k0 += nth * 4) {
        float4 h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + u * nth;
            h[u] = k < n4 ? h4[k] : z4;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + u * nth;
            if (k < n4) {
                if (c > 0)
                    x4[k] = make_float4(h[u].x / (float)c, h[u].y / (float)c, h[u].z / (float)c,
                                        h[u].w / (float)c);
                h4[k] = z4;
            }
        }
    }
}

__global__ void k_average(const DevGeom G, float* x, float* xh, const int32_t* cnt) {
    average_body(G, x, xh, cnt, hw_block());
}

__device__ __forceinline__ void apply_pending_body(float* r, float* d, int64_t n,
                                                   const VBlock& vb) {
    pdl_trigger();
    pdl_wait();
    for (int64_t i = (int64_t)vb.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)vb.gx * blockDim.x) {
        float dv = d[i];
        if (dv != 0.f) {
            r[i] -= dv;
            d[i] = 0.f;
        }
    }
}

__global__ void k_apply_pending(float* r, float* d, int64_t n) {
    apply_pending_body(r, d, n, hw_block());
}

__device__ __forceinline__ void tile_to_rowmajor_body(const DevGeom& G, const float* xt,
                                                      float* out, const VBlock& vb) {
    const int j = vb.y;
    const DevTile t = G.tiles[j];
    const int64_t nv = (int64_t)t.n[0] * t.n[1] * t.n[2];
    for (int64_t v = (int64_t)vb.x * blockDim.x + threadIdx.x; v < nv;
         v += (int64_t)vb.gx * blockDim.x) {
        int x0 = (int)(v % t.n[0]);
        int64_t rest = v / t.n[0];
        int x1 = (int)(rest % t.n[1]);
        int x2 = (int)(rest / t.n[1]);
        int64_t gi = ((int64_t)(t.lo[2] + x2) * G.ny + t.lo[1] + x1) * G.nx + t.lo[0] + x0;
        out[gi] = xt[t.voff + v];
    }
}

__global__ void k_tile_to_rowmajor(const DevGeom G, const float* xt, float* out) {
    tile_to_rowmajor_body(G, xt, out, hw_block());
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


// ---------------------------------------------------------------------------
// Batch executor: one persistent launch that runs the kernels of many solves.
//
// The host lists, per problem, the kernels its solve would launch (ray table or
// max |r| pass, backprojection, conversion, dual forward, epilogue, epoch
// closes, x out) as tasks of `units` thread blocks each.  On the device every
// problem has a work word (its current task, next unit) and a count of the
// current task's completed units.  An executor block takes a chunk of units
// from the current task of a problem that has units left (atomic add on the
// work word), starting from its home problem and moving on to the others; runs
// them with the task's kernel body and virtual block indices; and adds them to
// the completed count.  The block that completes a task's last unit publishes
// the problem's next task (release: the task's writes are visible to the
// blocks that then take its units).  So a block never waits for a dependency;
// it only idles when no problem has units left, and that idling is bounded
// (wait_ns of GPU time without work): then the status word is set and every
// block stops.
// ---------------------------------------------------------------------------
// Task kinds; the forward and the scatter come in three lane counts (1, 2, 4
// lanes per ray: kind + 0, 1, 2).
enum ExecKind : int32_t {
    kExTable2, kExTable3, kExRmax, kExGather2, kExGather3, kExConvert, kExEpilogue, kExApply,
    kExAverage, kExClear, kExXout,
    kExScatter2 = 16, kExScatter3 = 19, kExFwdTable2 = 22, kExFwdTable3 = 25, kExFwdInline2 = 28,
    kExFwdInline3 = 31
};
inline int lane_variant(int L) { return L == 4 ? 2 : (L == 2 ? 1 : 0); }

struct ExecMisc {
    DevGeom G;
    float* x;
    float* xh;
    int32_t* cnt;
    float* r;
    float* d;
    int64_t n;
    const float* xt;
    float* out;
};

struct ExecTask {
    int32_t kind;
    int32_t problem;
    uint32_t gx, gy, gz;
    uint32_t units;
    uint32_t need;   // completed units that complete the task (= units)
    uint32_t chunk;  // units one executor block takes at a time
    const WorkItem* items;
    const StepDesc* steps;
    union {
        TableArgs table;
        BPArgs bp;
        ScatterArgs sc;
        FwdSolverArgs fwd;
        EpiArgs epi;
        ExecMisc misc;
    } a;
};

struct ExecArgs {
    const ExecTask* tasks;        // per problem, contiguous, in solve order
    const int* first;             // [problem + 1]: first task of each problem
    int n_problems;
    int n_active;                 // problems with at least one task
    unsigned long long* work;     // [problem]: current task << 32 | next unit
    unsigned* done;               // [problem]: completed units of the current task
    unsigned* finished;           // problems whose last task completed
    int* status;                  // 0, or 1 once the idle bound ran out
    long long wait_ns;
};

__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ void clear_counts_body(int32_t* cnt, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) cnt[k] = 0;
}

// One wrapper per task kind, not inlined: each kernel body keeps its own
// register allocation inside the executor.
#define CSGD_EXEC_WRAP(name, call)                                                     \
    __device__ __noinline__ void name(const ExecTask& T, const VBlock& vb) { call; }
CSGD_EXEC_WRAP(ex_table2, (ray_table_body<2, true>(T.a.table, T.items, vb)))
CSGD_EXEC_WRAP(ex_table3, (ray_table_body<3, true>(T.a.table, T.items, vb)))
CSGD_EXEC_WRAP(ex_rmax, (slot_rmax_body(T.a.table, T.items, vb)))
CSGD_EXEC_WRAP(ex_gather2, (backproject_solver_body<2>(T.a.bp, T.items, T.steps, vb)))
CSGD_EXEC_WRAP(ex_gather3, (backproject_solver_body<3>(T.a.bp, T.items, T.steps, vb)))
CSGD_EXEC_WRAP(ex_convert, (scatter_convert_body(T.a.sc, vb)))
#define CSGD_EXEC_WRAP_L(name, L)                                                       \
    CSGD_EXEC_WRAP(ex_scatter2_##name, (scatter_body<2, L>(T.a.sc, vb)))                \
    CSGD_EXEC_WRAP(ex_scatter3_##name, (scatter_body<3, L>(T.a.sc, vb)))                \
    CSGD_EXEC_WRAP(ex_fwd_table2_##name, (forward_dual_body<2, L, true, true>(T.a.fwd, vb)))  \
    CSGD_EXEC_WRAP(ex_fwd_table3_##name, (forward_dual_body<3, L, true, true>(T.a.fwd, vb)))  \
    CSGD_EXEC_WRAP(ex_fwd_inline2_##name, (forward_dual_body<2, L, false, true>(T.a.fwd, vb))) \
    CSGD_EXEC_WRAP(ex_fwd_inline3_##name, (forward_dual_body<3, L, false, true>(T.a.fwd, vb)))
CSGD_EXEC_WRAP_L(l1, 1)
CSGD_EXEC_WRAP_L(l2, 2)
CSGD_EXEC_WRAP_L(l4, 4)
#undef CSGD_EXEC_WRAP_L
CSGD_EXEC_WRAP(ex_epilogue, (epilogue_body(T.a.epi, vb)))
CSGD_EXEC_WRAP(ex_apply, (apply_pending_body(T.a.misc.r, T.a.misc.d, T.a.misc.n, vb)))
CSGD_EXEC_WRAP(ex_average, (average_body(T.a.misc.G, T.a.misc.x, T.a.misc.xh, T.a.misc.cnt, vb)))
CSGD_EXEC_WRAP(ex_clear, (clear_counts_body(T.a.misc.cnt, (int)T.a.misc.n)))
CSGD_EXEC_WRAP(ex_xout, (tile_to_rowmajor_body(T.a.misc.G, T.a.misc.xt, T.a.misc.out, vb)))
#undef CSGD_EXEC_WRAP

__device__ __forceinline__ void run_unit(const ExecTask& T, unsigned long long w) {
    VBlock vb;
    vb.gx = T.gx;
    vb.gy = T.gy;
    vb.gz = T.gz;
    vb.x = (unsigned)(w % T.gx);
    vb.y = (unsigned)((w / T.gx) % T.gy);
    vb.z = (unsigned)(w / ((unsigned long long)T.gx * T.gy));
    switch (T.kind) {
        case kExTable2: ex_table2(T, vb); break;
        case kExTable3: ex_table3(T, vb); break;
        case kExRmax: ex_rmax(T, vb); break;
        case kExGather2: ex_gather2(T, vb); break;
        case kExGather3: ex_gather3(T, vb); break;
        case kExConvert: ex_convert(T, vb); break;
#define CSGD_EXEC_CASES(base, fn)                      \
        case base: fn##_l1(T, vb); break;              \
        case base + 1: fn##_l2(T, vb); break;          \
        case base + 2: fn##_l4(T, vb); break;
        CSGD_EXEC_CASES(kExScatter2, ex_scatter2)
        CSGD_EXEC_CASES(kExScatter3, ex_scatter3)
        CSGD_EXEC_CASES(kExFwdTable2, ex_fwd_table2)
        CSGD_EXEC_CASES(kExFwdTable3, ex_fwd_table3)
        CSGD_EXEC_CASES(kExFwdInline2, ex_fwd_inline2)
        CSGD_EXEC_CASES(kExFwdInline3, ex_fwd_inline3)
#undef CSGD_EXEC_CASES
        case kExEpilogue: ex_epilogue(T, vb); break;
        case kExApply: ex_apply(T, vb); break;
        case kExAverage: ex_average(T, vb); break;
        case kExClear: ex_clear(T, vb); break;
        case kExXout: ex_xout(T, vb); break;
        default: break;
    }
}

constexpr int kExecThreads = 256;

static_assert(sizeof(ExecTask) % 8 == 0 && alignof(ExecTask) >= 8, "8-byte copies of a task");
constexpr int kTaskWords = (int)(sizeof(ExecTask) / 8);

__global__ void __launch_bounds__(kExecThreads, 4) k_executor(const ExecArgs e) {
    __shared__ int s_task, s_p;
    __shared__ unsigned s_u, s_n;
    // the claimed task's descriptor and arguments, copied into shared memory
    // once per task: the bodies read their arguments from there (a stand-alone
    // kernel has them in its parameter space) instead of from the task list
    __shared__ unsigned long long s_tw[kTaskWords];
    __shared__ int s_cached;
    if (threadIdx.x == 0) s_cached = -1;
    // thread 0's state: the home problem (where the block last found work), the
    // chunk it claims there, and the chunk run last (counted as done before
    // the next claim)
    int home = (int)(blockIdx.x % (unsigned)e.n_problems);
    unsigned claim = 1;
    int prev_task = -1, prev_p = 0;
    unsigned prev_n = 0;
    long long idle_since = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            if (prev_task >= 0) {
                // the last chunk's writes, then its count; the block that
                // completes a task publishes the problem's next one
                __threadfence();
                const ExecTask& T = e.tasks[prev_task];
                if (atomicAdd(e.done + prev_p, prev_n) + prev_n == T.need) {
                    e.done[prev_p] = 0;
                    __threadfence();
                    const int k = prev_task - e.first[prev_p];
                    if (k + 1 == e.first[prev_p + 1] - e.first[prev_p]) atomicAdd(e.finished, 1u);
                    atomicExch(e.work + prev_p, (unsigned long long)(k + 1) << 32);
                }
                prev_task = -1;
            }
            int task = -1, pf = 0;
            unsigned u0 = 0, n = 0;
            if (ld_relaxed_gpu(e.status)) {
                task = -2;
            } else {
                for (int probe = 0; probe < e.n_problems && task < 0; ++probe) {
                    const int p = (home + probe) % e.n_problems;
                    const int ntask = e.first[p + 1] - e.first[p];
                    if (probe > 0) {
                        // another problem: look before claiming
                        const unsigned long long w = ld_relaxed_gpu_u64(e.work + p);
                        const int k = (int)(w >> 32);
                        if (k >= ntask || (unsigned)w >= e.tasks[e.first[p] + k].units) continue;
                        claim = e.tasks[e.first[p] + k].chunk;
                    }
                    // claim `claim` units; whatever task the problem is at by
                    // then, they are units of that task (exactly `claim` of them)
                    const unsigned long long got = atomicAdd(e.work + p, (unsigned long long)claim);
                    const int k2 = (int)(got >> 32);
                    if (k2 >= ntask) continue;
                    const ExecTask& T = e.tasks[e.first[p] + k2];
                    const unsigned u = (unsigned)got;
                    if (u >= T.units) continue;
                    task = e.first[p] + k2;
                    pf = p;
                    u0 = u;
                    n = min(claim, T.units - u);
                    home = p;  // stay with this problem while it has work
                    claim = T.chunk;
                }
                if (task < 0) {
                    if (ld_relaxed_gpu((const int*)e.finished) >= e.n_active) {
                        task = -2;
                    } else {
                        const long long now = global_ns();
                        if (idle_since < 0) idle_since = now;
                        if (now - idle_since > e.wait_ns) {
                            atomicExch(e.status, 1);
                            task = -2;
                        } else {
                            __nanosleep(64);
                        }
                    }
                } else {
                    idle_since = -1;
                    __threadfence();  // the task's inputs were published before its units
                    prev_task = task;
                    prev_p = pf;
                    prev_n = n;
                }
            }
            s_task = task;
            s_p = pf;
            s_u = u0;
            s_n = n;
        }
        __syncthreads();
        const int task = s_task;
        if (task == -2) return;
        if (task >= 0) {
            if (task != s_cached) {
                const unsigned long long* src =
                    reinterpret_cast<const unsigned long long*>(e.tasks + task);
                for (int i = threadIdx.x; i < kTaskWords; i += blockDim.x) s_tw[i] = src[i];
                __syncthreads();
                if (threadIdx.x == 0) s_cached = task;
            }
            const ExecTask& T = *reinterpret_cast<const ExecTask*>(s_tw);
            const unsigned u0 = s_u, n = s_n;
            for (unsigned w = u0; w < u0 + n; ++w) {
                run_unit(T, w);
                __syncthreads();
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// Launch with programmatic stream serialization: the kernel may be scheduled
// before the previous kernel of the stream has finished and waits for it with
// pdl_wait (kernels of the solver's batch sequence).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Resident backprojection CTAs per SM for C view groups (occupancy of the
// compiled kernel), looked up once per device.
static int bp_resident(int dim, int C) {
    static std::mutex mu;
    static int cache[kNoAllocMaxDevices][2][kBPMaxChunks + 1] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return 1;
    std::lock_guard<std::mutex> lk(mu);
    int& n = cache[dev][dim == 3][C];
    if (n == 0) {
        int r = 0;
        cudaError_t e = dim == 2
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_backproject_solver<2>, kBPVox * C, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_backproject_solver<3>, kBPVox * C, 0);
        n = (e == cudaSuccess && r > 0) ? r : 1;
    }
    return n;
}

BPPlan plan_backprojection(const DevGeom& G, const DevTile& tile, int nslots, int views,
                           int sm_count, int force_groups) {
    // Estimated time for C view groups: (waves of CTAs) x (views per thread +
    // a fixed cost of staging, counted as 4 views) / (issue efficiency, taken
    // as proportional to resident warps below 32 per SM).  Ties go to the
    // smaller C.
    BPPlan p;
    p.blocks = bp_blocks(tile, G.dim);
    const int64_t grid = (int64_t)p.blocks * std::max(1, nslots);
    views = std::max(1, views);
    double best = 0.0;
    p.C = 1;
    for (int C = 1; C <= kBPMaxChunks; ++C) {
        const int64_t per_sm = bp_resident(G.dim, C);
        const int64_t cap = per_sm * sm_count;
        const int64_t waves = (grid + cap - 1) / cap;
        const double ctas_per_sm = std::min<double>((double)per_sm, (double)grid / sm_count);
        const double eff = std::min(1.0, ctas_per_sm * (kBPVox / 32) * C / 32.0);
        const double est = (double)waves * ((views + C - 1) / C + 4) / eff;
        if (C == 1 || est < best) {
            best = est;
            p.C = C;
        }
        if (views <= C) break;
    }
    if (force_groups >= 1 && force_groups <= kBPMaxChunks) p.C = force_groups;
    return p;
}

static cudaError_t launch_bp_common(const DevGeom& G, const BPPlan& plan, int nslots,
                                    cudaStream_t s, const BPArgs& a, const InlineItems* inl,
                                    const WorkItem* items, const StepDesc* steps) {
    const dim3 grid((unsigned)plan.blocks, 1, (unsigned)nslots);
    const dim3 block((unsigned)(kBPVox * plan.C));
    if (inl) {
        if (G.dim == 2) k_backproject_inline<2><<<grid, block, 0, s>>>(a, *inl);
        else k_backproject_inline<3><<<grid, block, 0, s>>>(a, *inl);
    } else {
        if (G.dim == 2) return launch_pdl(k_backproject_solver<2>, grid, block, s, a, items, steps);
        return launch_pdl(k_backproject_solver<3>, grid, block, s, a, items, steps);
    }
    return cudaGetLastError();
}

// Rows of a per-item grid: enough CTAs per item to cover its rays with ~4
// passes, at most 16.
static int item_rows(int64_t max_item_rays) {
    int64_t rows = (max_item_rays + 4 * 256 - 1) / (4 * 256);
    return (int)std::max<int64_t>(1, std::min<int64_t>(rows, 16));
}

static cudaError_t launch_table(const DevGeom& G, int n_items, int64_t max_item_rays,
                                cudaStream_t s, const TableArgs& t, const InlineItems* inl,
                                const WorkItem* items) {
    if (n_items <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_items, (unsigned)item_rows(max_item_rays));
    if (inl) {
        if (G.dim == 2) k_ray_table_inline<2><<<grid, 256, 0, s>>>(t, *inl);
        else k_ray_table_inline<3><<<grid, 256, 0, s>>>(t, *inl);
    } else {
        if (G.dim == 2) return launch_pdl(k_ray_table_solver<2>, grid, dim3(256), s, t, items);
        return launch_pdl(k_ray_table_solver<3>, grid, dim3(256), s, t, items);
    }
    return cudaGetLastError();
}

// Lanes per ray: enough threads for ~2048 per SM when rays are few.
int lanes_per_ray(int64_t rays, int sm_count) {
    int64_t want = (int64_t)2048 * sm_count;
    if (rays * 2 > want) return 1;
    if (rays * 4 > want) return 2;
    return 4;
}

template <int DIM>
static void project_inline_L(int L, dim3 grid, const DevGeom& G, const InlineItems& it,
                             const float* x, float* out, int accumulate, cudaStream_t s) {
    if (L == 1) k_project_inline<DIM, 1><<<grid, kFwdThreads, 0, s>>>(G, it, x, out, accumulate);
    else if (L == 2) k_project_inline<DIM, 2><<<grid, kFwdThreads, 0, s>>>(G, it, x, out, accumulate);
    else k_project_inline<DIM, 4><<<grid, kFwdThreads, 0, s>>>(G, it, x, out, accumulate);
}

cudaError_t launch_project_inline(const DevGeom& G, const InlineItems& it, const float* x,
                                  float* out, int accumulate, int sm_count, cudaStream_t s) {
    if (it.step.n_rays <= 0) return cudaSuccess;
    int L = lanes_per_ray(it.step.n_rays, sm_count);
    dim3 grid((unsigned)((it.step.n_rays * L + kFwdThreads - 1) / kFwdThreads));
    if (G.dim == 2) project_inline_L<2>(L, grid, G, it, x, out, accumulate, s);
    else project_inline_L<3>(L, grid, G, it, x, out, accumulate, s);
    return cudaGetLastError();
}

cudaError_t launch_backproject_inline(const DevGeom& G, const DevTile& tile,
                                      const InlineItems& it, const float* r, float* g,
                                      int accumulate, RayRec* table, int sm_count,
                                      cudaStream_t s) {
    TableArgs ta;
    ta.G = G;
    ta.j = it.step.j;
    ta.w_begin = 0;
    ta.r = r;
    ta.table = table;
    ta.slot_stride = 0;
    ta.rmax = nullptr;
    int64_t max_item = 0;
    for (int k = 0; k < it.n; ++k)
        max_item = std::max<int64_t>(max_item, (int64_t)(it.items[k].u1 - it.items[k].u0) *
                                                   (it.items[k].v1 - it.items[k].v0));
    cudaError_t e = launch_table(G, it.n, max_item, s, ta, &it, nullptr);
    if (e != cudaSuccess) return e;
    BPPlan plan = plan_backprojection(G, tile, 1, it.n, sm_count);
    BPArgs a;
    a.G = G;
    a.first = 0;
    a.table = table;
    a.table_stride = 0;
    a.xt = nullptr;
    a.gout = g;
    a.mode = 1;
    a.accumulate = accumulate;
    a.slot_stride = 0;
    a.gg_part = nullptr;
    a.gg_stride = 0;
    a.nnz_slot = nullptr;
    e = launch_bp_common(G, plan, 1, s, a, &it, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Backprojection without allocation
//
// Callers that cannot allocate device memory at the time they run (code inside a
// pre-planned real-time loop, a host that hands out all device memory up front,
// an embedding that forbids cudaMalloc after start-up) use this variant.  Its
// ray table lives in a fixed array in the module's global memory instead of a
// per-call allocation: every GPU that loads the library holds the array until
// the process exits.  All calls share it, so calls that overlap on the GPU (two
// streams, or two host threads) race on it.  Each launch writes every record it
// reads before reading it, so nothing needs clearing between calls.
// ---------------------------------------------------------------------------
static __device__ __align__(256) RayRec g_noalloc_table[kNoAllocMaxRays];

namespace {
std::mutex g_noalloc_mu;
RayRec* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

cudaError_t noalloc_table_address(int device, RayRec** out) {
    // Host code cannot use the array's name as a device address: look the
    // address up once per device, with that device current (the caller's).
    if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_table);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = (RayRec*)ptr;
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

template <bool TABLE>
static cudaError_t launch_forward(int dim, int L, dim3 grid, cudaStream_t s, const FwdSolverArgs& f) {
    const dim3 block(kFwdThreads);
    if (dim == 2) {
        if (L == 1) return launch_pdl(k_forward_dual<2, 1, TABLE>, grid, block, s, f);
        if (L == 2) return launch_pdl(k_forward_dual<2, 2, TABLE>, grid, block, s, f);
        return launch_pdl(k_forward_dual<2, 4, TABLE>, grid, block, s, f);
    }
    if (L == 1) return launch_pdl(k_forward_dual<3, 1, TABLE>, grid, block, s, f);
    if (L == 2) return launch_pdl(k_forward_dual<3, 2, TABLE>, grid, block, s, f);
    return launch_pdl(k_forward_dual<3, 4, TABLE>, grid, block, s, f);
}

cudaError_t launch_batch(const DevGeom& G, const DevTile& tile, const WorkItem* items,
                         const StepDesc* steps, const BatchLaunch& b, const SolverBuffers& sb,
                         int sm_count, cudaStream_t s, cudaEvent_t* ev) {
    if (ev) cudaEventRecord(ev[0], s);
    const bool scatter = b.bp_groups == kBPScatter;
    const bool brick = b.bp_groups <= kBPBrick && b.bp_groups >= kBPBrickLast;
    const int sh = brick ? kBPBrick - b.bp_groups : 0;  // brick shape index
    BPPlan plan = plan_backprojection(G, tile, b.nslots, (b.n_items + b.nslots - 1) / b.nslots,
                                      sm_count, scatter || brick ? 0 : b.bp_groups);
    const int L = b.fwd_lanes == 1 || b.fwd_lanes == 2 || b.fwd_lanes == 4
                      ? b.fwd_lanes : lanes_per_ray(b.max_rays * b.nslots, sm_count);
    int64_t nb = (b.max_rays * L + kFwdThreads - 1) / kFwdThreads;
    if (nb < 1) nb = 1;
    if (nb > sb.max_fwd_blocks || nb > sb.qq_stride) return cudaErrorInvalidValue;
    // 1. g_J = (A_I^J)^T r_I per slot: ray table, then voxel-driven sums
    TableArgs ta;
    ta.G = G;
    ta.j = b.j;
    ta.w_begin = b.w_begin;
    ta.r = sb.r;
    ta.table = sb.table;
    ta.slot_stride = sb.table_stride;
    ta.rmax = sb.rmax;
    // the gather reads a ray table; the scatter and the bricks set their lines
    // up themselves (the scatter after a pass for each slot's max |r|)
    cudaError_t e = cudaSuccess;
    if (scatter) {
        if (b.n_items > 0)
            e = launch_pdl(k_slot_rmax, dim3((unsigned)b.n_items, (unsigned)item_rows(b.max_item_rays)),
                           dim3(256), s, ta, items);
    } else if (!brick) {
        e = launch_table(G, b.n_items, b.max_item_rays, s, ta, nullptr, items);
    }
    if (e != cudaSuccess) return e;
    int n_gg = plan.blocks;
    if (brick) {
        BrickArgs ba;
        ba.G = G;
        ba.items = items;
        ba.steps = steps;
        ba.first = b.first;
        ba.r = sb.r;
        ba.sb = sb;
        n_gg = brick_count(tile, G.dim, sh);
        if (n_gg > sb.gg_stride) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)n_gg, b.nslots), block(kBrickThreads);
        if (G.dim == 2)
            e = sh == 0 ? launch_pdl(k_backproject_brick<2, 0>, grid, block, s, ba)
              : sh == 1 ? launch_pdl(k_backproject_brick<2, 1>, grid, block, s, ba)
                        : launch_pdl(k_backproject_brick<2, 2>, grid, block, s, ba);
        else
            e = sh == 0 ? launch_pdl(k_backproject_brick<3, 0>, grid, block, s, ba)
              : sh == 1 ? launch_pdl(k_backproject_brick<3, 1>, grid, block, s, ba)
                        : launch_pdl(k_backproject_brick<3, 2>, grid, block, s, ba);
        if (e != cudaSuccess) return e;
    } else if (scatter) {
        ScatterArgs sa;
        sa.G = G;
        sa.items = items;
        sa.steps = steps;
        sa.first = b.first;
        sa.lane_factor = L > 1 ? 2.f : 1.f;
        sa.sb = sb;
        dim3 grid((unsigned)nb, b.nslots);
        if (G.dim == 2) {
            if (L == 1) e = launch_pdl(k_backproject_scatter<2, 1>, grid, dim3(kFwdThreads), s, sa);
            else if (L == 2) e = launch_pdl(k_backproject_scatter<2, 2>, grid, dim3(kFwdThreads), s, sa);
            else e = launch_pdl(k_backproject_scatter<2, 4>, grid, dim3(kFwdThreads), s, sa);
        } else {
            if (L == 1) e = launch_pdl(k_backproject_scatter<3, 1>, grid, dim3(kFwdThreads), s, sa);
            else if (L == 2) e = launch_pdl(k_backproject_scatter<3, 2>, grid, dim3(kFwdThreads), s, sa);
            else e = launch_pdl(k_backproject_scatter<3, 4>, grid, dim3(kFwdThreads), s, sa);
        }
        if (e != cudaSuccess) return e;
        const int64_t tv = (int64_t)tile.n[0] * tile.n[1] * tile.n[2];
        n_gg = conv_blocks(tv);
        if (n_gg > sb.gg_stride) return cudaErrorInvalidValue;
        e = launch_pdl(k_scatter_convert, dim3((unsigned)n_gg, b.nslots), dim3(kConvThreads), s, sa);
        if (e != cudaSuccess) return e;
    } else {
        if (plan.blocks > sb.gg_stride) return cudaErrorInvalidValue;
        BPArgs a;
        a.G = G;
        a.first = b.first;
        a.table = sb.table;
        a.table_stride = sb.table_stride;
        a.xt = sb.x;
        a.gout = sb.g;
        a.mode = 0;
        a.accumulate = 0;
        a.slot_stride = sb.g_stride;
        a.gg_part = sb.gg_part;
        a.gg_stride = sb.gg_stride;
        a.nnz_slot = sb.nnz_slot;
        e = launch_bp_common(G, plan, b.nslots, s, a, nullptr, items, steps);
        if (e != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], s);
    // 2. p = A x_J, q = A g_J, ||q||^2, mu
    FwdSolverArgs f;
    f.G = G;
    f.items = items;
    f.steps = steps;
    f.first = b.first;
    f.sync_epoch = b.sync_epoch;
    f.n_gg = n_gg;
    f.sb = sb;
    dim3 grid((unsigned)nb, b.nslots);
    // only the gather builds a ray table; otherwise the forward sets its lines up
    if (brick || scatter) e = launch_forward<false>(G.dim, L, grid, s, f);
    else e = launch_forward<true>(G.dim, L, grid, s, f);
    if (e == cudaSuccess) e = cudaGetLastError();
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
    ea.w_begin = b.w_begin;
    ea.n_items = b.n_items;
    ea.sync_epoch = b.sync_epoch;
    ea.sb = sb;
    const int rows = item_rows(b.max_item_rays);
    const int64_t tv = (int64_t)tile.n[0] * tile.n[1] * tile.n[2];
    const int64_t vox_blocks = std::max<int64_t>(1, (tv + (int64_t)kEpiThreads * rows - 1) /
                                                       ((int64_t)kEpiThreads * rows));
    e = launch_pdl(k_epilogue, dim3((unsigned)(b.n_items + vox_blocks), rows), dim3(kEpiThreads), s, ea);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (ev) cudaEventRecord(ev[3], s);
    return e;
}

// ---------------------------------------------------------------------------
// Batch executor plan (host side)
// ---------------------------------------------------------------------------
struct ExecPlan {
    std::vector<std::vector<ExecTask>> lists;  // per problem, in solve order
    ExecTask* d_tasks = nullptr;
    int* d_first = nullptr;
    unsigned long long* d_work = nullptr;
    unsigned* d_done = nullptr;
    unsigned* d_finished = nullptr;
    int* d_status = nullptr;
    int n_tasks = 0;
    int n_active = 0;               // problems with at least one task
    unsigned long long blocks = 0;  // thread blocks of all tasks
    int grid = 0;
    long long wait_ns = 0;
};

static ExecTask exec_task(int kind, int problem, int64_t gx, int64_t gy, int64_t gz,
                          const WorkItem* items, const StepDesc* steps) {
    ExecTask t;
    memset(&t, 0, sizeof(t));
    t.kind = kind;
    t.problem = problem;
    t.gx = (uint32_t)std::max<int64_t>(1, gx);
    t.gy = (uint32_t)std::max<int64_t>(1, gy);
    t.gz = (uint32_t)std::max<int64_t>(1, gz);
    t.units = t.gx * t.gy * t.gz;
    t.items = items;
    t.steps = steps;
    return t;
}

ExecPlan* exec_plan_new(int n_problems) {
    ExecPlan* P = new (std::nothrow) ExecPlan;
    if (P) P->lists.resize(std::max(0, n_problems));
    return P;
}

void exec_plan_free(ExecPlan* P) {
    if (!P) return;
    cudaFree(P->d_tasks);
    cudaFree(P->d_first);
    cudaFree(P->d_work);
    cudaFree(P->d_done);
    cudaFree(P->d_finished);
    cudaFree(P->d_status);
    delete P;
}

// The kernels of one batch of a solve (launch_batch) as executor tasks: the
// same arguments and grids for 256-thread blocks, the solver's lanes per ray
// (b.fwd_lanes, 1 if unset) in the forward and the scatter, four view groups
// per gather block, and the bricks' batches run by the scatter.
cudaError_t exec_plan_add_batch(ExecPlan* P, int problem, const DevGeom& G, const DevTile& tile,
                                const WorkItem* items, const StepDesc* steps, const BatchLaunch& b,
                                const SolverBuffers& sb, int sm_count) {
    std::vector<ExecTask>& out = P->lists[problem];
    const bool scatter = b.bp_groups == kBPScatter ||
                         (b.bp_groups <= kBPBrick && b.bp_groups >= kBPBrickLast);
    const bool d2 = G.dim == 2;
    const int L = b.fwd_lanes == 2 || b.fwd_lanes == 4 ? b.fwd_lanes : 1;
    const int lv = lane_variant(L);
    TableArgs ta;
    ta.G = G;
    ta.j = b.j;
    ta.w_begin = b.w_begin;
    ta.r = sb.r;
    ta.table = sb.table;
    ta.slot_stride = sb.table_stride;
    ta.rmax = sb.rmax;
    const int rows = item_rows(b.max_item_rays);
    const int64_t tv = (int64_t)tile.n[0] * tile.n[1] * tile.n[2];
    int n_gg = 0;
    if (scatter) {
        if (b.n_items > 0) {
            ExecTask t = exec_task(kExRmax, problem, b.n_items, rows, 1, items, steps);
            t.a.table = ta;
            out.push_back(t);
        }
        ScatterArgs sa;
        sa.G = G;
        sa.items = items;
        sa.steps = steps;
        sa.first = b.first;
        sa.lane_factor = L > 1 ? 2.f : 1.f;
        sa.sb = sb;
        const int64_t nb = (b.max_rays * L + kExecThreads - 1) / kExecThreads;
        ExecTask t = exec_task((d2 ? kExScatter2 : kExScatter3) + lv, problem, nb, b.nslots, 1, items,
                               steps);
        t.a.sc = sa;
        out.push_back(t);
        static_assert(kExecThreads == kConvThreads, "the conversion runs in executor blocks");
        n_gg = conv_blocks(tv);
        if (n_gg > sb.gg_stride) return cudaErrorInvalidValue;
        t = exec_task(kExConvert, problem, n_gg, b.nslots, 1, items, steps);
        t.a.sc = sa;
        out.push_back(t);
    } else {
        if (b.n_items > 0) {
            ExecTask t = exec_task(d2 ? kExTable2 : kExTable3, problem, b.n_items, rows, 1, items, steps);
            t.a.table = ta;
            out.push_back(t);
        }
        const BPPlan plan = plan_backprojection(G, tile, b.nslots, (b.n_items + b.nslots - 1) / b.nslots,
                                                sm_count, kExecThreads / kBPVox);
        if (plan.blocks > sb.gg_stride || plan.C * kBPVox != kExecThreads) return cudaErrorInvalidValue;
        BPArgs a;
        a.G = G;
        a.first = b.first;
        a.table = sb.table;
        a.table_stride = sb.table_stride;
        a.xt = sb.x;
        a.gout = sb.g;
        a.mode = 0;
        a.accumulate = 0;
        a.slot_stride = sb.g_stride;
        a.gg_part = sb.gg_part;
        a.gg_stride = sb.gg_stride;
        a.nnz_slot = sb.nnz_slot;
        ExecTask t = exec_task(d2 ? kExGather2 : kExGather3, problem, plan.blocks, 1, b.nslots, items,
                               steps);
        t.a.bp = a;
        out.push_back(t);
        n_gg = plan.blocks;
    }
    const int64_t nb = std::max<int64_t>(1, (b.max_rays * L + kExecThreads - 1) / kExecThreads);
    if (nb > sb.max_fwd_blocks || nb > sb.qq_stride) return cudaErrorInvalidValue;
    FwdSolverArgs f;
    f.G = G;
    f.items = items;
    f.steps = steps;
    f.first = b.first;
    f.sync_epoch = b.sync_epoch;
    f.n_gg = n_gg;
    f.sb = sb;
    const int fk = (scatter ? (d2 ? kExFwdInline2 : kExFwdInline3) : (d2 ? kExFwdTable2 : kExFwdTable3)) + lv;
    ExecTask t = exec_task(fk, problem, nb, b.nslots, 1, items, steps);
    t.a.fwd = f;
    out.push_back(t);
    EpiArgs ea;
    ea.G = G;
    ea.items = items;
    ea.steps = steps;
    ea.first = b.first;
    ea.nslots = b.nslots;
    ea.j = b.j;
    ea.w_begin = b.w_begin;
    ea.n_items = b.n_items;
    ea.sync_epoch = b.sync_epoch;
    ea.sb = sb;
    const int64_t vox_blocks = std::max<int64_t>(1, (tv + (int64_t)kEpiThreads * rows - 1) /
                                                       ((int64_t)kEpiThreads * rows));
    t = exec_task(kExEpilogue, problem, b.n_items + vox_blocks, rows, 1, items, steps);
    t.a.epi = ea;
    out.push_back(t);
    return cudaSuccess;
}

// An epoch close (launch_epoch_close) as tasks: pending residual change (epoch
// sync), averages, clearing the candidate counts.
void exec_plan_add_close(ExecPlan* P, int problem, const DevGeom& G, const SolverBuffers& sb,
                         int64_t n_rays, int64_t max_tile_voxels, int sync_epoch) {
    std::vector<ExecTask>& L = P->lists[problem];
    ExecMisc m;
    memset(&m, 0, sizeof(m));
    m.G = G;
    m.x = sb.x;
    m.xh = sb.xh;
    m.cnt = sb.cnt;
    m.r = sb.r;
    m.d = sb.d;
    m.n = n_rays;
    if (sync_epoch) {
        ExecTask t = exec_task(kExApply, problem, std::min<int64_t>((n_rays + 255) / 256, 4096), 1, 1,
                               nullptr, nullptr);
        t.a.misc = m;
        L.push_back(t);
    }
    ExecTask t = exec_task(kExAverage, problem, std::min<int64_t>((max_tile_voxels / 4 + 1023) / 1024, 1024),
                           G.n_tiles, 1, nullptr, nullptr);
    t.a.misc = m;
    L.push_back(t);
    m.n = G.n_tiles;
    t = exec_task(kExClear, problem, 1, 1, 1, nullptr, nullptr);
    t.a.misc = m;
    L.push_back(t);
}

void exec_plan_add_xout(ExecPlan* P, int problem, const DevGeom& G, const float* xt, float* out,
                        int64_t max_tile_voxels) {
    ExecMisc m;
    memset(&m, 0, sizeof(m));
    m.G = G;
    m.xt = xt;
    m.out = out;
    ExecTask t = exec_task(kExXout, problem, std::min<int64_t>((max_tile_voxels + 255) / 256, 1024),
                           G.n_tiles, 1, nullptr, nullptr);
    t.a.misc = m;
    P->lists[problem].push_back(t);
}

// Upload the problems' task lists (contiguous, per problem); a task's chunk is
// the units an executor block takes at a time: one for a task of fewer than
// 128 blocks, up to 16 of a large one (about 64 claims per task).
cudaError_t exec_plan_finalize(ExecPlan* P, int64_t wait_ns, int stall_last, int sm_count) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_executor, kExecThreads, 0);
    if (e != cudaSuccess) return e;
    P->grid = std::max(1, per_sm) * std::max(1, sm_count);
    std::vector<ExecTask> all;
    std::vector<int> first;
    for (size_t p = 0; p < P->lists.size(); ++p) {
        first.push_back((int)all.size());
        P->n_active += P->lists[p].empty() ? 0 : 1;
        for (size_t k = 0; k < P->lists[p].size(); ++k) {
            ExecTask t = P->lists[p][k];
            t.need = t.units;
            if (stall_last && p == 0 && k + 1 == P->lists[p].size()) t.need += 1;  // never complete
            t.chunk = (uint32_t)std::min<int64_t>(16, std::max<int64_t>(1, (int64_t)t.units / 64));
            P->blocks += t.units;
            all.push_back(t);
        }
    }
    first.push_back((int)all.size());
    if (all.empty()) return cudaErrorInvalidValue;
    P->n_tasks = (int)all.size();
    P->wait_ns = wait_ns;
    const size_t np = std::max<size_t>(1, P->lists.size());
    e = cudaMalloc(&P->d_tasks, sizeof(ExecTask) * all.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->d_first, sizeof(int) * first.size());
    if (e == cudaSuccess) e = cudaMalloc(&P->d_work, sizeof(unsigned long long) * np);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_done, sizeof(unsigned) * np);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_finished, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_status, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_tasks, all.data(), sizeof(ExecTask) * all.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice);
    return e;
}

// Capturable: work words, counts and status cleared, then the persistent launch.
cudaError_t exec_plan_launch(ExecPlan* P, cudaStream_t s) {
    const size_t np = std::max<size_t>(1, P->lists.size());
    cudaError_t e = cudaMemsetAsync(P->d_work, 0, sizeof(unsigned long long) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_done, 0, sizeof(unsigned) * np, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_finished, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->d_status, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    ExecArgs a;
    a.tasks = P->d_tasks;
    a.first = P->d_first;
    a.n_problems = (int)P->lists.size();
    a.n_active = P->n_active;
    a.work = P->d_work;
    a.done = P->d_done;
    a.finished = P->d_finished;
    a.status = P->d_status;
    a.wait_ns = P->wait_ns;
    k_executor<<<P->grid, kExecThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t exec_plan_status(ExecPlan* P, int* status) {
    return cudaMemcpy(status, P->d_status, sizeof(int), cudaMemcpyDeviceToHost);
}

void exec_plan_info(const ExecPlan* P, int* n_tasks, int64_t* n_units, int* grid) {
    *n_tasks = P->n_tasks;
    *n_units = (int64_t)P->blocks;
    *grid = P->grid;
}

cudaError_t launch_epoch_close(const DevGeom& G, const SolverBuffers& sb, int64_t n_rays,
                               int64_t max_tile_voxels, int sync_epoch, cudaStream_t s) {
    if (sync_epoch) {
        int64_t nb = std::min<int64_t>((n_rays + 255) / 256, 4096);
        cudaError_t e = launch_pdl(k_apply_pending, dim3((unsigned)std::max<int64_t>(nb, 1)), dim3(256),
                                   s, sb.r, sb.d, n_rays);
        if (e != cudaSuccess) return e;
    }
    int64_t nb = std::min<int64_t>((max_tile_voxels / 4 + 1023) / 1024, 1024);
    cudaError_t e = launch_pdl(k_average, dim3((unsigned)std::max<int64_t>(nb, 1), G.n_tiles), dim3(256),
                               s, G, sb.x, sb.xh, (const int32_t*)sb.cnt);
    if (e == cudaSuccess) e = cudaGetLastError();
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
