// Device helpers: ray set-up (a1), incremental Siddon traversal (the forward
// products) and small reductions.
//
// A_i^j is the length of line i inside voxel j (Sec. II-A).  The forward walks
// and the voxel-driven backprojection's slab clip both evaluate the crossing
// parameter of a plane as t = (plane - q) * (1/d) in tile-centred coordinates,
// with the same operations, so the forward and adjoint operators see
// bit-identical lengths for the same line and voxel.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.h"

namespace csgd {

// Tile-centred reference point q and unit direction d of the line through bin
// (ku, kv) of view V, for the tile whose per (view, tile) constants are E.
__device__ __forceinline__ void ray_setup(const DevGeom& G, const DevView& V, const DevVT& E,
                                          int ku, int kv, float q[3], float d[3]) {
    if (G.kind == FAN_2D_CURVED) {
        // direction at angle gamma_k from the central ray; the point at the tile
        // centre's depth D is offset laterally by D (tan gamma_k - tan gamma_k0),
        // written as D sin(gamma_k - gamma_k0) / (cos gamma_k cos gamma_k0) so that
        // nothing cancels.
        float gam = ((float)ku - G.cu) * G.pu;
        float sg, cg;
        sincosf(gam, &sg, &cg);
        float del = (float)(ku - E.k0u) * G.pu;
        float lat = E.U[0] * sinf(del) * (E.U[1] / cg);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q[a] = fmaf(lat, V.eu[a], E.B[a]);
            d[a] = cg * V.dc[a] + sg * V.eu[a];
        }
        return;
    }
    float du = (float)(ku - E.k0u), dv = (float)(kv - E.k0v);
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = fmaf(dv, E.V[a], fmaf(du, E.U[a], E.B[a]));
    if (G.kind == PARALLEL_2D) {
#pragma unroll
        for (int a = 0; a < 3; ++a) d[a] = V.dc[a];
        return;
    }
    float u = ((float)ku - G.cu) * G.pu;
    float w = ((float)kv - G.cv) * G.pv;
    float n2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        d[a] = fmaf(w, V.ev[a], fmaf(u, V.eu[a], V.sdd * V.dc[a]));
        n2 = fmaf(d[a], d[a], n2);
    }
    float inv = 1.0f / sqrtf(n2);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] *= inv;
}

// Box of voxels for a traversal: tile-centred lower corner, size, index strides.
struct Box {
    float lo[3];
    int n[3];
    int stride[3];
    int base;
};

// Reciprocal direction used by every plane crossing: 1/d, infinite where d = 0
// (__frcp_rn: the correctly rounded reciprocal, the value 1.0f / d has).
__device__ __forceinline__ void reciprocal(const float d[3], float inv[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) inv[a] = d[a] != 0.f ? __frcp_rn(d[a]) : INFINITY;
}

// Parameter interval [tin, tout) of the line q + t d inside the box, given
// inv = 1/d; false if the line misses it.  A plane crossing is always
// evaluated as (plane - q) * inv.
template <int DIM>
__device__ __forceinline__ bool clip(const float q[3], const float inv[3], const Box& b,
                                     float* tin, float* tout) {
    float t0 = -INFINITY, t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (isfinite(inv[a])) {
            float ta = (b.lo[a] - q[a]) * inv[a];
            float tb = (b.lo[a] + (float)b.n[a] - q[a]) * inv[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (!(q[a] >= b.lo[a] && q[a] < b.lo[a] + (float)b.n[a])) {
            return false;
        }
    }
    *tin = t0;
    *tout = t1;
    return t0 < t1;
}

// ---------------------------------------------------------------------------
// Lines that only touch a tile.  A line through a corner of a tile (2D) or
// along one of its edges (3D) meets it in exact geometry with length 0, so it
// gives the block A_I^J no entry (the FP64 oracle's Siddon drops such gaps as
// structural zeros).  The FP32 set-up places a line to about 1e-5 voxel, and
// may clip a sliver off the tile instead: of length up to ~1e-5 / sin(phi) for
// a line at angle phi to the axes.  A block whose only support is such
// slivers (a detector sub-area that meets the tile's shadow only at its edge,
// with a bin centre exactly on that edge) would get q = A g of the order of the
// sliver length squared times r and an exact line search mu ~ 1 / length^2.
// So whenever the FP32 clip enters and leaves the tile through faces of two
// different axes and its extent along one of them is below kSliverExtent (a
// hundred times the FP32 placement error), the chord is recomputed in FP64 from
// the unrounded frame, and a line whose exact chord is at most kTouchChord has
// no support in the tile.  Lines with a genuine chord are left as they are.
// ---------------------------------------------------------------------------
constexpr float kSliverExtent = 1.0f / 1024.0f;
constexpr double kTouchChord = 1e-9;  // voxel units
// q[0] of a line that has no support in the tile: every slab of the tile is
// then empty for it (clip fails, slab clips give length 0)
constexpr float kNoSupport = 1e30f;

// The clip of `clip` that also reports whether the chord [tin, tout] is an
// edge sliver (entry and exit faces of different axes, extent along one of
// them below kSliverExtent).  Same arithmetic as clip.
template <int DIM>
__device__ __forceinline__ bool clip_sliver(const float q[3], const float inv[3], const Box& b,
                                            float* tin, float* tout, bool* sliver) {
    float t0 = -INFINITY, t1 = INFINITY;
    float e0 = 0.f, e1 = 0.f;  // |1/d| of the entry and exit axes
    bool in_set = false, out_set = false;
    int ain = -1, aout = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        if (isfinite(inv[a])) {
            float ta = (b.lo[a] - q[a]) * inv[a];
            float tb = (b.lo[a] + (float)b.n[a] - q[a]) * inv[a];
            const float lo = fminf(ta, tb), hi = fmaxf(ta, tb);
            if (lo > t0) { t0 = lo; e0 = fabsf(inv[a]); ain = a; in_set = true; }
            if (hi < t1) { t1 = hi; e1 = fabsf(inv[a]); aout = a; out_set = true; }
        } else if (!(q[a] >= b.lo[a] && q[a] < b.lo[a] + (float)b.n[a])) {
            *sliver = false;
            return false;
        }
    }
    *tin = t0;
    *tout = t1;
    const float L = t1 - t0;
    *sliver = in_set && out_set && ain != aout && fminf(L / e0, L / e1) < kSliverExtent;
    return t0 < t1;
}

// The exact line of bin (ku, kv) of a view, in FP64 from the unrounded frame V
// (the line the per (view, tile) FP32 constants round), in the coordinates of
// the tile whose centre is T (voxel units): p0 + s d.  The functions below are
// the cold path of the line set-up (rare lines only): they take scalars, are
// not inlined, and keep their FP64 arithmetic out of the set-up of every line.
__device__ __forceinline__ void exact_line(const DevView64& V, int kind, float cu, float cv,
                                           double pu, double pv, int ku, int kv, const float T[3],
                                           double p0[3], double d[3]) {
    if (kind == PARALLEL_2D) {
        const double s = ((double)ku - (double)cu) * pu;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p0[a] = s * V.eu[a] - (double)T[a];
            d[a] = V.dc[a];
        }
    } else if (kind == FAN_2D_CURVED) {
        double sg, cg;
        sincos(((double)ku - (double)cu) * pu, &sg, &cg);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p0[a] = V.S[a] - (double)T[a];
            d[a] = cg * V.dc[a] + sg * V.eu[a];
        }
    } else {
        const double u = ((double)ku - (double)cu) * pu;
        const double w = ((double)kv - (double)cv) * pv;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p0[a] = V.S[a] - (double)T[a];
            d[a] = V.sdd * V.dc[a] + u * V.eu[a] + w * V.ev[a];
        }
    }
}

// Chord (voxel units) of that exact line through the tile of centre T and size
// n; at most 0 when it misses the tile.  Half-open faces as in the walk: a line
// parallel to an axis meets the tile when lo <= q < hi.
__device__ __noinline__ double exact_chord_of(const DevView64* V, int kind, int dim, float cu,
                                              float cv, double pu, double pv, int ku, int kv,
                                              float T0, float T1, float T2, int n0, int n1,
                                              int n2) {
    const float T[3] = {T0, T1, T2};
    const int n[3] = {n0, n1, n2};
    double p0[3], d[3];
    exact_line(*V, kind, cu, cv, pu, pv, ku, kv, T, p0, d);
    double t0 = -INFINITY, t1 = INFINITY, dn = 0.0;
    for (int a = 0; a < dim; ++a) {
        const double lo = -0.5 * (double)n[a], hi = 0.5 * (double)n[a];
        dn += d[a] * d[a];
        if (d[a] == 0.0) {
            if (!(p0[a] >= lo && p0[a] < hi)) return -1.0;
        } else {
            const double ta = (lo - p0[a]) / d[a], tb = (hi - p0[a]) / d[a];
            t0 = fmax(t0, fmin(ta, tb));
            t1 = fmin(t1, fmax(ta, tb));
        }
    }
    return (t1 - t0) * sqrt(dn);
}

__device__ __forceinline__ double exact_chord(const DevGeom& G, int view, int ku, int kv,
                                              const DevTile& t) {
    return exact_chord_of(G.views64 + view, G.kind, G.dim, G.cu, G.cv, G.pu_d, G.pv_d, ku, kv, t.T[0],
                          t.T[1], t.T[2], t.n[0], t.n[1], t.n[2]);
}

// Coordinate along axis ax of a line parallel to that axis's planes, placed on
// the same side of its nearest voxel face as the exact (FP64) line: the FP32
// set-up may put a line that lies exactly on a face (a view at a multiple of
// 90 degrees and a bin on a face), or within rounding of one, on either side,
// and so in the wrong voxel column (or tile) over its whole length.  A line
// exactly on a face goes to the voxel above it (half-open voxels), one ulp
// above the face, so that (face - q) / d is never 0 / 0 either.
__device__ __noinline__ float parallel_coord_of(const DevView64* V, int kind, float cu, float cv,
                                                double pu, double pv, int ku, int kv, float T0,
                                                float T1, float T2, int n_ax, int ax) {
    const float T[3] = {T0, T1, T2};
    double p0[3], d[3];
    exact_line(*V, kind, cu, cv, pu, pv, ku, kv, T, p0, d);
    const double e = p0[ax];
    const double hn = 0.5 * (double)n_ax;
    const double f = rint(e + hn) - hn;  // nearest face (an exact float)
    const float ff = (float)f, qa = (float)e;
    return e >= f ? fmaxf(qa, nextafterf(ff, INFINITY)) : fminf(qa, nextafterf(ff, -INFINITY));
}

__device__ __forceinline__ float parallel_coord(const DevGeom& G, int view, int ku, int kv,
                                                const DevTile& t, int ax) {
    return parallel_coord_of(G.views64 + view, G.kind, G.cu, G.cv, G.pu_d, G.pv_d, ku, kv, t.T[0],
                             t.T[1], t.T[2], t.n[ax], ax);
}

// Incremental Siddon walk of the line q + t d through the box over t in
// [tin, tout] (inside the box), given inv = 1/d.  Calls f(index, length) for
// every voxel the line crosses, in order, with the running linear index base +
// sum_a i_a * stride_a; lengths are >= 0 (a zero length can occur where the line
// passes exactly through an edge).  Plane crossings are (plane - q) * inv, the
// same values `clip` and the voxel-driven backprojection compute, so lengths do
// not depend on the box or sub-range a walk runs over.  Returns the number of
// positive lengths.  Indices never leave the box, which also bounds the number
// of iterations.
template <int DIM, class F>
__device__ __forceinline__ int walk(const float q[3], const float inv[3], const Box& b, float tin,
                                    float tout, F&& f) {
    int i[3], st[3];
    float pl[3], tn[3];
    int idx = b.base;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const bool moves = isfinite(inv[a]);
        // the start position only picks the first voxel: a rounding error there
        // gives a zero-length first segment and the walk moves on
        float pa = moves ? q[a] + tin / inv[a] : q[a];
        int ia = (int)floorf(pa - b.lo[a]);
        ia = ia < 0 ? 0 : (ia >= b.n[a] ? b.n[a] - 1 : ia);
        i[a] = ia;
        const bool up = moves && inv[a] > 0.f;
        st[a] = up ? 1 : -1;
        pl[a] = b.lo[a] + (float)(ia + (up ? 1 : 0));
        tn[a] = moves ? (pl[a] - q[a]) * inv[a] : INFINITY;
        idx += ia * b.stride[a];
    }
    float tc = tin;
    int cnt = 0;
    if (DIM == 2) {
        // branch-free advance: lanes of a warp that step along different axes
        // execute the same instructions
        float tx = tn[0], ty = tn[1];
        int ix = i[0], iy = i[1];
        float px = pl[0], py = pl[1];
        const int sx = st[0], sy = st[1];
        const int dsx = sx * b.stride[0], dsy = sy * b.stride[1];
        const float fsx = (float)sx, fsy = (float)sy;
        const unsigned nx = (unsigned)b.n[0], ny = (unsigned)b.n[1];
        for (;;) {
            const bool bx = tx <= ty;
            const float t = fminf(bx ? tx : ty, tout);
            const float len = fmaxf(t - tc, 0.f);
            f(idx, len);
            cnt += len > 0.f;
            if (t >= tout) break;
            tc = t;
            ix += bx ? sx : 0;
            iy += bx ? 0 : sy;
            idx += bx ? dsx : dsy;
            px += bx ? fsx : 0.f;
            py += bx ? 0.f : fsy;
            const float nxt = (px - q[0]) * inv[0];
            const float nyt = (py - q[1]) * inv[1];
            tx = bx ? nxt : tx;
            ty = bx ? ty : nyt;
            if ((unsigned)ix >= nx || (unsigned)iy >= ny) break;
        }
    } else {
        float tx = tn[0], ty = tn[1], tz = tn[2];
        int ix = i[0], iy = i[1], iz = i[2];
        float px = pl[0], py = pl[1], pz = pl[2];
        for (;;) {
            bool bx = tx <= ty && tx <= tz;
            bool by = !bx && ty <= tz;
            float tm = bx ? tx : (by ? ty : tz);
            float t = fminf(tm, tout);
            float len = fmaxf(t - tc, 0.f);
            f(idx, len);
            cnt += len > 0.f;
            if (t >= tout) break;
            tc = t;
            if (bx) {
                ix += st[0];
                if ((unsigned)ix >= (unsigned)b.n[0]) break;
                idx += st[0] * b.stride[0];
                px += (float)st[0];
                tx = (px - q[0]) * inv[0];
            } else if (by) {
                iy += st[1];
                if ((unsigned)iy >= (unsigned)b.n[1]) break;
                idx += st[1] * b.stride[1];
                py += (float)st[1];
                ty = (py - q[1]) * inv[1];
            } else {
                iz += st[2];
                if ((unsigned)iz >= (unsigned)b.n[2]) break;
                idx += st[2] * b.stride[2];
                pz += (float)st[2];
                tz = (pz - q[2]) * inv[2];
            }
        }
    }
    return cnt;
}

// Whole traversal of the box: clip, then walk.
// The 2D walk producing its crossings in batches of B: f(idx, len) receives
// arrays of B entries once per batch.  Same crossings, same arithmetic and the
// same order as walk<2>; a batch lets the caller have B independent loads in
// flight.  No per-step bounds test: while t < tout the voxel is inside the box,
// because a plane coordinate is an exact float (lo + integer) and the crossing
// of the box's far face, (face - q) * inv, is bit-identical to the exit
// parameter of clip, so the walk reaches t = tout before it could step past
// it; a start index one voxel behind the line only gives a zero-length first
// segment.  Once t = tout every later entry of the batch has length exactly 0
// (t stays at tout), so there is no per-step end test either: an entry of
// length 0 carries a meaningless index, and the caller uses an index only
// where the length is positive (and masks it with the box size).  The batch
// count is capped at the number of faces the box has.
template <int B, class F>
__device__ __forceinline__ void walk2_batched(const float q[3], const float inv[3], const Box& b,
                                             float tin, float tout, F&& f) {
    int ix, iy;
    float px, py, tx, ty;
    int sx, sy;
    {
        const bool mx = isfinite(inv[0]), my = isfinite(inv[1]);
        const float pa = mx ? q[0] + tin / inv[0] : q[0];
        const float pb = my ? q[1] + tin / inv[1] : q[1];
        ix = min(max((int)floorf(pa - b.lo[0]), 0), b.n[0] - 1);
        iy = min(max((int)floorf(pb - b.lo[1]), 0), b.n[1] - 1);
        const bool ux = mx && inv[0] > 0.f, uy = my && inv[1] > 0.f;
        sx = ux ? 1 : -1;
        sy = uy ? 1 : -1;
        px = b.lo[0] + (float)(ix + (ux ? 1 : 0));
        py = b.lo[1] + (float)(iy + (uy ? 1 : 0));
        tx = mx ? (px - q[0]) * inv[0] : INFINITY;
        ty = my ? (py - q[1]) * inv[1] : INFINITY;
    }
    int idx = b.base + ix * b.stride[0] + iy * b.stride[1];
    const int dsx = sx * b.stride[0], dsy = sy * b.stride[1];
    const float fsx = (float)sx, fsy = (float)sy;
    const int max_batches = (b.n[0] + b.n[1] + 2) / B + 1;
    float tc = tin;
    for (int it = 0; tc < tout && it < max_batches; ++it) {
        int id[B];
        float ln[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const float t = fminf(fminf(tx, ty), tout);
            ln[u] = fmaxf(t - tc, 0.f);
            id[u] = idx;
            tc = t;
            // only the axis whose plane is crossed advances (x on ties)
            if (tx <= ty) {
                idx += dsx;
                px += fsx;
                tx = (px - q[0]) * inv[0];
            } else {
                idx += dsy;
                py += fsy;
                ty = (py - q[1]) * inv[1];
            }
        }
        f(id, ln);
    }
}

// The 3D walk in batches of B, branch-free, with the same guarantees and the
// same arithmetic as walk<3> (see walk2_batched).
template <int B, class F>
__device__ __forceinline__ void walk3_batched(const float q[3], const float inv[3], const Box& b,
                                             float tin, float tout, F&& f) {
    float p[3], tn[3], fs[3];
    int ds[3];
    int idx = b.base;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool m = isfinite(inv[a]);
        const float pa = m ? q[a] + tin / inv[a] : q[a];
        const int ia = min(max((int)floorf(pa - b.lo[a]), 0), b.n[a] - 1);
        const bool up = m && inv[a] > 0.f;
        fs[a] = up ? 1.f : -1.f;
        ds[a] = (up ? 1 : -1) * b.stride[a];
        p[a] = b.lo[a] + (float)(ia + (up ? 1 : 0));
        tn[a] = m ? (p[a] - q[a]) * inv[a] : INFINITY;
        idx += ia * b.stride[a];
    }
    const int max_batches = (b.n[0] + b.n[1] + b.n[2] + 3) / B + 1;
    float tc = tin;
    for (int it = 0; tc < tout && it < max_batches; ++it) {
        int id[B];
        float ln[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const float m = fminf(fminf(tn[0], tn[1]), tn[2]);
            const float t = fminf(m, tout);
            ln[u] = fmaxf(t - tc, 0.f);
            id[u] = idx;
            tc = t;
            // only the axis whose plane is crossed advances (x, then y, on ties).
            // Branch-free: the three candidate plane parameters are computed and
            // the crossed axis's is selected (a branch diverges across the lanes
            // of a warp, which cross different axes; an infinite or NaN
            // candidate of an axis the line never crosses is never selected)
            const bool cx = tn[0] == m, cy = !cx && tn[1] == m, cz = !cx && !cy;
            idx += cx ? ds[0] : (cy ? ds[1] : ds[2]);
            p[0] += cx ? fs[0] : 0.f;
            p[1] += cy ? fs[1] : 0.f;
            p[2] += cz ? fs[2] : 0.f;
            const float n0 = (p[0] - q[0]) * inv[0], n1 = (p[1] - q[1]) * inv[1],
                        n2 = (p[2] - q[2]) * inv[2];
            tn[0] = cx ? n0 : tn[0];
            tn[1] = cy ? n1 : tn[1];
            tn[2] = cz ? n2 : tn[2];
        }
        f(id, ln);
    }
}

// Programmatic dependent launch.  pdl_trigger lets the next kernel of the
// stream (launched with programmatic stream serialization) be scheduled while
// this one runs; pdl_wait blocks until the previous kernel of the stream has
// completed and its memory is visible.  A kernel calls pdl_wait before it reads
// anything an earlier kernel writes and before its first global write, so the
// chain of waits orders every kernel after all earlier ones.  Both are no-ops
// in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Compensated (Kahan) accumulator: the stand-alone projection's ray sums and
// the backprojection's per-voxel sums over views.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Running sum of FP32 terms kept exactly as an unevaluated pair s + c
// (Knuth's TwoSum gives each addition's rounding error exactly; the errors are
// added into c, whose own rounding is second order, O(n u^2)).  Used where
// many FP32 partials are added: FP32 ALU work instead of FP64.
struct TwoSumF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float t = s + v;
        const float bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// FP32 butterfly sum of non-negative terms (squares): a tree of depth 5, so the
// result is within 5 u of the exact sum (u = 2^-24).  GB300's FP64 pipe runs
// at about 1/64 of the FP32 rate, so per-thread terms are reduced in FP32 up to
// the CTA and only CTA partials are added in FP64.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (deterministic); every thread gets the result.
// `sh` must hold blockDim.x / 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh[k];
    return s;
}

// Ray index of bin (ku, kv) of view v.
__device__ __forceinline__ int64_t ray_index(const DevGeom& G, int v, int ku, int kv) {
    return ((int64_t)v * G.nv + kv) * G.nu + ku;
}

// The work item holding ray k of a slot whose items are [w0, w1) (binary search
// on the items' ray offsets).
__device__ __forceinline__ int find_item(const WorkItem* items, int w0, int w1, int64_t k) {
    int lo = w0, hi = w1 - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (items[mid].ray_off <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace csgd
