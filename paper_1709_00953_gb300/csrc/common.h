// Internal data layout shared by the host code and the CUDA kernels.
//
// Everything the kernels read about the scan lives in four small device
// tables built once per partition:
//   DevView  per view: the source and the detector frame, FP32, in voxel units;
//   DevVT    per (view, tile): the tile-centred reference point of the ray
//            through bin (k0u, k0v), its steps per bin, the conservative
//            rectangle of bins whose rays can meet the tile, and where that
//            rectangle's slice of the z store starts;
//   DevTile  per tile: origin and size in voxels, centre in voxel units;
//   WorkItem per (step, view): the bins of one view to process for one step.
// Ray set-up uses only tile-centred FP32 quantities whose magnitude is of the
// order of the tile, so that the Siddon lengths keep ~1e-6 voxel precision even
// when the source is a thousand voxels away (the FP64 parts are folded into the
// per (view, tile) constants on the host).
#pragma once
#include <stdint.h>

namespace csgd {

enum Kind { PARALLEL_2D = 0, FAN_2D_FLAT = 1, FAN_2D_CURVED = 2, CONE_3D = 3, CUSTOM_3D = 4 };

struct DevView {
    float S[3];    // source (voxel units); unused for the parallel beam
    float dc[3];   // central direction (unit)
    float eu[3];   // detector u axis (unit)
    float ev[3];   // detector v axis (unit)
    float sdd;     // source-detector distance (voxel units)
    float pad[3];
};

// Per view, FP64, voxel units: the same frame as DevView before rounding.
// Used only for the exact-geometry check of lines that the FP32 set-up finds
// grazing a tile's edge (see touches_only in device.cuh).
struct DevView64 {
    double S[3], dc[3], eu[3], ev[3];
    double sdd;
};

struct DevVT {
    float B[3];    // Q(k0u, k0v) - T: tile-centred point on the reference ray
    float U[3];    // Q step per u bin (flat / parallel); curved: U[0] = depth of
                   // the tile centre, U[1] = 1 / cos(gamma_k0)
    float V[3];    // Q step per v bin
    int32_t k0u, k0v;
    int32_t u0, u1, v0, v1;  // bins [u0,u1) x [v0,v1) whose rays may meet the tile
    float hw_u, hw_v;  // half-width (bins) of the shadow of one voxel of the tile:
                       // the bins whose lines can meet a voxel are within hw of the
                       // bin coordinate of the voxel's centre
    int64_t zoff;  // start of this rectangle's slice of the z store
};

struct DevTile {
    int32_t lo[3];  // first voxel per axis
    int32_t n[3];   // voxels per axis
    float T[3];     // centre (voxel units, grid centred on the origin)
    int64_t voff;   // start of the tile in tile-major volume storage
};

struct alignas(16) WorkItem {
    int32_t view;
    int32_t slot;          // step slot within a launch
    int32_t u0, u1, v0, v1;  // bins to process (inside the DevVT rectangle)
    int64_t ray_off;       // prefix of rays of this slot before this item
};

struct DevGeom {
    int32_t kind;
    int32_t dim;
    int32_t nx, ny, nz;
    int32_t nu, nv, n_views;
    int32_t n_tiles;
    float pu, pv;          // bin pitch in voxel units (radians for the curved arc)
    float cu, cv;          // (nu-1)/2, (nv-1)/2
    float inv_pu, inv_pv;  // 1 / pu, 1 / pv
    float h;               // voxel edge (world units): lengths are scaled by h
    double pu_d, pv_d;     // pu, pv in FP64
    const DevView* views;
    const DevView64* views64;
    const DevVT* vt;       // [view][tile]
    const DevTile* tiles;
};

// Per-ray table of one launch (ray set-up done once, read by the backprojection
// and the dual forward): tile-centred point q, reciprocal direction 1/d
// (infinite where d = 0) and the residual r of the ray.
struct alignas(16) RayRec {
    float a[4];  // q[0], q[1], inv[0], inv[1]
    float b[4];  // r, q[2], inv[2], index of the ray in the sinogram (int bits, < 2^31)
};

// One step of the solver as the kernels see it.
struct StepDesc {
    int32_t j;             // tile
    int32_t w0, w1;        // work items [w0, w1)
    float terms;           // bound on the lines of the step through one voxel of the
                           // tile (per view, the bins within hw_u, hw_v of the voxel)
    int64_t n_rays;        // rays covered by the work items
    int64_t step;          // global step index (for the history)
    double beta;
};

}  // namespace csgd
