// Host-side objects behind the C ABI: geometry, partition, schedule.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/csgd.h"
#include "common.h"

namespace csgd {

struct Frame {
    double S[3], dc[3], eu[3], ev[3];
    double sdd;
};

struct Geometry {
    int kind = 0, dim = 2;
    int n[3] = {1, 1, 1};
    double h = 1.0;
    int n_views = 0;
    std::vector<double> angles, poses;
    int nu = 1, nv = 1;
    double pu = 1.0, pv = 1.0, sod = 0.0, sdd = 0.0;
    std::vector<Frame> frames;  // FP64, world units
    int64_t n_rays() const { return (int64_t)n_views * nu * nv; }
    int64_t n_voxels() const { return (int64_t)n[0] * n[1] * n[2]; }
};

struct Partition {
    const Geometry* g = nullptr;
    int tiles[3] = {1, 1, 1};
    std::vector<int> edges[3];
    int vb_count = 1, du = 1, dv = 1;
    std::vector<int> view_block_of;
    std::vector<std::vector<int>> views_of_vb;
    std::vector<int> u_edges, v_edges;
    int m = 0, n = 0;
    std::vector<double> PS, PT, P;  // P_S [m*n], P_T [n], P = P_S / P_T [m*n]
    std::vector<DevView> views_h;
    std::vector<DevView64> views64_h;
    std::vector<DevVT> vt_h;        // [view * n + tile]
    std::vector<DevTile> tiles_h;
    int64_t z_floats = 0;
    int64_t max_tile_voxels = 0;
    int device = 0;
    DevView* d_views = nullptr;
    DevView64* d_views64 = nullptr;
    DevVT* d_vt = nullptr;
    DevTile* d_tiles = nullptr;
    DevGeom dg{};
    // row block helpers
    void row_block_parts(int i, int* vb, int* dvv, int* duu) const {
        *duu = i % du;
        *dvv = (i / du) % dv;
        *vb = i / (du * dv);
    }
    void subrect(int i, int* u0, int* u1, int* v0, int* v1) const {
        int vb, dvv, duu;
        row_block_parts(i, &vb, &dvv, &duu);
        *u0 = u_edges[duu];
        *u1 = u_edges[duu + 1];
        *v0 = v_edges[dvv];
        *v1 = v_edges[dvv + 1];
    }
    const std::vector<int>& views_of(int i) const {
        int vb, dvv, duu;
        row_block_parts(i, &vb, &dvv, &duu);
        return views_of_vb[vb];
    }
    const DevVT& vt(int view, int j) const { return vt_h[(size_t)view * n + j]; }
};

// geometry / partition construction (host_geometry.cpp)
int geometry_from_desc(const csgd_geometry_desc* d, Geometry* g, std::string* err);
int partition_build(const Geometry* g, const csgd_partition_desc* d, Partition* p,
                    std::string* err);

// work items of one step: every view of every row block in `rows`, clipped to the
// tile's shadow rectangle; returns the number of rays; appends to `out`.
int64_t build_work_items(const Partition& p, const int* rows, int n_rows, int j, int slot,
                         std::vector<WorkItem>* out);

// schedule (host_schedule.cpp)
struct SplitMix64 {
    uint64_t state;
    explicit SplitMix64(uint64_t seed) : state(seed) {}
    uint64_t next();
    double uniform();
};

struct ColumnBatch {
    int j;
    std::vector<std::vector<int>> groups;
};

std::vector<ColumnBatch> epoch_schedule(SplitMix64& rng, const Partition& p,
                                        const csgd_solver_params& prm, int64_t epoch);

}  // namespace csgd
