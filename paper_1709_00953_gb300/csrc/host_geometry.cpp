// Geometry, block partition (Eq. e1, Sec. II-D) and importance table (Alg. 3).
//
// Everything here runs once per scan on the host in FP64.  Its products are
//   - the importance table P(I,J) = P_S(I,J) / P_T(J) of Alg. 3, where P_S is the
//     area of tile J's shadow on the detector sub-area of row block I summed over
//     I's views and P_T the area of its shadow on the whole detector summed over
//     all views (bin units; the shadow is the exact interval / convex hull of the
//     projected tile corners);
//   - the per (view, tile) ray constants and shadow rectangles the kernels use.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>

#include "host.h"

namespace csgd {

static inline double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

int geometry_from_desc(const csgd_geometry_desc* d, Geometry* g, std::string* err) {
    if (!d) {
        *err = "geometry desc is NULL";
        return CSGD_ERR_INVALID_ARG;
    }
    if (d->kind < CSGD_PARALLEL_2D || d->kind > CSGD_CUSTOM_3D) {
        *err = "unknown geometry kind";
        return CSGD_ERR_INVALID_ARG;
    }
    g->kind = d->kind;
    g->dim = (d->kind <= CSGD_FAN_2D_CURVED) ? 2 : 3;
    g->n[0] = d->n[0];
    g->n[1] = d->n[1];
    g->n[2] = g->dim == 3 ? d->n[2] : 1;
    for (int a = 0; a < 3; ++a)
        if (g->n[a] < 1 || g->n[a] > (1 << 16)) {
            *err = "voxel counts must be in [1, 65536]";
            return CSGD_ERR_INVALID_ARG;
        }
    // the kernels index voxels (and a tile's voxels) with 32-bit integers
    if ((int64_t)g->n[0] * g->n[1] * g->n[2] >= ((int64_t)1 << 31)) {
        *err = "too many voxels (the grid must hold fewer than 2^31)";
        return CSGD_ERR_INVALID_ARG;
    }
    if (!(d->h > 0) || !std::isfinite(d->h)) {
        *err = "voxel edge h must be positive";
        return CSGD_ERR_INVALID_ARG;
    }
    g->h = d->h;
    if (d->n_views < 1) {
        *err = "n_views must be positive";
        return CSGD_ERR_INVALID_ARG;
    }
    g->n_views = d->n_views;
    g->nu = d->nu;
    g->nv = g->dim == 3 ? d->nv : 1;
    if (g->nu < 1 || g->nv < 1 || g->nu > 32768 || g->nv > 32768) {
        *err = "detector bin counts must be in [1, 32768]";
        return CSGD_ERR_INVALID_ARG;
    }
    if (g->n_rays() >= ((int64_t)1 << 31)) {
        *err = "too many rays";
        return CSGD_ERR_INVALID_ARG;
    }
    g->pu = d->pu;
    g->pv = g->dim == 3 ? d->pv : 1.0;
    if (!(g->pu > 0) || !(g->pv > 0)) {
        *err = "detector pitch must be positive";
        return CSGD_ERR_INVALID_ARG;
    }
    g->sod = d->sod;
    g->sdd = d->sdd;
    g->frames.resize(g->n_views);
    // circumscribed radius of the grid
    double R = 0.5 * g->h * sqrt((double)g->n[0] * g->n[0] + (double)g->n[1] * g->n[1] +
                                 (g->dim == 3 ? (double)g->n[2] * g->n[2] : 0.0));
    if (d->kind == CSGD_CUSTOM_3D) {
        if (!d->poses) {
            *err = "CUSTOM_3D needs poses";
            return CSGD_ERR_INVALID_ARG;
        }
        g->poses.assign(d->poses, d->poses + 12 * (size_t)d->n_views);
        for (int v = 0; v < g->n_views; ++v) {
            const double* p = &g->poses[12 * (size_t)v];
            Frame& f = g->frames[v];
            double cs[3];
            for (int a = 0; a < 3; ++a) {
                f.S[a] = p[a];
                cs[a] = p[3 + a] - p[a];
                f.eu[a] = p[6 + a];
                f.ev[a] = p[9 + a];
            }
            f.sdd = sqrt(dot3(cs, cs));
            if (!(f.sdd > 0)) {
                *err = "pose with detector centre at the source";
                return CSGD_ERR_INVALID_ARG;
            }
            for (int a = 0; a < 3; ++a) f.dc[a] = cs[a] / f.sdd;
            if (fabs(dot3(f.eu, f.eu) - 1) > 1e-9 || fabs(dot3(f.ev, f.ev) - 1) > 1e-9 ||
                fabs(dot3(f.eu, f.ev)) > 1e-9 || fabs(dot3(f.eu, f.dc)) > 1e-9 ||
                fabs(dot3(f.ev, f.dc)) > 1e-9) {
                *err = "pose axes must be orthonormal and perpendicular to C - S";
                return CSGD_ERR_INVALID_ARG;
            }
            if (!(sqrt(dot3(f.S, f.S)) > R)) {
                *err = "source inside the grid's circumscribed sphere";
                return CSGD_ERR_INVALID_ARG;
            }
        }
        return CSGD_OK;
    }
    if (!d->angles) {
        *err = "angles are required";
        return CSGD_ERR_INVALID_ARG;
    }
    g->angles.assign(d->angles, d->angles + d->n_views);
    if (d->kind != CSGD_PARALLEL_2D) {
        if (!(g->sod > R)) {
            *err = "sod must exceed the grid's circumscribed radius";
            return CSGD_ERR_INVALID_ARG;
        }
        if (d->kind != CSGD_FAN_2D_CURVED && !(g->sdd > 0)) {
            *err = "sdd must be positive";
            return CSGD_ERR_INVALID_ARG;
        }
        if (d->kind == CSGD_FAN_2D_CURVED && !(g->pu * g->nu < 3.1)) {
            *err = "curved detector spans more than pi";
            return CSGD_ERR_INVALID_ARG;
        }
    }
    for (int v = 0; v < g->n_views; ++v) {
        double t = g->angles[v];
        if (!std::isfinite(t)) {
            *err = "angles must be finite";
            return CSGD_ERR_INVALID_ARG;
        }
        Frame& f = g->frames[v];
        // a view at a multiple of 90 degrees is axis-aligned: cos and sin below
        // 1e-12 (cos(pi/2) evaluates to 6e-17) are exactly 0, so that rays along an
        // axis have no spurious 1e-16 tilt whose face crossings no FP32 set-up
        // could place
        double c = cos(t), s = sin(t);
        if (std::fabs(c) < 1e-12) c = 0.0;
        if (std::fabs(s) < 1e-12) s = 0.0;
        f.dc[0] = -c; f.dc[1] = -s; f.dc[2] = 0;
        f.eu[0] = -s; f.eu[1] = c; f.eu[2] = 0;
        f.ev[0] = 0; f.ev[1] = 0; f.ev[2] = 1;
        f.S[0] = g->sod * c; f.S[1] = g->sod * s; f.S[2] = 0;
        f.sdd = g->sdd;
    }
    return CSGD_OK;
}

// ---------------------------------------------------------------------------
// detector coordinates of world points (bin k covers [k, k+1))
// ---------------------------------------------------------------------------
static void detector_coord(const Geometry& g, const Frame& f, const double* P, double* wu,
                           double* wv) {
    if (g.kind == CSGD_PARALLEL_2D) {
        *wu = dot3(P, f.eu) / g.pu + 0.5 * g.nu;
        *wv = 0.5;
        return;
    }
    double rel[3] = {P[0] - f.S[0], P[1] - f.S[1], P[2] - f.S[2]};
    double depth = dot3(rel, f.dc);
    if (g.kind == CSGD_FAN_2D_CURVED) {
        *wu = atan2(dot3(rel, f.eu), depth) / g.pu + 0.5 * g.nu;
        *wv = 0.5;
        return;
    }
    double lam = f.sdd / depth;
    *wu = lam * dot3(rel, f.eu) / g.pu + 0.5 * g.nu;
    *wv = g.dim == 3 ? lam * dot3(rel, f.ev) / g.pv + 0.5 * g.nv : 0.5;
}

// ---------------------------------------------------------------------------
// 2D polygon helpers (convex hull, rectangle clip, area)
// ---------------------------------------------------------------------------
struct P2 {
    double x, y;
};

static double cross(const P2& o, const P2& a, const P2& b) {
    return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
}

static std::vector<P2> hull(std::vector<P2> pts) {
    std::sort(pts.begin(), pts.end(), [](const P2& a, const P2& b) {
        return a.x < b.x || (a.x == b.x && a.y < b.y);
    });
    pts.erase(std::unique(pts.begin(), pts.end(),
                          [](const P2& a, const P2& b) { return a.x == b.x && a.y == b.y; }),
              pts.end());
    if (pts.size() < 3) return pts;
    std::vector<P2> h(2 * pts.size());
    size_t k = 0;
    for (size_t i = 0; i < pts.size(); ++i) {
        while (k >= 2 && cross(h[k - 2], h[k - 1], pts[i]) <= 0) --k;
        h[k++] = pts[i];
    }
    for (size_t i = pts.size() - 1, t = k + 1; i-- > 0;) {
        while (k >= t && cross(h[k - 2], h[k - 1], pts[i]) <= 0) --k;
        h[k++] = pts[i];
    }
    h.resize(k - 1);
    return h;
}

static std::vector<P2> clip_half(const std::vector<P2>& in, int axis, double c, bool keep_ge) {
    std::vector<P2> out;
    size_t n = in.size();
    for (size_t k = 0; k < n; ++k) {
        const P2& cur = in[k];
        const P2& prev = in[(k + n - 1) % n];
        double vc = axis == 0 ? cur.x : cur.y;
        double vp = axis == 0 ? prev.x : prev.y;
        bool ic = keep_ge ? vc >= c : vc <= c;
        bool ip = keep_ge ? vp >= c : vp <= c;
        if (ic != ip) {
            double t = (c - vp) / (vc - vp);
            P2 q{prev.x + (cur.x - prev.x) * t, prev.y + (cur.y - prev.y) * t};
            if (axis == 0) q.x = c; else q.y = c;
            out.push_back(q);
        }
        if (ic) out.push_back(cur);
    }
    return out;
}

static double area(const std::vector<P2>& p) {
    if (p.size() < 3) return 0.0;
    double s = 0.0;
    for (size_t k = 0; k < p.size(); ++k) {
        const P2& a = p[k];
        const P2& b = p[(k + 1) % p.size()];
        s += a.x * b.y - a.y * b.x;
    }
    return 0.5 * fabs(s);
}

static double clipped_area(const std::vector<P2>& poly, double x0, double x1, double y0,
                           double y1) {
    std::vector<P2> q = poly;
    q = clip_half(q, 0, x0, true);
    if (q.empty()) return 0.0;
    q = clip_half(q, 0, x1, false);
    if (q.empty()) return 0.0;
    q = clip_half(q, 1, y0, true);
    if (q.empty()) return 0.0;
    q = clip_half(q, 1, y1, false);
    return area(q);
}

// ---------------------------------------------------------------------------
// partition
// ---------------------------------------------------------------------------
static std::vector<int> splits(int n, int parts) {
    std::vector<int> e(parts + 1);
    for (int k = 0; k <= parts; ++k) e[k] = (int)(((int64_t)k * n) / parts);
    return e;
}

static void tile_corners(const Geometry& g, const DevTile& t, std::vector<std::array<double, 3>>* c);

int partition_build(const Geometry* gp, const csgd_partition_desc* d, Partition* p,
                    std::string* err) {
    const Geometry& g = *gp;
    if (!d) {
        *err = "partition desc is NULL";
        return CSGD_ERR_INVALID_ARG;
    }
    p->g = gp;
    for (int a = 0; a < 3; ++a) {
        int t = a < g.dim ? d->tiles[a] : 1;
        if (t < 1 || t > g.n[a]) {
            *err = "tiles per axis must be in [1, voxels along that axis]";
            return CSGD_ERR_INVALID_ARG;
        }
        p->tiles[a] = t;
        p->edges[a] = splits(g.n[a], t);
    }
    p->du = d->det_blocks_u;
    p->dv = g.dim == 3 ? d->det_blocks_v : 1;
    if (p->du < 1 || p->du > g.nu || p->dv < 1 || p->dv > g.nv) {
        *err = "detector sub-areas per axis must be in [1, bins along that axis]";
        return CSGD_ERR_INVALID_ARG;
    }
    p->u_edges = splits(g.nu, p->du);
    p->v_edges = splits(g.nv, p->dv);
    p->view_block_of.assign(g.n_views, 0);
    if (d->view_block_of) {
        int mx = -1;
        for (int v = 0; v < g.n_views; ++v) {
            int b = d->view_block_of[v];
            if (b < 0 || b >= g.n_views) {
                *err = "view_block_of entries must be in [0, n_views)";
                return CSGD_ERR_INVALID_ARG;
            }
            p->view_block_of[v] = b;
            mx = std::max(mx, b);
        }
        p->vb_count = mx + 1;
    } else {
        if (d->view_blocks < 1 || d->view_blocks > g.n_views) {
            *err = "view_blocks must be in [1, n_views]";
            return CSGD_ERR_INVALID_ARG;
        }
        p->vb_count = d->view_blocks;
        std::vector<int> e = splits(g.n_views, p->vb_count);
        for (int b = 0; b < p->vb_count; ++b)
            for (int v = e[b]; v < e[b + 1]; ++v) p->view_block_of[v] = b;
    }
    p->views_of_vb.assign(p->vb_count, {});
    for (int v = 0; v < g.n_views; ++v) p->views_of_vb[p->view_block_of[v]].push_back(v);
    for (int b = 0; b < p->vb_count; ++b)
        if (p->views_of_vb[b].empty()) {
            *err = "every view set must hold at least one view";
            return CSGD_ERR_INVALID_ARG;
        }
    p->m = p->vb_count * p->du * p->dv;
    p->n = p->tiles[0] * p->tiles[1] * p->tiles[2];
    if ((int64_t)p->m * p->n > (int64_t)1 << 28 || p->n > 65535 || p->m > 65534) {
        *err = "too many blocks (at most 65535 tiles and 65534 row blocks)";
        return CSGD_ERR_INVALID_ARG;
    }

    // ---- tiles ----
    const double hv = 1.0;  // device tables are in voxel units
    p->tiles_h.resize(p->n);
    int64_t voff = 0;
    p->max_tile_voxels = 0;
    for (int j = 0; j < p->n; ++j) {
        int tx = j % p->tiles[0], ty = (j / p->tiles[0]) % p->tiles[1],
            tz = j / (p->tiles[0] * p->tiles[1]);
        int tc[3] = {tx, ty, tz};
        DevTile& t = p->tiles_h[j];
        int64_t nv = 1;
        for (int a = 0; a < 3; ++a) {
            t.lo[a] = p->edges[a][tc[a]];
            t.n[a] = p->edges[a][tc[a] + 1] - p->edges[a][tc[a]];
            t.T[a] = (float)(a < g.dim ? (-0.5 * g.n[a] + t.lo[a] + 0.5 * t.n[a]) * hv : 0.0);
            nv *= t.n[a];
        }
        t.voff = voff;
        voff += nv;
        p->max_tile_voxels = std::max(p->max_tile_voxels, nv);
    }

    // ---- views (FP32, voxel units) ----
    p->views_h.resize(g.n_views);
    p->views64_h.resize(g.n_views);
    for (int v = 0; v < g.n_views; ++v) {
        const Frame& f = g.frames[v];
        DevView& dv = p->views_h[v];
        DevView64& d64 = p->views64_h[v];
        memset(&dv, 0, sizeof(dv));
        for (int a = 0; a < 3; ++a) {
            d64.S[a] = f.S[a] / g.h;
            d64.dc[a] = f.dc[a];
            d64.eu[a] = f.eu[a];
            d64.ev[a] = f.ev[a];
            dv.S[a] = (float)d64.S[a];
            dv.dc[a] = (float)f.dc[a];
            dv.eu[a] = (float)f.eu[a];
            dv.ev[a] = (float)f.ev[a];
        }
        d64.sdd = f.sdd / g.h;
        dv.sdd = (float)d64.sdd;
    }

    // ---- per (view, tile): shadow, P tables, ray constants ----
    p->PS.assign((size_t)p->m * p->n, 0.0);
    p->PT.assign(p->n, 0.0);
    p->vt_h.resize((size_t)g.n_views * p->n);
    const double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
    const double pu_v = g.kind == CSGD_FAN_2D_CURVED ? g.pu : g.pu / g.h;  // voxel units
    const double pv_v = g.pv / g.h;
    int64_t zoff = 0;
    std::vector<std::array<double, 3>> corners;
    for (int v = 0; v < g.n_views; ++v) {
        const Frame& fw = g.frames[v];
        // frame in voxel units
        Frame f = fw;
        for (int a = 0; a < 3; ++a) f.S[a] = fw.S[a] / g.h;
        f.sdd = fw.sdd / g.h;
        int vb = p->view_block_of[v];
        for (int j = 0; j < p->n; ++j) {
            const DevTile& t = p->tiles_h[j];
            tile_corners(g, t, &corners);
            // shadow in bin coordinates (world units in, same as voxel units scaled)
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            std::vector<P2> pts;
            for (auto& c : corners) {
                double wc[3] = {c[0] * g.h, c[1] * g.h, c[2] * g.h};
                double wu, wv;
                detector_coord(g, fw, wc, &wu, &wv);
                umin = std::min(umin, wu);
                umax = std::max(umax, wu);
                vmin = std::min(vmin, wv);
                vmax = std::max(vmax, wv);
                pts.push_back({wu, wv});
            }
            // importance areas
            std::vector<P2> poly;
            if (g.dim == 3) poly = hull(pts);
            // overlaps below 1e-9 bin units are rounding slivers (a shadow edge on
            // a sub-area boundary) and count as none
            auto overlap = [&](double u0, double u1, double v0, double v1) {
                double a = g.dim == 2 ? std::max(0.0, std::min(umax, u1) - std::max(umin, u0))
                                      : clipped_area(poly, u0, u1, v0, v1);
                return a > 1e-9 ? a : 0.0;
            };
            p->PT[j] += overlap(0, g.nu, 0, g.nv);
            for (int dvv = 0; dvv < p->dv; ++dvv)
                for (int duu = 0; duu < p->du; ++duu) {
                    int i = (vb * p->dv + dvv) * p->du + duu;
                    p->PS[(size_t)i * p->n + j] +=
                        overlap(p->u_edges[duu], p->u_edges[duu + 1], p->v_edges[dvv],
                                p->v_edges[dvv + 1]);
                }
            // conservative rectangle of bins whose centre lines can meet the tile
            DevVT& e = p->vt_h[(size_t)v * p->n + j];
            memset(&e, 0, sizeof(e));
            int u0 = (int)std::max(0.0, ceil(umin - 0.5) - 1.0);
            int u1 = (int)std::min((double)g.nu, floor(umax - 0.5) + 2.0);
            int v0 = 0, v1 = 1;
            if (g.dim == 3) {
                v0 = (int)std::max(0.0, ceil(vmin - 0.5) - 1.0);
                v1 = (int)std::min((double)g.nv, floor(vmax - 0.5) + 2.0);
            }
            if (u1 <= u0 || v1 <= v0) {
                u0 = u1 = v0 = v1 = 0;
            }
            e.u0 = u0;
            e.u1 = u1;
            e.v0 = v0;
            e.v1 = v1;
            e.zoff = zoff;
            zoff += (int64_t)(u1 - u0) * (v1 - v0);
            // Half-width of a voxel's shadow, in bins.  Neighbouring lines of one
            // detector row are at least `spacing` apart everywhere in the tile (lines
            // of a fan meet at the source at an angle of at least `ang` per bin, and
            // every point of the tile is at least dmin from the source), so the lines
            // within half a voxel diagonal of a voxel's centre lie within
            // (diagonal / 2) / spacing bins of the line through the centre.
            {
                double dmin = 0.0;
                if (g.kind != CSGD_PARALLEL_2D) {
                    double d2 = 0.0;
                    for (int a = 0; a < g.dim; ++a) {
                        double lo = t.T[a] - 0.5 * t.n[a], hi = t.T[a] + 0.5 * t.n[a];
                        double c = std::min(std::max(f.S[a], lo), hi);
                        d2 += (f.S[a] - c) * (f.S[a] - c);
                    }
                    dmin = sqrt(d2);
                }
                double umax = 0.5 * g.nu * pu_v;
                double vmax = g.dim == 3 ? 0.5 * g.nv * pv_v : 0.0;
                auto spacing_of = [&](double pitch) {
                    if (g.kind == CSGD_PARALLEL_2D) return pitch;
                    double ang = g.kind == CSGD_FAN_2D_CURVED
                                     ? pitch
                                     : pitch * f.sdd / (f.sdd * f.sdd + umax * umax + vmax * vmax);
                    return dmin * sin(std::min(ang, 1.0));
                };
                double half_diag = 0.5 * sqrt((double)g.dim) * 1.02;
                double su = spacing_of(pu_v);
                e.hw_u = (float)(su > 0 ? half_diag / su + 0.01 : 1e6);
                if (g.dim == 3) {
                    double sv = spacing_of(pv_v);
                    e.hw_v = (float)(sv > 0 ? half_diag / sv + 0.01 : 1e6);
                } else {
                    e.hw_v = 0.f;
                }
            }
            // ray constants (voxel units, tile-centred)
            double T[3] = {t.T[0], t.T[1], t.T[2]};
            if (g.kind == CSGD_PARALLEL_2D) {
                double L = dot3(T, f.eu);
                int k0 = (int)llround(L / pu_v + cu);
                double s0 = (k0 - cu) * pu_v;
                for (int a = 0; a < 3; ++a) {
                    e.B[a] = (float)((s0 - L) * f.eu[a]);
                    e.U[a] = (float)(pu_v * f.eu[a]);
                    e.V[a] = 0.f;
                }
                e.k0u = k0;
                e.k0v = 0;
            } else {
                double rel[3] = {T[0] - f.S[0], T[1] - f.S[1], T[2] - f.S[2]};
                double D = dot3(rel, f.dc);
                double Lu = dot3(rel, f.eu);
                double Lv = dot3(rel, f.ev);
                if (g.kind == CSGD_FAN_2D_CURVED) {
                    int k0 = (int)llround(atan2(Lu, D) / pu_v + cu);
                    double g0 = (k0 - cu) * pu_v;
                    double off = D * tan(g0) - Lu;
                    for (int a = 0; a < 3; ++a) {
                        e.B[a] = (float)(off * f.eu[a]);
                        e.V[a] = 0.f;
                    }
                    e.U[0] = (float)D;
                    e.U[1] = (float)(1.0 / cos(g0));
                    e.U[2] = 0.f;
                    e.k0u = k0;
                    e.k0v = 0;
                } else {
                    double lam = D / f.sdd;
                    int k0u = (int)llround(Lu / (lam * pu_v) + cu);
                    int k0v = g.dim == 3 ? (int)llround(Lv / (lam * pv_v) + cv) : 0;
                    double ou = lam * (k0u - cu) * pu_v - Lu;
                    double ov = g.dim == 3 ? lam * (k0v - cv) * pv_v - Lv : 0.0;
                    for (int a = 0; a < 3; ++a) {
                        e.B[a] = (float)(ou * f.eu[a] + ov * f.ev[a]);
                        e.U[a] = (float)(lam * pu_v * f.eu[a]);
                        e.V[a] = (float)(g.dim == 3 ? lam * pv_v * f.ev[a] : 0.0);
                    }
                    e.k0u = k0u;
                    e.k0v = k0v;
                }
            }
        }
    }
    p->z_floats = zoff;
    p->P.assign((size_t)p->m * p->n, 0.0);
    for (int i = 0; i < p->m; ++i)
        for (int j = 0; j < p->n; ++j)
            if (p->PT[j] > 0) p->P[(size_t)i * p->n + j] = p->PS[(size_t)i * p->n + j] / p->PT[j];

    // ---- device-facing header ----
    DevGeom& dg = p->dg;
    dg.kind = g.kind;
    dg.dim = g.dim;
    dg.nx = g.n[0];
    dg.ny = g.n[1];
    dg.nz = g.n[2];
    dg.nu = g.nu;
    dg.nv = g.nv;
    dg.n_views = g.n_views;
    dg.n_tiles = p->n;
    dg.pu = (float)pu_v;
    dg.pv = (float)pv_v;
    dg.pu_d = pu_v;
    dg.pv_d = pv_v;
    dg.cu = (float)cu;
    dg.cv = (float)cv;
    dg.inv_pu = (float)(1.0 / pu_v);
    dg.inv_pv = (float)(1.0 / pv_v);
    dg.h = (float)g.h;
    return CSGD_OK;
}

static void tile_corners(const Geometry& g, const DevTile& t,
                         std::vector<std::array<double, 3>>* c) {
    c->clear();
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        if (a < g.dim) {
            lo[a] = -0.5 * g.n[a] + t.lo[a];
            hi[a] = lo[a] + t.n[a];
        } else {
            lo[a] = hi[a] = 0.0;
        }
    }
    int nz = g.dim == 3 ? 2 : 1;
    for (int ix = 0; ix < 2; ++ix)
        for (int iy = 0; iy < 2; ++iy)
            for (int iz = 0; iz < nz; ++iz)
                c->push_back({ix ? hi[0] : lo[0], iy ? hi[1] : lo[1], iz ? hi[2] : lo[2]});
}

int64_t build_work_items(const Partition& p, const int* rows, int n_rows, int j, int slot,
                         std::vector<WorkItem>* out) {
    int64_t rays = 0;
    for (int r = 0; r < n_rows; ++r) {
        int i = rows[r];
        int su0, su1, sv0, sv1;
        p.subrect(i, &su0, &su1, &sv0, &sv1);
        for (int v : p.views_of(i)) {
            const DevVT& e = p.vt(v, j);
            int u0 = std::max(su0, e.u0), u1 = std::min(su1, e.u1);
            int v0 = std::max(sv0, e.v0), v1 = std::min(sv1, e.v1);
            if (u1 <= u0 || v1 <= v0) continue;
            WorkItem w;
            w.view = v;
            w.slot = slot;
            w.u0 = u0;
            w.u1 = u1;
            w.v0 = v0;
            w.v1 = v1;
            w.ray_off = rays;
            rays += (int64_t)(u1 - u0) * (v1 - v0);
            out->push_back(w);
        }
    }
    return rays;
}

}  // namespace csgd
