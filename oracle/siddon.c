/*
 * FP64 oracle for the system matrix of y = Ax + e (Sec. II-A).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark can check the CUDA path against a plain definition.
 *
 * Sec. II-A defines the entry A_i^j as the length of the intersection of ray i
 * with voxel j, computed "for example" with Siddon's method.  This file writes
 * that definition out the textbook way (parametric alpha-merge, Siddon 1985 /
 * Jacobs et al. 1998): collect the parameters at which the line crosses every
 * grid plane inside the grid, sort them, and assign each gap between consecutive
 * parameters to the voxel that contains the gap's midpoint.  No incremental
 * traversal, no tiling, no single precision: a different code path from the GPU.
 *
 * Conventions (the paper is silent on them):
 *   - the grid has dim = 2 or 3 axes, n[a] voxels of edge h along axis a, and
 *     its lower corner at lo[a] (world units); voxel (i0,i1,i2) is the half-open
 *     box [lo + i*h, lo + (i+1)*h) and its linear index is (i2*n1 + i1)*n0 + i0;
 *   - a ray is the full line org + t*dir (t real); the sources and detectors of
 *     the geometries used here lie outside the grid, so line and segment agree;
 *   - a line lying exactly on a grid plane belongs to the voxel on the + side
 *     of that plane (half-open voxels);
 *   - gaps shorter than 1e-12*h are structural zeros and are not emitted.
 *
 * Entry points (all FP64, all loops plain):
 *   oracle_siddon_count  - number of non-zeros of each ray (row of A);
 *   oracle_siddon_fill   - CSR column indices and lengths of those rows;
 *   oracle_project_box   - out_i = sum_{j in box} A_ij x_j       (A_I^J x_J);
 *   oracle_backproject_box - g_j += sum_i A_ij r_i for j in box ((A_I^J)^T r_I);
 *   oracle_count_box     - number of non-zeros of A_I^J (rays x box).
 * A "box" is an index range [blo, bhi) per axis; it selects the column block J.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int dim;
    int64_t n[3];
    double h;
    double lo[3];
} grid_t;

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Callback-free enumeration: fills (col, len) pairs of one ray into the given
 * buffers and returns the count.  alpha is a scratch buffer of at least
 * n0+n1+n2+8 doubles. */
static int64_t ray_entries(const grid_t* g, const double* o, const double* d,
                           double* alpha, int64_t* cols, double* lens) {
    double amin = -INFINITY, amax = INFINITY;
    int64_t fixed_idx[3] = {0, 0, 0};
    int a;
    /* 1. the parameter interval of the line inside the grid's bounding box */
    for (a = 0; a < g->dim; ++a) {
        double blo = g->lo[a], bhi = g->lo[a] + (double)g->n[a] * g->h;
        if (d[a] == 0.0) {
            /* parallel to the planes of this axis: inside iff lo <= o < hi */
            if (!(o[a] >= blo && o[a] < bhi)) return 0;
            fixed_idx[a] = (int64_t)floor((o[a] - blo) / g->h);
            if (fixed_idx[a] >= g->n[a]) fixed_idx[a] = g->n[a] - 1;
        } else {
            double a0 = (blo - o[a]) / d[a];
            double a1 = (bhi - o[a]) / d[a];
            double lo_a = a0 < a1 ? a0 : a1;
            double hi_a = a0 < a1 ? a1 : a0;
            if (lo_a > amin) amin = lo_a;
            if (hi_a < amax) amax = hi_a;
        }
    }
    if (!(amin < amax)) return 0;

    /* 2. parameters of every plane crossing strictly inside (amin, amax) */
    int64_t na = 0;
    alpha[na++] = amin;
    alpha[na++] = amax;
    for (a = 0; a < g->dim; ++a) {
        if (d[a] == 0.0) continue;
        for (int64_t k = 0; k <= g->n[a]; ++k) {
            double plane = g->lo[a] + (double)k * g->h;
            double t = (plane - o[a]) / d[a];
            if (t > amin && t < amax) alpha[na++] = t;
        }
    }
    /* 3. merge = sort */
    qsort(alpha, (size_t)na, sizeof(double), cmp_double);

    /* 4. each gap belongs to the voxel containing its midpoint */
    double dnorm = 0.0;
    for (a = 0; a < g->dim; ++a) dnorm += d[a] * d[a];
    dnorm = sqrt(dnorm);
    int64_t cnt = 0;
    for (int64_t k = 0; k + 1 < na; ++k) {
        double len = (alpha[k + 1] - alpha[k]) * dnorm;
        if (!(len > 1e-12 * g->h)) continue;
        double am = 0.5 * (alpha[k] + alpha[k + 1]);
        int64_t idx[3] = {0, 0, 0};
        int inside = 1;
        for (a = 0; a < g->dim; ++a) {
            if (d[a] == 0.0) {
                idx[a] = fixed_idx[a];
            } else {
                double p = o[a] + am * d[a];
                idx[a] = (int64_t)floor((p - g->lo[a]) / g->h);
            }
            if (idx[a] < 0 || idx[a] >= g->n[a]) inside = 0;
        }
        if (!inside) continue;
        int64_t col = idx[0];
        if (g->dim >= 2) col += g->n[0] * idx[1];
        if (g->dim == 3) col += g->n[0] * g->n[1] * idx[2];
        cols[cnt] = col;
        lens[cnt] = len;
        ++cnt;
    }
    return cnt;
}

static void make_grid(grid_t* g, int dim, const int64_t* n, double h, const double* lo) {
    g->dim = dim;
    for (int a = 0; a < 3; ++a) {
        g->n[a] = a < dim ? n[a] : 1;
        g->lo[a] = a < dim ? lo[a] : 0.0;
    }
    g->h = h;
}

static int64_t max_entries(const grid_t* g) {
    return g->n[0] + g->n[1] + g->n[2] + 8;
}

static int in_box(const grid_t* g, int64_t col, const int64_t* blo, const int64_t* bhi) {
    int64_t i0 = col % g->n[0];
    int64_t rest = col / g->n[0];
    int64_t i1 = rest % g->n[1];
    int64_t i2 = rest / g->n[1];
    int64_t idx[3] = {i0, i1, i2};
    for (int a = 0; a < g->dim; ++a)
        if (idx[a] < blo[a] || idx[a] >= bhi[a]) return 0;
    return 1;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

int64_t oracle_siddon_count(int dim, const int64_t* n, double h, const double* lo,
                            int64_t n_rays, const double* org, const double* dir,
                            int64_t* counts) {
    grid_t g;
    make_grid(&g, dim, n, h, lo);
    int64_t cap = max_entries(&g);
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        double* alpha = (double*)malloc(sizeof(double) * (size_t)cap);
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        double* lens = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_rays; ++i) {
            counts[i] = ray_entries(&g, org + 3 * i, dir + 3 * i, alpha, cols, lens);
            total += counts[i];
        }
        free(alpha);
        free(cols);
        free(lens);
    }
    return total;
}

void oracle_siddon_fill(int dim, const int64_t* n, double h, const double* lo,
                        int64_t n_rays, const double* org, const double* dir,
                        const int64_t* offsets, int64_t* out_cols, double* out_vals) {
    grid_t g;
    make_grid(&g, dim, n, h, lo);
    int64_t cap = max_entries(&g);
#pragma omp parallel
    {
        double* alpha = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_rays; ++i) {
            ray_entries(&g, org + 3 * i, dir + 3 * i, alpha, out_cols + offsets[i],
                        out_vals + offsets[i]);
        }
        free(alpha);
    }
}

void oracle_project_box(int dim, const int64_t* n, double h, const double* lo,
                        int64_t n_rays, const double* org, const double* dir,
                        const int64_t* blo, const int64_t* bhi, const double* x,
                        double* out) {
    grid_t g;
    make_grid(&g, dim, n, h, lo);
    int64_t cap = max_entries(&g);
#pragma omp parallel
    {
        double* alpha = (double*)malloc(sizeof(double) * (size_t)cap);
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        double* lens = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_rays; ++i) {
            int64_t c = ray_entries(&g, org + 3 * i, dir + 3 * i, alpha, cols, lens);
            double s = 0.0;
            for (int64_t k = 0; k < c; ++k)
                if (in_box(&g, cols[k], blo, bhi)) s += lens[k] * x[cols[k]];
            out[i] = s;
        }
        free(alpha);
        free(cols);
        free(lens);
    }
}

int64_t oracle_count_box(int dim, const int64_t* n, double h, const double* lo,
                         int64_t n_rays, const double* org, const double* dir,
                         const int64_t* blo, const int64_t* bhi) {
    grid_t g;
    make_grid(&g, dim, n, h, lo);
    int64_t cap = max_entries(&g);
    int64_t total = 0;
#pragma omp parallel reduction(+ : total)
    {
        double* alpha = (double*)malloc(sizeof(double) * (size_t)cap);
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        double* lens = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_rays; ++i) {
            int64_t c = ray_entries(&g, org + 3 * i, dir + 3 * i, alpha, cols, lens);
            for (int64_t k = 0; k < c; ++k) total += in_box(&g, cols[k], blo, bhi);
        }
        free(alpha);
        free(cols);
        free(lens);
    }
    return total;
}

void oracle_backproject_box(int dim, const int64_t* n, double h, const double* lo,
                            int64_t n_rays, const double* org, const double* dir,
                            const int64_t* blo, const int64_t* bhi, const double* r,
                            double* gout) {
    grid_t g;
    make_grid(&g, dim, n, h, lo);
    int64_t cap = max_entries(&g);
    int64_t bw[3] = {1, 1, 1}, bl[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        bl[a] = blo[a];
        bw[a] = bhi[a] - blo[a];
        if (bw[a] <= 0) return;
    }
    int64_t nbox = bw[0] * bw[1] * bw[2];
    int nt = oracle_num_threads();
    /* per-thread partial sums over the box, added afterwards in thread order so
     * that the result does not depend on scheduling */
    double* part = (double*)calloc((size_t)nt * (size_t)nbox, sizeof(double));
    int64_t chunk = (n_rays + nt - 1) / (nt > 0 ? nt : 1);
#pragma omp parallel num_threads(nt)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* alpha = (double*)malloc(sizeof(double) * (size_t)cap);
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
        double* lens = (double*)malloc(sizeof(double) * (size_t)cap);
        double* mine = part + (int64_t)tid * nbox;
        int64_t i0 = (int64_t)tid * chunk, i1 = i0 + chunk;
        if (i1 > n_rays) i1 = n_rays;
        for (int64_t i = i0; i < i1; ++i) {
            int64_t c = ray_entries(&g, org + 3 * i, dir + 3 * i, alpha, cols, lens);
            for (int64_t k = 0; k < c; ++k) {
                if (!in_box(&g, cols[k], blo, bhi)) continue;
                int64_t v0 = cols[k] % g.n[0];
                int64_t rest = cols[k] / g.n[0];
                int64_t v1 = rest % g.n[1], v2 = rest / g.n[1];
                int64_t local = ((v2 - bl[2]) * bw[1] + (v1 - bl[1])) * bw[0] + (v0 - bl[0]);
                mine[local] += lens[k] * r[i];
            }
        }
        free(alpha);
        free(cols);
        free(lens);
    }
    for (int t = 0; t < nt; ++t) {
        const double* p = part + (int64_t)t * nbox;
        for (int64_t l = 0; l < nbox; ++l) {
            int64_t v0 = l % bw[0];
            int64_t rest = l / bw[0];
            int64_t v1 = rest % bw[1], v2 = rest / bw[1];
            int64_t col = ((v2 + bl[2]) * g.n[1] + (v1 + bl[1])) * g.n[0] + (v0 + bl[0]);
            gout[col] += p[l];
        }
    }
    free(part);
}
