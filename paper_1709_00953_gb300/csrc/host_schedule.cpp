// Random block choice of Alg. 3 / Alg. 4 and the mixed weights of Sec. III-D.
//
// The paper does not name a generator.  The rules below are fixed so that any
// implementation of them (this one, or an independent one used as a check)
// produces the same schedule draw for draw:
//   - SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), u = (next >> 11) * 2^-53;
//   - per epoch: Fisher-Yates permutation of the n column blocks (i = n-1 .. 1,
//     swap with floor(u (i+1))), first ceil(gamma n) kept in order;
//   - per column block: ceil(alpha m / s) groups of s draws without
//     replacement; a draw walks the remaining blocks in index order and takes
//     the first whose running weight sum exceeds u * (remaining total); drawing
//     stops when the remaining total is not positive;
//   - weights: P(I,J) (importance), 1 (uniform), P + theta (P_max - P) with
//     theta = min(1, epoch * theta_step) and P_max over the row blocks of the
//     same view set (mixed); sequential = Alg. 2's fixed order.
// FP64 sums are accumulated in index order (compiled with -ffp-contract=off) so
// that the comparisons are reproducible across machines.
#include <math.h>

#include <algorithm>

#include "host.h"

namespace csgd {

uint64_t SplitMix64::next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double SplitMix64::uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }

static int ceil_count(double frac, double total, double div) {
    double v = ceil(frac * total / div - 1e-9);
    return v < 0 ? 0 : (int)v;
}

std::vector<ColumnBatch> epoch_schedule(SplitMix64& rng, const Partition& p,
                                        const csgd_solver_params& prm, int64_t epoch) {
    const int n = p.n, m = p.m;
    const int s = prm.group_size < 1 ? 1 : prm.group_size;
    std::vector<ColumnBatch> out;
    int ncols = ceil_count(prm.gamma, n, 1.0);
    std::vector<int> cols;
    if (prm.sampling == CSGD_SAMPLE_SEQUENTIAL) {
        for (int j = 0; j < std::min(ncols, n); ++j) cols.push_back(j);
    } else {
        std::vector<int> perm(n);
        for (int j = 0; j < n; ++j) perm[j] = j;
        for (int i = n - 1; i >= 1; --i) {
            int k = (int)(rng.uniform() * (double)(i + 1));
            std::swap(perm[i], perm[k]);
        }
        for (int j = 0; j < std::min(ncols, n); ++j) cols.push_back(perm[j]);
    }
    const int n_groups = ceil_count(prm.alpha, m, s);
    std::vector<double> w(m);
    for (int j : cols) {
        ColumnBatch cb;
        cb.j = j;
        if (prm.sampling == CSGD_SAMPLE_SEQUENTIAL) {
            int total = std::min(n_groups * s, m);
            for (int g0 = 0; g0 < total; g0 += s) {
                std::vector<int> grp;
                for (int i = g0; i < std::min(g0 + s, total); ++i) grp.push_back(i);
                cb.groups.push_back(grp);
            }
            out.push_back(cb);
            continue;
        }
        // weights of every row block for this column block
        for (int i = 0; i < m; ++i) {
            double pij = p.P[(size_t)i * n + j];
            if (prm.sampling == CSGD_SAMPLE_UNIFORM) w[i] = 1.0;
            else w[i] = pij;
        }
        if (prm.sampling == CSGD_SAMPLE_MIXED) {
            double theta = std::min(1.0, (double)epoch * prm.theta_step);
            for (int i = 0; i < m; ++i) {
                int vb, a, b;
                p.row_block_parts(i, &vb, &a, &b);
                double pmax = 0.0;
                for (int i2 = vb * p.du * p.dv; i2 < (vb + 1) * p.du * p.dv; ++i2)
                    pmax = std::max(pmax, p.P[(size_t)i2 * n + j]);
                double pij = p.P[(size_t)i * n + j];
                w[i] = pij + theta * (pmax - pij);
            }
        }
        std::vector<int> remaining(m);
        for (int i = 0; i < m; ++i) remaining[i] = i;
        bool done = false;
        for (int gi = 0; gi < n_groups && !done; ++gi) {
            std::vector<int> grp;
            for (int d = 0; d < s; ++d) {
                double total = 0.0;
                for (int i : remaining) total += w[i];
                if (!(total > 0.0)) {
                    done = true;
                    break;
                }
                double thr = rng.uniform() * total;
                double acc = 0.0;
                int pick = -1;
                for (int i : remaining) {
                    acc += w[i];
                    if (acc > thr) {
                        pick = i;
                        break;
                    }
                }
                if (pick < 0) {
                    for (int i : remaining)
                        if (w[i] > 0.0) pick = i;
                }
                remaining.erase(std::find(remaining.begin(), remaining.end(), pick));
                grp.push_back(pick);
            }
            if (!grp.empty()) cb.groups.push_back(grp);
        }
        out.push_back(cb);
    }
    return out;
}

}  // namespace csgd
