"""Random choice of (I, J) blocks: Alg. 2, Alg. 3, Alg. 4 and mixed sampling (oracle).

Test infrastructure only (see the package docstring).

The paper names the choices but not the random number generator.  So that the
library and this oracle can agree draw for draw, both implement, each from its
published definition, the same generator and the same way of consuming it:

* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15,
  then the 64-bit finaliser; a uniform double is (next() >> 11) * 2^-53.
* Column blocks (Alg. 3: "select a column block J randomly", gamma n of them
  per epoch): a Fisher-Yates shuffle of 0..n-1 (i from n-1 down to 1, swap
  with floor(u (i+1))), keeping the first ceil(gamma n) entries in order.
* Row blocks for one column block (Alg. 3 inner loop; Alg. 4 groups of s):
  ceil(alpha m / s) groups of s draws each, without replacement.  A draw takes
  u, walks the remaining blocks in index order accumulating their weights, and
  takes the first block whose running sum exceeds u * (sum of remaining
  weights).  Drawing stops early when no block with positive weight is left;
  a partly filled last group is kept.
* Weights: importance w = P(I, J) (Alg. 3, Alg. 4); uniform w = 1 (the equal
  probability choice of Sec. II-C); mixed (Sec. III-D)
  w = P + theta_e (P_max - P) where P_max is the largest P(., J) among the row
  blocks that share the views of I, theta_e = min(1, e * theta_step) in epoch e
  (counted from 0; the paper raises theta by 1/40 per epoch); sequential
  (Alg. 2 as printed): columns 0..n-1 and rows 0..m-1 in order, no randomness.
* The generator state runs on across epochs; an epoch draws its column
  permutation first, then the row draws of each selected column in order.

Pinned in ``tests/test_oracle_schedule.py`` by the published SplitMix64 output
for seed 0, exhaustive checks of the without-replacement walk on tiny tables
and a chi-square test of first-draw frequencies against P.
"""
from __future__ import annotations

import math

import numpy as np

MASK = (1 << 64) - 1

SEQUENTIAL, UNIFORM, IMPORTANCE, MIXED = 0, 1, 2, 3


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood 2014), exact 64-bit integer arithmetic."""

    def __init__(self, seed: int):
        self.state = int(seed) & MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


def ceil_count(frac: float, total: int, div: int = 1) -> int:
    """ceil(frac * total / div) with a 1e-9 guard against rounding up exact integers."""
    return max(0, int(math.ceil(frac * total / div - 1e-9)))


def column_order(rng: SplitMix64, n: int, gamma: float, sampling: int):
    """Column blocks visited in one epoch (Alg. 3: k = 1 .. gamma n)."""
    k = ceil_count(gamma, n)
    if sampling == SEQUENTIAL:
        return list(range(min(k, n)))
    perm = list(range(n))
    for i in range(n - 1, 0, -1):
        jj = int(rng.uniform() * (i + 1))
        perm[i], perm[jj] = perm[jj], perm[i]
    return perm[:k]


def row_weights(P: np.ndarray, j: int, sampling: int, epoch: int, theta_step: float,
                view_block_of_row) -> np.ndarray:
    """Selection weights of every row block for column block j."""
    m = P.shape[0]
    if sampling in (UNIFORM, SEQUENTIAL):
        return np.ones(m)
    p = P[:, j].astype(np.float64)
    if sampling == IMPORTANCE:
        return p.copy()
    theta = min(1.0, epoch * theta_step)
    vb = np.asarray(view_block_of_row)
    pmax = np.zeros(m)
    for b in np.unique(vb):
        sel = vb == b
        pmax[sel] = p[sel].max()
    return p + theta * (pmax - p)


def draw_groups(rng: SplitMix64, w: np.ndarray, alpha: float, s: int, sampling: int):
    """Groups of row blocks for one column block (Alg. 3 inner loop / Alg. 4)."""
    m = w.shape[0]
    n_groups = ceil_count(alpha, m, s)
    if sampling == SEQUENTIAL:
        order = list(range(min(n_groups * s, m)))
        return [order[g * s:(g + 1) * s] for g in range((len(order) + s - 1) // s)]
    remaining = list(range(m))
    groups = []
    done = False
    for _ in range(n_groups):
        grp = []
        for _ in range(s):
            total = 0.0
            for i in remaining:
                total += w[i]
            if not (total > 0.0):
                done = True
                break
            thr = rng.uniform() * total
            acc = 0.0
            pick = None
            for i in remaining:
                acc += w[i]
                if acc > thr:
                    pick = i
                    break
            if pick is None:  # rounding: take the last block with positive weight
                pick = [i for i in remaining if w[i] > 0.0][-1]
            remaining.remove(pick)
            grp.append(pick)
        if grp:
            groups.append(grp)
        if done:
            break
    return groups


def epoch_schedule(rng: SplitMix64, P: np.ndarray, params: dict, epoch: int,
                   view_block_of_row) -> list:
    """One epoch: [(j, [group, group, ...]), ...] in execution order."""
    n = P.shape[1]
    sampling = params["sampling"]
    cols = column_order(rng, n, params["gamma"], sampling)
    out = []
    for j in cols:
        w = row_weights(P, j, sampling, epoch, params.get("theta_step", 1.0 / 40.0),
                        view_block_of_row)
        out.append((j, draw_groups(rng, w, params["alpha"], params["group_size"], sampling)))
    return out


def flatten(epochs: list) -> list:
    """Flat integer encoding shared with the library's schedule export.

    Per epoch: n_cols, then per column: j, n_groups, then per group: size, rows...
    """
    flat = []
    for ep in epochs:
        flat.append(len(ep))
        for j, groups in ep:
            flat.append(j)
            flat.append(len(groups))
            for g in groups:
                flat.append(len(g))
                flat.extend(g)
    return flat
