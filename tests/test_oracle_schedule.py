"""Pins of the oracle's block choice (Alg. 3 / Alg. 4 sampling, Sec. III-D mixed)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import schedule as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        vals = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    g = S.SplitMix64(0)
    assert [g.next() for _ in range(len(vals))] == vals


def test_uniform_double_range_and_resolution():
    g = S.SplitMix64(123)
    u = np.array([g.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    # 53-bit grid: u * 2^53 is an integer
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)


def test_first_draw_frequencies_follow_p():
    """Alg. 3: a row block is drawn with probability proportional to P(I, J)."""
    w = np.array([0.05, 0.4, 0.0, 0.25, 0.3])
    counts = np.zeros(5)
    N = 100000
    for seed in range(N):
        g = S.SplitMix64(seed)
        grp = S.draw_groups(g, w, alpha=1.0 / 5, s=1, sampling=S.IMPORTANCE)
        counts[grp[0][0]] += 1
    assert counts[2] == 0
    nz = w > 0
    chi2, p = stats.chisquare(counts[nz], N * w[nz] / w.sum())
    assert p > 1e-3


def test_without_replacement_sequence_probabilities():
    """Second draw given the first: P(b | a) = w_b / (W - w_a) (sampling without
    replacement), checked exactly by enumerating ordered pairs."""
    w = np.array([1.0, 2.0, 3.0])
    N = 60000
    pairs = {}
    for seed in range(N):
        g = S.SplitMix64(10_000_000 + seed)
        grp = S.draw_groups(g, w, alpha=2.0 / 3, s=2, sampling=S.IMPORTANCE)
        assert len(grp) == 1 and len(grp[0]) == 2 and grp[0][0] != grp[0][1]
        pairs[tuple(grp[0])] = pairs.get(tuple(grp[0]), 0) + 1
    keys = sorted(pairs)
    exp = np.array([w[a] / 6 * w[b] / (6 - w[a]) for a, b in keys]) * N
    obs = np.array([pairs[k] for k in keys])
    assert len(keys) == 6
    assert stats.chisquare(obs, exp)[1] > 1e-3


def test_group_counts_and_early_stop():
    g = S.SplitMix64(1)
    w = np.ones(10)
    grp = S.draw_groups(g, w, alpha=0.5, s=2, sampling=S.UNIFORM)
    assert [len(x) for x in grp] == [2, 2, 2]  # ceil(0.5 * 10 / 2) = 3 groups of 2
    assert len(set(sum(grp, []))) == 6
    # alpha = 1, s = 4, m = 10: 3 groups, the last one partly filled
    grp = S.draw_groups(S.SplitMix64(2), w, alpha=1.0, s=4, sampling=S.UNIFORM)
    assert [len(x) for x in grp] == [4, 4, 2]
    # zero weights stop the draws: only two blocks can ever be drawn
    w2 = np.array([0, 0.5, 0, 0.5, 0.0])
    grp = S.draw_groups(S.SplitMix64(3), w2, alpha=1.0, s=1, sampling=S.IMPORTANCE)
    assert sorted(sum(grp, [])) == [1, 3]


def test_fisher_yates_is_uniform():
    n = 4
    N = 48000
    counts = {}
    for seed in range(N):
        perm = tuple(S.column_order(S.SplitMix64(seed), n, 1.0, S.UNIFORM))
        counts[perm] = counts.get(perm, 0) + 1
    assert len(counts) == math.factorial(n)
    obs = np.array(list(counts.values()))
    assert stats.chisquare(obs)[1] > 1e-3


def test_gamma_takes_a_prefix_and_sequential_order():
    cols = S.column_order(S.SplitMix64(5), 16, 0.2, S.UNIFORM)
    assert len(cols) == 4 and len(set(cols)) == 4  # ceil(0.2 * 16) = 4
    assert S.column_order(None, 5, 1.0, S.SEQUENTIAL) == [0, 1, 2, 3, 4]
    assert S.draw_groups(None, np.ones(5), 1.0, 2, S.SEQUENTIAL) == [[0, 1], [2, 3], [4]]


def test_mixed_weights_ramp():
    """Sec. III-D: w = P + theta (P_max - P) within one projection; theta reaches 1 after
    40 epochs at the paper's step of 1/40, where all sub-areas of a view are equal."""
    P = np.array([[0.1], [0.3], [0.2], [0.4]])
    vb = [0, 0, 1, 1]
    w0 = S.row_weights(P, 0, S.MIXED, 0, 1 / 40, vb)
    np.testing.assert_allclose(w0, P[:, 0])
    w20 = S.row_weights(P, 0, S.MIXED, 20, 1 / 40, vb)
    np.testing.assert_allclose(w20, [0.2, 0.3, 0.3, 0.4])
    w40 = S.row_weights(P, 0, S.MIXED, 45, 1 / 40, vb)
    np.testing.assert_allclose(w40, [0.3, 0.3, 0.4, 0.4])
