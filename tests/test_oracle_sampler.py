"""Pins of the oracle's sampler against the Chung-Lu model itself.

Section 3: each pair (i, j), i < j, is an edge independently with probability
min(w_i w_j / S, 1); the skip algorithm (Algorithm 1) must reproduce exactly
that law, produce no self-loops or parallel edges, and run in O(n + m).
"""
import math
from collections import Counter

import numpy as np
import pytest

import oracle
from paper_1406_1215_gb300 import inputs


def pair_probs(w):
    w = np.asarray(w, dtype=np.float64)
    S = w.sum()
    n = len(w)
    P = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            P[i, j] = min(w[i] * w[j] / S, 1.0)
    return P


def sample_many(w, seeds, heavy_w=oracle.HEAVY_W_DEFAULT):
    n = len(w)
    X = np.zeros((n, n), dtype=np.int64)
    edge_sets = []
    for s in seeds:
        g = oracle.Graph(w, s, heavy_w)
        E = g.generate()
        assert np.all(E[:, 0] < E[:, 1])
        X[E[:, 0], E[:, 1]] += 1
        edge_sets.append(set(map(tuple, E.tolist())))
    return X, edge_sets


TINY = [
    np.array([9, 7, 5, 4, 3, 3, 2, 1, 1, 0], dtype=np.int32),  # capped pairs + a zero weight
    np.array([4, 4, 4, 4, 4, 4, 4, 4], dtype=np.int32),  # equal weights (ER)
    np.array([20, 2, 2, 1, 1, 1, 1, 1, 1, 1, 0, 0], dtype=np.int32),  # one hub, trailing zeros
    np.array([6.5, 4.25, 3.0, 2.75, 1.5, 0.3], dtype=np.float64),  # double weights, capped
]


@pytest.mark.parametrize("idx", range(len(TINY)))
def test_pair_frequencies_chi_square(idx):
    w = TINY[idx]
    N = 20000
    X, _ = sample_many(w, range(N), heavy_w=3.0 if idx == 2 else oracle.HEAVY_W_DEFAULT)
    P = pair_probs(w)
    n = len(w)
    chi2, dof = 0.0, 0
    for i in range(n):
        for j in range(i + 1, n):
            p = P[i, j]
            if p == 1.0:
                assert X[i, j] == N
            elif p == 0.0:
                assert X[i, j] == 0
            else:
                chi2 += (X[i, j] - N * p) ** 2 / (N * p * (1 - p))
                dof += 1
    # chi-square with dof degrees of freedom: mean dof, sd sqrt(2 dof); 5 sd margin
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


def test_pairs_are_independent():
    w = TINY[0]
    N = 20000
    X, sets = sample_many(w, range(100000, 100000 + N))
    P = pair_probs(w)
    # consecutive candidates of one row and pairs across rows
    for e1, e2 in [((1, 2), (1, 3)), ((2, 3), (2, 4)), ((1, 3), (2, 3)), ((3, 4), (3, 5)), ((0, 9), (1, 8))]:
        both = sum(1 for s in sets if e1 in s and e2 in s)
        p = P[e1] * P[e2]
        sd = math.sqrt(N * p * (1 - p)) + 1e-9
        assert abs(both - N * p) < 5 * sd + 1e-9, (e1, e2, both, N * p)


def test_simple_graph_invariants_config1():
    w, seed = inputs.workload("pl_n1e5")
    g = oracle.Graph(w, seed)
    E = g.generate()
    assert np.all(E[:, 0] < E[:, 1])
    key = E[:, 0] * len(w) + E[:, 1]
    assert np.all(np.diff(key) > 0)  # canonical order, no duplicates
    N, S, var = oracle.expected_edges_i32(w)
    assert abs(len(E) - N / S) < 6 * math.sqrt(var)


def test_expected_edges_closed_form_matches_bruteforce():
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = int(rng.integers(2, 400))
        w = np.sort(rng.integers(0, 60, n).astype(np.int32))[::-1].copy()
        if rng.random() < 0.3:
            w[: max(1, n // 20)] += 500  # create capped pairs
            w = np.sort(w)[::-1].copy()
        N, S, _ = oracle.expected_edges_i32(w)
        assert N == oracle.expected_edges_bruteforce_i32(w)
        # and against the definition in exact rationals
        Nref = sum(min(int(w[i]) * int(w[j]), S) for i in range(n) for j in range(i + 1, n))
        assert N == Nref


def test_mean_edge_count_over_seeds():
    w = inputs.powerlaw_degrees(3000, 2.2, 2, 300, 9)
    N, S, var = oracle.expected_edges_i32(w)
    ms = np.array([len(oracle.Graph(w, s).generate()) for s in range(400)])
    assert abs(ms.mean() - N / S) < 5 * math.sqrt(var / len(ms))
    assert 0.7 * var < ms.var() < 1.4 * var


def test_erdos_renyi_special_case():
    n, c = 2000, 10
    w = inputs.constant_weights(n, c)
    p = c / n
    ms, row0 = [], []
    for s in range(300):
        g = oracle.Graph(w, s)
        E = g.generate()
        ms.append(len(E))
        row0.append(int((E[:, 0] == 0).sum()))
    M = n * (n - 1) // 2
    ms = np.array(ms)
    assert abs(ms.mean() - M * p) < 5 * math.sqrt(M * p * (1 - p) / len(ms))
    row0 = np.array(row0)
    assert abs(row0.mean() - (n - 1) * p) < 5 * math.sqrt((n - 1) * p * (1 - p) / len(row0))


def brute_items(w, heavy_w):
    n = len(w)
    items = []
    H = int(np.sum(np.asarray(w, dtype=np.float64) >= heavy_w))
    for u in range(H):
        if u + 1 >= n:
            continue
        for k in range((u + 1) >> 16, ((n - 1) >> 16) + 1):
            items.append((u, k, max(u + 1, k << 16), min(n, (k + 1) << 16)))
    for u in range(H, n - 1):
        items.append((u, 0xFFFFFFFF, u + 1, n))
    return items


def test_item_space_matches_enumeration():
    n = 3 * 65536 + 123
    w = np.ones(n, dtype=np.int32)
    w[:70000] = 3
    w[:5] = 50
    for heavy_w in (1e9, 50.0, 3.0):
        g = oracle.Graph(w, 1, heavy_w)
        ref = brute_items(w, heavy_w)
        assert g.n_items == len(ref)
        rng = np.random.default_rng(0)
        idx = set(rng.integers(0, len(ref), 3000).tolist()) | {0, len(ref) - 1}
        if g.n_heavy_items:
            idx |= {g.n_heavy_items - 1, g.n_heavy_items}
        for i in sorted(idx):
            u, seg, j0, end = g.item_bounds(i)
            assert (u, seg, j0, end) == ref[i], i


def test_heavy_segments_sample_the_same_law():
    """A heavy row cut into 2^16-wide v-segments restarts the skip loop at each
    segment; pair probabilities across the cut must still be w_u w_v / S."""
    n = 65536 + 2000
    w = np.full(n, 2, dtype=np.int32)
    w[:3] = 2000
    S = int(w.sum())
    N = 3000
    cnt = Counter()
    per_seg = np.zeros(2)
    for s in range(N):
        g = oracle.Graph(w, s, heavy_w=1000.0)
        for it in range(g.n_heavy_items):
            u, seg, j0, end = g.item_bounds(it)
            if u != 0:
                continue
            v = g.generate_item(it)
            per_seg[seg] += len(v)
            for x in v[(v >= 65536 - 600) & (v < 65536 + 600)]:
                cnt[int(x)] += 1
    # expected edges of row 0 per segment
    p_small = 2000 * 2 / S
    exp0 = (2 * min(1.0, 2000 * 2000 / S) + (65536 - 3) * p_small) * N
    exp1 = (n - 65536) * p_small * N
    assert abs(per_seg[0] - exp0) < 5 * math.sqrt(exp0)
    assert abs(per_seg[1] - exp1) < 5 * math.sqrt(exp1)
    # the 1200 nodes straddling the cut: same per-node rate on both sides
    left = sum(cnt[v] for v in range(65536 - 600, 65536))
    right = sum(cnt[v] for v in range(65536, 65536 + 600))
    e = 600 * p_small * N
    assert abs(left - e) < 5 * math.sqrt(e) and abs(right - e) < 5 * math.sqrt(e)


def test_validation_flags():
    assert oracle.Graph(np.array([1, 2], dtype=np.int32), 0).status == 1
    assert oracle.Graph(np.array([2, -1], dtype=np.int32), 0).status == 2
    assert oracle.Graph(np.array([2.0, np.nan]), 0).status == 2
    g = oracle.Graph(np.array([5], dtype=np.int32), 0)
    assert g.status == 0 and g.n_items == 0
    g = oracle.Graph(np.zeros(10, dtype=np.int32), 0)
    assert g.n_items == 9 and len(g.generate()) == 0


def test_work_is_linear_in_n_plus_m():
    """Section 3: the skip algorithm does O(n + m) work.  Loop iterations =
    accepted + rejected candidates + one terminating draw per item; on a
    power law the rejections are few, so iterations stay near m + items.  A
    sampler that kept p at its initial value (still exact in law) would do
    far more iterations and fails here."""
    w, seed = inputs.workload("pl_n1e5")
    g = oracle.Graph(w, seed)
    st = oracle.Stats()
    m = int(g.count_items(stats=st).sum())
    assert m + g.n_items <= st.iterations < 1.2 * (m + g.n_items)
