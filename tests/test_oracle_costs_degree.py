"""Pins of the oracle's cost model, partition rule and expected degrees.

* Lemma 1: c_u >= c_v for u < v (light rows).
* Eq. 4: the total cost equals (number of items) + (expected edges, uncapped).
* Eq. 3 and Algorithm 2: the Calc-Cost prefix over P simulated processors
  equals the sequential prefix; partition boundaries satisfy
  C_{n_i - 1} < i Zbar <= C_{n_i}; a node belongs to partition floor(C_u/Zbar).
* Section 3: with no capped pair, E[d_i] = w_i - w_i^2 / S.
* Capped expected degree and its adjoint against O(n^2) brute force and
  central finite differences.
"""

import numpy as np

import oracle
from paper_1406_1215_gb300 import inputs


def test_lemma1_costs_non_increasing():
    w = inputs.powerlaw_degrees(20000, 2.3, 2, 500, 4)
    g = oracle.Graph(w, 1)
    c = g.item_costs()
    light = c[g.n_heavy_items:]
    assert np.all(np.diff(light) <= 1e-12)


def test_eq4_total_cost():
    w = inputs.powerlaw_degrees(50000, 2.3, 2, 900, 5)
    for heavy_w in (1e9, 300.0):
        g = oracle.Graph(w, 1, heavy_w)
        c = g.item_costs()
        wl = w.astype(np.float64)
        S = wl.sum()
        # uncapped expected edges sum_{u<v} w_u w_v / S = ((sum w)^2 - sum w^2) / (2 S)
        em = (S * S - (wl * wl).sum()) / (2 * S)
        assert abs(c.sum() - (g.n_items + em)) < 1e-9 * c.sum()


def test_calc_cost_matches_sequential_prefix():
    rng = np.random.default_rng(1)
    c = rng.random(10007) * 5 + 1
    seq = np.cumsum(c)
    for P in (1, 2, 7, 64, 1000):
        C = oracle.calc_cost(c, P)
        assert np.allclose(C, seq, rtol=1e-12)


def test_ucp_boundaries_follow_eq3():
    w = inputs.powerlaw_degrees(30000, 2.2, 2, 2000, 6)
    g = oracle.Graph(w, 1, 400.0)
    c = g.item_costs()
    C = np.cumsum(c)
    for T in (1, 3, 16, 256, 5000):
        st = oracle.ucp_starts(c, T)
        Zbar = C[-1] / T
        assert st[0] == 0 and st[-1] == len(c)
        assert np.all(np.diff(st) >= 0)
        for i in range(1, T):
            ni = st[i]
            assert C[ni] >= i * Zbar * (1 - 1e-12)
            if ni > 0:
                assert C[ni - 1] < i * Zbar * (1 + 1e-12)
        # node u belongs to partition floor(C_u / Zbar) (away from exact ties)
        part = np.searchsorted(st, np.arange(len(c)), side="right") - 1
        q = C / Zbar
        ok = np.abs(q - np.round(q)) > 1e-9
        assert np.all(np.minimum(np.floor(q[ok]), T - 1) == part[ok])
        # each partition's cost is at most Zbar plus its largest item
        costs = np.add.reduceat(c, st[:-1][np.diff(st) > 0])
        assert costs.max() <= Zbar + c.max() + 1e-9


def test_uncapped_expected_degree_closed_form():
    w = np.sort(np.random.default_rng(2).random(500) * 5 + 1)[::-1].copy()
    S = oracle.weight_sum_f64(w)
    assert (w[0] * w[0]) < S
    E = oracle.expected_degree(w)
    assert np.allclose(E, w - w * w / S, rtol=1e-13, atol=0)


def test_expected_degree_against_bruteforce_capped():
    d = inputs.powerlaw_degrees(2000, 2.1, 2, 600, 7).astype(np.float64)
    S = oracle.weight_sum_f64(d)
    assert d[0] * d[0] > 10 * S  # strong capping
    E = oracle.expected_degree(d)
    Eb = oracle.expected_degree(d, brute=True)
    assert np.max(np.abs(E - Eb) / Eb) < 1e-12


def loss(w, d):
    E = oracle.expected_degree(w)
    return float(np.sum((E - d) ** 2 / d))


def test_adjoint_against_bruteforce_and_finite_differences():
    d = inputs.powerlaw_degrees(300, 2.1, 2, 120, 8).astype(np.float64)
    rng = np.random.default_rng(3)
    w = np.sort(d * (1 + 0.05 * rng.random(len(d))))[::-1].copy()
    E = oracle.expected_degree(w)
    gE = 2 * (E - d) / d
    g = oracle.expected_degree_adjoint(w, gE)
    gb = oracle.expected_degree_adjoint(w, gE, brute=True)
    assert np.max(np.abs(g - gb)) < 1e-10 * np.max(np.abs(gb))
    # central differences of L on a sample of coordinates
    for k in list(range(0, 300, 23)) + [1, 2, 299]:
        h = 1e-6 * w[k]
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (loss(wp, d) - loss(wm, d)) / (2 * h)
        assert abs(fd - g[k]) < 1e-5 * (abs(g[k]) + 1e-3 * np.max(np.abs(g))), (k, fd, g[k])


def test_pairwise_adjoint_pins():
    """The O(n^2) pairwise gradient against the O(n^3) term-by-term brute force
    (n = 200) and the O(n log n) threshold form (n = 2000), capped pairs included."""
    for n, dmax, seed in ((200, 100, 9), (2000, 600, 10)):
        d = inputs.powerlaw_degrees(n, 2.1, 2, dmax, seed).astype(np.float64)
        rng = np.random.default_rng(seed)
        w = np.sort(d * (1 + 0.05 * rng.random(n)))[::-1].copy()
        S = oracle.weight_sum_f64(w)
        assert w[0] * w[0] > 4 * S  # some pairs are capped
        E = oracle.expected_degree(w, S)
        gE = 2 * (E - d) / d
        gp = oracle.expected_degree_adjoint(w, gE, S, pairwise=True)
        gf = oracle.expected_degree_adjoint(w, gE, S)
        assert np.max(np.abs(gp - gf)) < 1e-11 * np.max(np.abs(gf)), n
        if n <= 200:
            gb = oracle.expected_degree_adjoint(w, gE, S, brute=True)
            assert np.max(np.abs(gp - gb)) < 1e-11 * np.max(np.abs(gb))
