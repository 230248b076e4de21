"""Load balance of the paper's partitions (Section 4: Eq. 1-3, Lemmas 2-3, the
comparison of Figs. 1 and 5), reproduced with the oracle on CPU.

Work of an item = its realized loop iterations minus rejections, i.e. its edge
count + 1 (one terminating draw), which is what Eq. 1 models by c = e + 1.
Partitions of the item sequence over P processors:
  CP  consecutive blocks of equal item count,
  RRP round robin (item i to processor i mod P),
  UCP uniform cost partitioning (Eq. 3: boundaries where the cost prefix
      crosses multiples of Zbar = C_total / P).
Claims checked: UCP balances realized work to within the largest single item
(Lemma 2: every part's cost lies within c_max of Zbar) plus sampling noise;
UCP beats RRP, which beats CP by an order of magnitude on a power law; and the
cost model predicts each part's realized work (runtime proportional to cost).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1406_1215_gb300 import inputs

CASES = {
    "pl_n1e5": (inputs.workload("pl_n1e5")[0], 42),
    "pl_g2.1_n3e5": (inputs.powerlaw_degrees(300000, 2.1, 2, 3000, 9), 5),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, seed = CASES[request.param]
    g = oracle.Graph(w, seed)
    work = g.count_items().astype(np.float64) + 1.0
    return request.param, work, g.item_costs()


def parts(x, starts):
    return np.array([x[starts[p]:starts[p + 1]].sum() for p in range(len(starts) - 1)])


@pytest.mark.parametrize("P", [16, 64, 256])
def test_ucp_balances_realized_work(case, P):
    name, work, c = case
    n = len(work)
    st = oracle.ucp_starts(c, P)
    zbar = c.sum() / P
    cost = parts(c, st)
    assert np.all(np.abs(cost - zbar) <= c.max() + 1e-6 * zbar)  # Lemma 2
    ucp = parts(work, st)
    cp = parts(work, np.array([p * n // P for p in range(P + 1)]))
    rrp = np.array([work[p::P].sum() for p in range(P)])
    imb = {k: v.max() / v.mean() for k, v in (("ucp", ucp), ("cp", cp), ("rrp", rrp))}
    noise = 6.0 / math.sqrt(zbar)
    assert imb["ucp"] <= 1.0 + c.max() / zbar + noise, (name, P, imb)
    assert imb["ucp"] <= imb["rrp"] <= imb["cp"], (name, P, imb)
    assert imb["cp"] > 5.0, (name, P, imb)
    # runtime proportional to cost: each part's realized work within sampling noise of its cost
    # (capped pairs make the realized work only smaller: allow 2% for them)
    assert np.all(np.abs(ucp - cost) <= 6.0 * np.sqrt(cost) + 0.02 * cost), (name, P)


def node_costs(g: "oracle.Graph", n: int, c_items: np.ndarray) -> np.ndarray:
    """Eq. 1 node costs c_u = e_u + 1 from the oracle's item costs (a heavy row's
    segments summed back into its row; every item's cost carries the +1, so a row
    of k items gets k - 1 subtracted)."""
    rows = np.array([g.item_bounds(i)[0] for i in range(g.n_items)], dtype=np.int64)
    c = np.bincount(rows, weights=c_items, minlength=n)
    k = np.bincount(rows, minlength=n)
    c = c - np.maximum(k - 1, 0)
    c[k == 0] = 1.0  # a row without items (the last) still costs its own work
    return c


@pytest.mark.parametrize("P", [7, 64, 256])
def test_lemma3_round_robin_nodes(P):
    """Lemma 3 (RRP over nodes, Section 4): for i < j, c(V_i) >= c(V_j) (by Lemma 1) and
    c(V_i) - c(V_j) <= e_i, plus 1 when V_j holds one node fewer (the appendix proof uses
    that V_j's last node costs at least 1); hence below w_i + 1 <= w_0 + 1."""
    w = inputs.powerlaw_degrees(20000, 2.1, 2, 800, 11)
    g = oracle.Graph(w, 3)
    n = len(w)
    c = node_costs(g, n, g.item_costs())
    e = c - 1.0
    assert np.all(np.diff(c) <= 1e-9)  # Lemma 1
    cv = np.array([c[p::P].sum() for p in range(P)])
    size = np.array([len(range(p, n, P)) for p in range(P)])
    assert np.all(np.diff(cv) <= 1e-6)
    for i in range(P):
        for j in range(i + 1, P):
            bound = e[i] + (1.0 if size[i] > size[j] else 0.0)
            assert cv[i] - cv[j] <= bound + 1e-6, (i, j, cv[i] - cv[j], bound)
            assert cv[i] - cv[j] < w[i] + 1.0
            assert cv[i] - cv[j] < w[0] + 1.0
