"""The GPU's task split against the paper's cost model and partition rule
(Section 4): per-item costs of Eq. 1-2 (Eq. 6 for light rows), the cost
prefix of Calc-Cost (Algorithm 2) and the lower boundaries of Eq. 3, read
back through cl_plan_tasks and checked against the CPU oracle.

The GPU charges an item c0 = 4 edges of fixed work where Eq. 1 charges 1,
and rounds each cost to 1/16 of an edge from single precision; the tests add
the difference (3) to the oracle's costs and allow that rounding.  Checked:
  * every GPU item cost equals the oracle's Eq. 1 cost + 3 up to the rounding;
  * every boundary n_t is the first item with C_i >= t * Zbar on the GPU's own
    integer prefix (Eq. 3, exact);
  * the oracle's own Eq. 3 routine, given the GPU's costs, finds the same
    boundaries (up to ties decided by double rounding);
  * every task's cost lies within the largest item cost of Zbar (Lemma 2);
  * the consecutive partition (CP) gives each task the same number of rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu

C0_DIFF = 3.0  # GPU c0 = 4 edges, Eq. 1's constant = 1


def gpu_tasks(P, w, seed, heavy_w, tasks=0, partition=0):
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(cuda(w), seed, heavy_w=heavy_w, tasks=tasks, partition=partition)
    T = P.cl_plan_tasks(g.plan)
    ts = torch.empty(T + 1, dtype=torch.int64, device="cuda")
    cp = torch.empty(max(g.n_items, 1), dtype=torch.int64, device="cuda")
    P.cl_plan_tasks(g.plan, ts, cp)
    torch.cuda.synchronize()
    n_items = g.n_items
    g.close()
    return T, ts.cpu().numpy(), cp[:n_items].cpu().numpy(), n_items


CASES = {
    # gamma 2.1 power law with many heavy rows (heavy_w 256): rows cut into 5 segments each
    "pl_g2.1_n3e5_heavy": (lambda: inputs.powerlaw_degrees(300_000, 2.1, 2, 3000, 9), 5, 256.0),
    # the n = 10^7 workload (gamma 2.5 on [10, 10^4])
    "pl_n1e7": (lambda: inputs.workload("pl_n1e7")[0], 42, 8192.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("tasks", [0, 1000])
def test_task_split_follows_eq3_and_lemma2(name, tasks):
    P = lib()
    mk, seed, heavy_w = CASES[name]
    w = mk()
    T, ts, C, n_items = gpu_tasks(P, w, seed, heavy_w, tasks=tasks)
    g = oracle.Graph(w, seed, heavy_w)
    assert n_items == g.n_items
    if tasks:
        assert T == tasks
    c_or = g.item_costs() + C0_DIFF  # Eq. 1 costs with the GPU's per-item constant
    # per-item costs: 1/16-edge units, single-precision products
    c_gpu = np.diff(np.concatenate([[0], C])).astype(np.float64) / 16.0
    e_or = c_or - 1.0 - C0_DIFF
    tol = 1.0 / 32.0 + 2.0 ** -19 * e_or + 1e-9
    bad = np.abs(c_gpu - c_or) > tol
    assert not bad.any(), (name, int(bad.sum()), np.flatnonzero(bad)[:5])
    # Eq. 3 on the GPU's exact integer prefix: n_t = first i with C_i * T >= t * C_total
    Ctot = int(C[-1])
    assert Ctot * T < 2 ** 62
    assert ts[0] == 0 and ts[T] == n_items and np.all(np.diff(ts) >= 0)
    t = np.arange(1, T, dtype=np.int64)
    nt = ts[1:T]
    goal = t * Ctot
    at = np.where(nt < n_items, C[np.minimum(nt, n_items - 1)], np.iinfo(np.int64).max // 2 // T)
    before = np.where(nt > 0, C[np.maximum(nt - 1, 0)], -1)
    assert np.all(at * T >= goal), name
    assert np.all(before * T < goal), name
    # the oracle's Eq. 3 rule (or_ucp_starts, double precision) on the GPU's own costs gives the
    # same boundaries, except where a prefix value ties t * Zbar to double rounding
    c_g = np.diff(np.concatenate([[0], C])).astype(np.float64) / 16.0
    st_o = oracle.ucp_starts(c_g, T)
    mism = np.flatnonzero(st_o != ts)
    Cd = C.astype(np.float64) / 16.0
    for k in mism:
        goal_d = k * (Cd[-1] / T)
        near = [Cd[i] for i in (st_o[k], ts[k], st_o[k] - 1, ts[k] - 1) if 0 <= i < n_items]
        assert min(abs(x - goal_d) for x in near) <= 1e-9 * Cd[-1], (name, k, st_o[k], ts[k])
    assert len(mism) <= max(2, T // 1000), (name, len(mism))
    # Lemma 2: every task's cost is within the largest item cost of Zbar
    zbar = Ctot / T
    first = np.concatenate([[0], C])
    cost = first[ts[1:]] - first[ts[:-1]]
    cmax = np.max(np.diff(first))
    assert np.all(np.abs(cost - zbar) <= cmax + 1e-6), (name, float(np.max(np.abs(cost - zbar))), cmax)


def test_consecutive_partition_equal_rows():
    P = lib()
    w = inputs.powerlaw_degrees(300_000, 2.1, 2, 3000, 9)
    heavy_w = 256.0
    T, ts, _, n_items = gpu_tasks(P, w, 5, heavy_w, tasks=777, partition=1)
    g = oracle.Graph(w, 5, heavy_w)
    n = len(w)
    for t in range(T):
        row = t * n // T
        i = int(ts[t])
        # the first item of row `row` (rows without items -- the last row -- start the next row's)
        if i < n_items:
            u = g.item_bounds(i)[0]
            assert u >= row
            if i > 0:
                assert g.item_bounds(i - 1)[0] < row
        else:
            assert row >= n - 1
