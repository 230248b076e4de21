"""Load balance of the paper's partitions on the GPU (Section 4: CP, RRP,
UCP; Lemmas 2-3; the comparison of Figs. 1 and 5).

The count pass runs with one task per resident warp -- a static mapping of
tasks to warps, like the paper's P processors -- under Eq. 3's uniform cost
partition (UCP), round robin (RRP: task t holds the items t, t + T, ...) and
the consecutive partition (CP, equal node counts).  The paper's claims:
runtime follows cost; UCP balances it; RRP balances it nearly as well but
loses locality; CP, whose first tasks hold the heaviest rows, is far slower.
The output is the same under all three (checked).  With the per-task clock
(cl_plan_task_clock), each task's run time is compared with its Eq. 1 cost.
Prints the tables."""
import numpy as np
import pytest
import torch

from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu

PARTS = ((0, "UCP (Eq. 3)"), (2, "RRP"), (1, "CP"))


def resident_warps(P, w, seed):
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(w, seed)
    grid, block = P.cl_plan_launch_info(g.plan)
    g.close()
    return grid * block // 32


def count_run(P, w, seed, reps=3, clock=False, **tun):
    """Count-pass time (ms, mean of reps), the counts, and per task (Eq. 1 cost in
    edges, run time in ms) when clock is set."""
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(w, seed, **tun)
    T = P.cl_plan_tasks(g.plan)
    stamps = None
    if clock:
        stamps = torch.zeros(2 * T, dtype=torch.int64, device="cuda")
        P.cl_plan_task_clock(g.plan, stamps)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.count()  # warm-up
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        g.count()
    b.record()
    torch.cuda.synchronize()
    counts = g.counts[: g.n_items].clone()
    st = g.stats()
    per_task = None
    if clock:
        ts = torch.empty(T + 1, dtype=torch.int64, device="cuda")
        C = torch.empty(g.n_items, dtype=torch.int64, device="cuda")
        P.cl_plan_tasks(g.plan, ts, C)
        torch.cuda.synchronize()
        ts, C, s = ts.cpu().numpy(), C.cpu().numpy(), stamps.cpu().numpy()
        c = np.diff(np.concatenate([[0], C])).astype(np.float64) / 16.0  # item costs, edges
        if tun.get("partition", 0) == 2:
            cost = np.array([c[t::T].sum() for t in range(T)])
        else:
            first = np.concatenate([[0.0], np.cumsum(c)])
            cost = first[ts[1:]] - first[ts[:-1]]
        per_task = (cost, (s[1::2] - s[0::2]).astype(np.float64) / 1e6)
    g.close()
    assert st["error"] == 0
    return a.elapsed_time(b) / reps, counts, per_task


@pytest.mark.parametrize("workload", ["pl_n1e7"])
def test_partitions_static_and_dynamic(workload):
    P = lib()
    w_np, seed = inputs.workload(workload)
    w = cuda(w_np)
    warps = resident_warps(P, w, seed)
    rows, ms = [], {}
    ref = None
    for tasks in (warps, 0):
        for part, name in PARTS:
            t, c, _ = count_run(P, w, seed, tasks=tasks, partition=part)
            if ref is None:
                ref = c
            assert torch.equal(c, ref), name  # tasks only schedule work
            ms[(tasks, part)] = t
            rows.append((tasks or "default", name, t))
    print(f"\n{workload} count pass (resident warps {warps}): tasks, partition, ms")
    for r in rows:
        print(f"  {str(r[0]):>10} {r[1]:12s} {r[2]:9.2f}")
    ucp, rrp, cp = ms[(warps, 0)], ms[(warps, 2)], ms[(warps, 1)]
    # one task per warp: a launch lasts as long as its costliest task
    assert cp > 1.5 * ucp
    assert rrp < cp


def test_task_time_follows_cost():
    """Per-task run time against Eq. 1 cost with one task per resident warp.
    Under CP and RRP the task costs differ (CP: by orders of magnitude), and
    time must follow cost (Pearson correlation); under UCP the costs are equal
    to within one item (Lemma 2) and the run times must be close."""
    P = lib()
    w_np, seed = inputs.workload("pl_n1e7")
    w = cuda(w_np)
    warps = resident_warps(P, w, seed)
    out = {}
    for part, name in PARTS:
        _, _, (cost, secs) = count_run(P, w, seed, reps=1, clock=True, tasks=warps, partition=part)
        ok = secs > 0
        r = np.corrcoef(cost[ok], secs[ok])[0, 1] if ok.sum() > 2 and np.std(cost[ok]) > 0 else float("nan")
        out[name] = (r, cost, secs)
        print(f"\n{name}: tasks {len(cost)}, cost max/mean {cost.max() / cost.mean():.3f}, "
              f"time max/mean {secs.max() / secs[ok].mean():.3f}, corr(time, cost) {r:.3f}")
    assert out["CP"][0] >= 0.9
    r_cost, r_secs = out["UCP (Eq. 3)"][1], out["UCP (Eq. 3)"][2]
    assert r_cost.max() / r_cost.mean() < 1.5
    # UCP: run-time spread far below CP's
    cp_secs = out["CP"][2]
    assert r_secs.max() / r_secs.mean() < 0.5 * cp_secs.max() / cp_secs.mean()
