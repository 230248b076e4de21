"""Load balance of the paper's partitions on the GPU (Section 4, Figs. 1 and
5): the count pass with one task per resident warp -- a static mapping of
tasks to warps, like the paper's P processors -- under Eq. 3's uniform cost
partition (UCP) against the consecutive partition (CP, equal node counts).
The paper's claim is that runtime follows cost and UCP balances it; a
launch with one task per warp lasts as long as its costliest task, so CP,
whose first tasks hold the heaviest rows, must be much slower.  The output is
the same under both (checked), and with many tasks per warp (the default)
the dynamic task counter hides most of CP's imbalance.  Prints the table.
"""
import numpy as np
import pytest
import torch

from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def count_ms(w, seed, reps=3, **tun):
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(w, seed, **tun)
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
    g.close()
    assert st["error"] == 0
    return a.elapsed_time(b) / reps, counts


def test_ucp_balances_cp_does_not():
    lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    warps = sms * 4 * 8  # the count pass's resident warps (4 blocks of 256 per SM)
    w_np, seed = inputs.workload("pl_n1e7")
    w = cuda(w_np)
    rows = []
    ref = None
    for tasks in (warps, 0):
        for part, name in ((0, "UCP (Eq. 3)"), (1, "CP")):
            ms, c = count_ms(w, seed, tasks=tasks, partition=part)
            if ref is None:
                ref = c
            assert torch.equal(c, ref)  # tasks only schedule work
            rows.append((tasks or "64 x warps", name, ms))
    print("\npl_n1e7 count pass: tasks, partition, ms")
    for r in rows:
        print(f"  {str(r[0]):>12} {r[1]:12s} {r[2]:8.2f}")
    ucp_static, cp_static = rows[0][2], rows[1][2]
    assert cp_static > 1.5 * ucp_static
