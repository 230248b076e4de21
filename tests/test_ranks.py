"""The multi-rank path of bench.py on CPU: world size 2 over gloo (ranks are
replicas: each generates its own graph).  The whole-job figures are the
slowest rank's timed region and the sum of every rank's edges; each rank draws
its own graph; a rank that raises ends the job without hanging the other."""
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q, fail_rank):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=__import__("datetime").timedelta(seconds=20))
    try:
        if rank == fail_rank:
            raise RuntimeError("planted failure")
        elapsed = [1.5, 2.25][rank]
        edges = [1000.0, 3000.0][rank]
        t, m = bench.aggregate_ranks(dist, elapsed, edges, torch.device("cpu"))
        q.put((rank, t, m, bench.rank_seed(42, rank)))
    except Exception as e:  # report, then leave between steps
        q.put((rank, "error", str(e), None))
    finally:
        if rank != fail_rank:
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def _run(world, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=60) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    return sorted(out, key=lambda r: r[0])


def test_aggregate_is_max_time_and_sum_of_edges():
    out = _run(2)
    for rank, t, m, seed in out:
        assert t == 2.25 and m == 4000.0
    assert [r[3] for r in out] == [42, 43]


def test_single_rank_needs_no_collective():
    assert bench.aggregate_ranks(None, 1.25, 7.0, None) == (1.25, 7.0)


def test_failing_rank_does_not_hang_the_other():
    out = _run(2, fail_rank=1)
    assert out[1][1] == "error"
    assert out[0][1] == "error"  # the surviving rank's collective ends with an error (timeout/peer gone)
