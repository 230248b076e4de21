"""One-call generation (cl_generate: count, scan and emit with no host round
trip) against the CPU oracle and against the separate calls, element by
element: counts, offsets and the edge list must all be identical, whatever the
task count, block shape, staging slot size, edge type or number of graphs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def one_call(w, seed, etype=0, heavy_w=8192.0, slack=8, **tun):
    lib()
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(cuda(w) if isinstance(w, np.ndarray) else w, seed, heavy_w=heavy_w, **tun)
    m3 = g.generate(etype).shape[0]  # three-pass size
    c3 = g.counts[: g.n_items].clone()
    o3 = g.offsets.clone()
    dt = torch.int32 if etype == 0 else torch.int64
    edges = torch.full((m3 + slack, 2), -5, dtype=dt, device="cuda")
    g.counts.fill_(-1)
    g.offsets.fill_(-1)
    m = g.generate_into(edges, etype)
    st = g.stats()
    assert st["error"] == 0, st
    assert m == m3
    assert torch.equal(g.counts[: g.n_items], c3)
    assert torch.equal(g.offsets, o3)
    assert bool((edges[m:] == -5).all())
    out = edges[:m].cpu().numpy().astype(np.int64)
    g.close()
    return out


def oracle_edges(w, seed, heavy_w=8192.0):
    g = oracle.Graph(w, seed, heavy_w)
    return g.generate(counts=g.count_items())


def test_generate_matches_oracle_config1():
    w, seed = inputs.workload("pl_n1e5")
    assert np.array_equal(one_call(w, seed), oracle_edges(w, seed))


@pytest.mark.parametrize("tun", [{"tasks": 1}, {"tasks": 7}, {"tasks": 1 << 16}, {"block": 64}, {"block": 128},
                                 {"stage_factor": -1.0}, {"blocks_per_sm": 1}])
def test_generate_any_tuning(tun):
    w = inputs.powerlaw_degrees(60000, 2.2, 2, 3000, 51)
    assert np.array_equal(one_call(w, 3, **tun), oracle_edges(w, 3))


def test_generate_heavy_segments_int64():
    w = inputs.powerlaw_degrees(300000, 2.1, 2, 20000, 52)
    assert np.array_equal(one_call(w, 9, etype=1, heavy_w=600.0), oracle_edges(w, 9, heavy_w=600.0))


def test_generate_double_weights():
    w = np.sort(inputs.powerlaw_degrees(50000, 2.3, 3, 2000, 53).astype(np.float64) * 1.37)[::-1].copy()
    assert np.array_equal(one_call(w, 4), oracle_edges(w, 4))


def test_generate_batch_double_weights():
    # several graphs of double weights in one plan (the batched sampler with per-lane keys and
    # the float-float ln(1 - p) from doubles), each against the oracle
    lib()
    from paper_1406_1215_gb300.generator import Generator

    ws = [np.sort(inputs.powerlaw_degrees(n, 2.2, 2, max(3, int(n ** 0.5)), 70 + n % 5).astype(np.float64) *
                  (1.0 + 0.3 * (n % 3)))[::-1].copy() for n in (3000, 40000, 2, 25000)]
    seeds = [11, 12, 13, 14]
    g = Generator([cuda(w) for w in ws], seeds)
    E = g.generate().cpu().numpy().astype(np.int64)
    off = g.offsets.cpu().numpy()
    infos = [g.info(i) for i in range(len(ws))]
    g.close()
    for w, s, inf in zip(ws, seeds, infos):
        a, b = inf["item_begin"], inf["item_begin"] + inf["n_items"]
        assert np.array_equal(E[off[a]:off[b]], oracle_edges(w, s))


@pytest.mark.parametrize("partition", [0, 1])
def test_generate_batch_matches_singles(partition):
    # partition 1: the consecutive partition over the graphs' concatenated nodes
    lib()
    from paper_1406_1215_gb300.generator import Generator

    ws = [inputs.powerlaw_degrees(n, 2.4, 2, max(3, int(n ** 0.5)), 60 + n % 7) for n in (1000, 20000, 3, 70000, 1)]
    seeds = [5, 6, 7, 8, 9]
    g = Generator([cuda(w) for w in ws], seeds, partition=partition, tasks=0 if partition == 0 else 37)
    m3 = g.generate().shape[0]
    edges = torch.empty((m3, 2), dtype=torch.int32, device="cuda")
    assert g.generate_into(edges) == m3
    off = g.offsets.cpu().numpy()
    E = edges.cpu().numpy().astype(np.int64)
    for k, (w, sd) in enumerate(zip(ws, seeds)):
        a = int(off[g.info(k)["item_begin"]])
        b = int(off[g.info(k)["item_begin"] + g.info(k)["n_items"]])
        assert np.array_equal(E[a:b], oracle_edges(w, sd)), k
    g.close()


def test_generate_n1e7_counts_and_sampled_items():
    lib()
    w, seed = inputs.workload("pl_n1e7")
    E = one_call(w, seed)
    og = oracle.Graph(w, seed)
    rng = np.random.default_rng(8)
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(cuda(w), seed)
    g.count()
    g.scan(True)
    off = g.offsets.cpu().numpy()
    g.close()
    for a in [0, og.n_items - 50] + [int(x) for x in rng.integers(0, og.n_items - 50, 40)]:
        assert np.array_equal(E[int(off[a]):int(off[a + 50])], og.generate(a, a + 50)), a


def test_generate_capacity_error_and_reuse():
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    w = inputs.powerlaw_degrees(30000, 2.2, 3, 900, 54)
    g = Generator(cuda(w), 2)
    m = g.generate().shape[0]
    small = torch.full((m // 3, 2), -5, dtype=torch.int32, device="cuda")
    with pytest.raises(P.ClError) as e:
        g.generate_into(small)
    assert e.value.status == P.CL_ERR_CAPACITY
    g.stats()
    full = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    assert g.generate_into(full) == m
    assert np.array_equal(full.cpu().numpy().astype(np.int64), oracle_edges(w, 2))
    g.close()


@pytest.mark.parametrize("tun,etype", [({}, 0), ({"stage_factor": -1.0}, 0), ({"tasks": 3}, 1)])
def test_generate_small_degrees_wide_copy_claims(tun, etype):
    """Items of about one edge each: the copy kernel takes 256 items per claim."""
    w = inputs.powerlaw_degrees(300000, 2.9, 1, 40, 61)
    assert np.array_equal(one_call(w, 4, etype=etype, **tun), oracle_edges(w, 4))
