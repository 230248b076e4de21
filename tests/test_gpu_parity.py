"""Edge-list parity: the CUDA path (through the C ABI) against the CPU
oracle, element by element (bit-exact: the output is integer).

Workloads: the paper's power-law and Erdos-Renyi shapes (Section 5, Table 1
PL/ER rows) at sizes the oracle finishes in seconds, several tiles with
ragged tails, heavy-row segmentation, capped pairs, zero weights, the
degenerate graphs (n = 0, 1, 2), every tuning knob, chunked emit, batches.
"""
import math
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib, oracle_parallel, split_ranges

pytestmark = pytest.mark.gpu


def gpu_generate(w: np.ndarray, seed: int, heavy_w=8192.0, etype=0, **tun):
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(cuda(w), seed, heavy_w=heavy_w, **tun)
    E = g.generate(etype)
    counts = g.counts[: g.n_items].cpu().numpy().copy()
    st = g.stats()  # reads and clears the device error word
    out = E.cpu().numpy().astype(np.int64)
    g.close()
    assert st["error"] == 0, st
    return out, counts, st


def oracle_generate(w, seed, heavy_w=8192.0):
    g = oracle.Graph(w, seed, heavy_w)
    c = g.count_items()
    return g.generate(counts=c), c, g


def test_parity_config1_full():
    w, seed = inputs.workload("pl_n1e5")
    Eg, cg, st = gpu_generate(w, seed)
    Eo, co, _ = oracle_generate(w, seed)
    assert np.array_equal(cg, co)
    assert np.array_equal(Eg, Eo)
    assert st["error"] == 0 and st["ties"] == 0
    N, S, var = oracle.expected_edges_i32(w)
    assert abs(len(Eg) - N / S) < 6 * math.sqrt(var)


@pytest.mark.parametrize("etype", [0, 1])
def test_parity_int64_edges(etype):
    w = inputs.powerlaw_degrees(30000, 2.2, 2, 800, 21)
    Eg, _, _ = gpu_generate(w, 7, etype=etype)
    Eo, _, _ = oracle_generate(w, 7)
    assert np.array_equal(Eg, Eo)


SMALL = {
    "capped_zero": np.array([9, 7, 5, 4, 3, 3, 2, 1, 1, 0], dtype=np.int32),
    "equal": np.full(50, 4, dtype=np.int32),
    "hub_zeros": np.array([20, 2, 2, 1, 1, 1, 1, 1, 1, 1, 0, 0], dtype=np.int32),
    "all_zero": np.zeros(17, dtype=np.int32),
    "n2": np.array([5, 3], dtype=np.int32),
    "n1": np.array([5], dtype=np.int32),
    "dense_capped": np.array([100] * 30 + [50] * 30 + [1] * 40, dtype=np.int32),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_parity_small_graphs(name):
    w = SMALL[name]
    for seed in range(20):
        for hw in (8192.0, 3.0):
            Eg, cg, _ = gpu_generate(w, seed, heavy_w=hw)
            Eo, co, _ = oracle_generate(w, seed, hw)
            assert np.array_equal(cg, co), (name, seed, hw)
            assert np.array_equal(Eg.reshape(-1, 2)[: len(Eo)], Eo) and len(Eg) == len(Eo)


def test_parity_heavy_segments_many_tiles():
    # n > 3 * 2^16 with heavy rows split into several segments, ragged last segment
    n = 3 * 65536 + 4321
    w = inputs.powerlaw_degrees(n, 2.1, 3, 3000, 22)
    Eg, cg, _ = gpu_generate(w, 11, heavy_w=600.0)
    Eo, co, g = oracle_generate(w, 11, 600.0)
    assert g.n_heavy_items > 4 * 10
    assert np.array_equal(cg, co)
    assert np.array_equal(Eg, Eo)


def test_parity_erdos_renyi():
    w = inputs.constant_weights(200000, 30)
    Eg, cg, _ = gpu_generate(w, 5)
    Eo, co, _ = oracle_generate(w, 5)
    assert np.array_equal(Eg, Eo)
    M = 200000 * 199999 / 2
    p = 30 / 200000
    assert abs(len(Eg) - M * p) < 6 * math.sqrt(M * p)


def test_output_independent_of_tuning():
    w = inputs.powerlaw_degrees(60000, 2.3, 2, 2000, 23)
    ref, cref, _ = gpu_generate(w, 3, heavy_w=500.0)
    for tun in ({"tasks": 1}, {"tasks": 7}, {"tasks": 100000}, {"block": 32}, {"block": 128, "blocks_per_sm": 1},
                {"blocks_per_sm": 2, "tasks": 333}, {"no_stage": 1}, {"partition": 1},
                {"partition": 1, "tasks": 333},  # the paper's consecutive partition instead of Eq. 3
                {"partition": 2}, {"partition": 2, "tasks": 333},  # round robin
                {"partition": 2, "tasks": 333, "no_stage": 1},
                {"partition": 2, "stage_factor": -1.0},
                {"stage_factor": -1.0}):  # 8-entry slots: most items regenerated by cl_emit
        E, c, _ = gpu_generate(w, 3, heavy_w=500.0, **tun)
        assert np.array_equal(c, cref), tun
        assert np.array_equal(E, ref), tun


def test_chunked_emit_equals_full_emit():
    lib()
    from paper_1406_1215_gb300.generator import Generator

    w = inputs.powerlaw_degrees(50000, 2.4, 2, 900, 24)
    g = Generator(cuda(w), 9)
    full = g.generate().cpu().numpy()
    off = g.offsets.cpu().numpy()
    bounds = [0, 1, 17, 1000, 20000, g.n_items - 1, g.n_items]
    for a, b in zip(bounds[:-1], bounds[1:]):
        m = int(off[b] - off[a])
        buf = torch.full((max(m, 1), 2), -7, dtype=torch.int32, device="cuda")
        g.emit(buf, 0, a, b)
        torch.cuda.synchronize()
        assert np.array_equal(buf[:m].cpu().numpy(), full[off[a]:off[b]])
    g.close()


def test_capacity_error_writes_nothing():
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    w = inputs.powerlaw_degrees(20000, 2.4, 2, 500, 25)
    g = Generator(cuda(w), 9)
    g.count()
    m = g.scan(True)
    buf = torch.full((m - 1, 2), -7, dtype=torch.int32, device="cuda")
    g.emit(buf, 0)
    torch.cuda.synchronize()
    st = g.stats()
    assert st["error"] == 5  # CL_ERR_CAPACITY
    assert bool((buf == -7).all())
    g.close()


@pytest.mark.parametrize("bad,code", [
    (np.array([1, 2, 3], dtype=np.int32), 2),
    (np.array([3, -1, -2], dtype=np.int32), 3),
    (np.array([3.0, float("nan")]), 3),
    (np.array([3.0, float("inf")]), 3),
    (np.array([1.0, 2.0]), 2),
])
def test_validation_errors(bad, code):
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    with pytest.raises(P.ClError) as ei:
        Generator(cuda(bad), 1)
    assert ei.value.status == code


def test_misaligned_scratch_and_workspace_rejected():
    """cl_plan_create and cl_plan_build take 256-byte aligned device memory (the staging
    pool's 32-byte slot boundaries depend on it); an offset pointer is refused before any
    launch, and the aligned call that follows succeeds."""
    P = lib()
    w = cuda(np.array([9, 7, 7, 4, 2, 1], dtype=np.int32))
    g = [P.cl_graph(6, P.CL_W_I32, w.data_ptr(), 5, P.HEAVY_W_DEFAULT)]
    sb = P.cl_plan_scratch_bytes(1)
    scratch = torch.empty(sb + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.ClError) as ei:
        P.cl_plan_create(g, None, scratch.data_ptr() + 16, sb)
    assert ei.value.status == P.CL_ERR_INVALID_ARG
    plan = P.cl_plan_create(g, None, scratch, sb)
    try:
        wb = P.cl_plan_workspace_bytes(plan)
        ws = torch.empty(wb + 512, dtype=torch.uint8, device="cuda")
        with pytest.raises(P.ClError) as ei:
            P.cl_plan_build(plan, ws.data_ptr() + 32, wb)
        assert ei.value.status == P.CL_ERR_INVALID_ARG
        P.cl_plan_build(plan, ws, wb)
        torch.cuda.synchronize()
    finally:
        P.cl_plan_destroy(plan)


def test_empty_and_trivial_graphs():
    for n in (0, 1, 2, 3):
        w = (np.arange(n, 0, -1) * 3).astype(np.int32)
        for seed in range(5):
            E, c, _ = gpu_generate(w, seed)
            Eo, co, _ = oracle_generate(w, seed)
            assert np.array_equal(c, co)
            assert np.array_equal(E.reshape(-1, 2), Eo.reshape(-1, 2))


def test_batch_equals_single_graphs():
    lib()
    from paper_1406_1215_gb300.generator import Generator

    ws, seeds = [], []
    for g in range(12):
        n, gamma, a, b = inputs.batch_graph_params(g)
        n = min(n, 40000)
        ws.append(inputs.powerlaw_degrees(n, gamma, a, max(a, min(b, int(math.isqrt(n)))), 100 + g))
        seeds.append(g)
    ws.append(np.array([3], dtype=np.int32))  # a graph with no items
    seeds.append(99)
    gen = Generator([cuda(w) for w in ws], seeds)
    ref = [oracle_generate(w, s)[0] for w, s in zip(ws, seeds)]
    total = sum(len(r) for r in ref)
    edges = torch.full((total + 10, 2), -1, dtype=torch.int32, device="cuda")
    goff = torch.empty(len(ws) + 1, dtype=torch.int64, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    gen.generate_batch(edges, goff, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    go = goff.cpu().numpy()
    E = edges.cpu().numpy().astype(np.int64)
    assert go[-1] == total
    for i, r in enumerate(ref):
        assert np.array_equal(E[go[i]:go[i + 1]], r), i
    # too small a buffer: status says so and nothing is written
    small = torch.full((total - 1, 2), -1, dtype=torch.int32, device="cuda")
    gen.generate_batch(small, goff, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 5
    assert bool((small == -1).all())
    gen.close()


def test_parity_config2_counts_full_edges_sampled():
    """n = 10^7, gamma 2.5 on [10, 10^4]: every item's count and the edges of
    sampled item ranges (including all heavy items) against the oracle."""
    lib()
    from paper_1406_1215_gb300.generator import Generator

    w, seed = inputs.workload("pl_n1e7")
    g = Generator(cuda(w), seed)
    E = g.generate()
    counts = g.counts[: g.n_items].cpu().numpy()
    off = g.offsets.cpu().numpy()
    st = g.stats()
    n_items, nh = g.n_items, g.info(0)["n_items"]
    og = oracle.Graph(w, seed)
    assert og.n_items == n_items
    with tempfile.TemporaryDirectory() as td:
        parts = oracle_parallel(w, seed, 8192.0, split_ranges(n_items, 64), "count", td)
        co = np.concatenate([c for _, c, _ in sorted(parts, key=lambda x: x[0])])
        assert np.array_equal(counts, co)
        it_oracle = sum(s["iterations"] for _, _, s in parts)
        assert st["iterations"] == it_oracle
        rng = np.random.default_rng(0)
        starts = [0] + [og.n_heavy_items] + list(rng.integers(0, n_items - 500, 40))
        ranges = [(int(a), int(min(a + 500, n_items))) for a in starts] + [(n_items - 300, n_items)]
        eparts = oracle_parallel(w, seed, 8192.0, ranges, "edges", td)
    Eh = E.cpu().numpy()
    for (a, b), (_, eo) in zip(ranges, eparts):
        assert np.array_equal(Eh[off[a]:off[b]].astype(np.int64), eo), (a, b)
    g.close()


def test_regeneration_beyond_the_overflow_list():
    """With 8-entry slots, over 2^20 items outgrow their slot: the regeneration
    pass then walks every item instead of the list; output unchanged."""
    w = inputs.constant_weights(1_600_000, 60)
    ref, cref, _ = gpu_generate(w, 13, no_stage=1)
    E, c, _ = gpu_generate(w, 13, stage_factor=-1.0)
    assert int((c > 8).sum()) > (1 << 20)
    assert np.array_equal(c, cref)
    assert np.array_equal(E, ref)
    o = oracle.Graph(w, 13)
    rng = np.random.default_rng(1)
    for a in rng.integers(0, o.n_items - 20, 10):
        off = np.concatenate([[0], np.cumsum(cref.astype(np.int64))])
        assert np.array_equal(E[off[a]:off[a + 20]], o.generate(int(a), int(a) + 20))


def test_table1_er_network():
    """The paper's Table 1 ER row (1M nodes, 200M edges; tests/golden/table1_er.json):
    the edge count within 6 sd of the oracle's exact E[m], and sampled items equal to
    the oracle's."""
    import json
    import os

    lib()
    from paper_1406_1215_gb300.generator import Generator

    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_er.json")))
    n = gold["nodes"]
    w = inputs.constant_weights(n, round(2 * gold["edges"] / n))
    N, S, var = oracle.expected_edges_i32(w)
    g = Generator(cuda(w), 17)
    E = g.generate()
    m = E.shape[0]
    off = g.offsets.cpu().numpy()
    g.close()
    assert abs(m - N / S) < 6 * math.sqrt(var)
    assert abs(m - gold["edges"]) <= gold["edges_rounding"] + 6 * math.sqrt(var)
    og = oracle.Graph(w, 17)
    rng = np.random.default_rng(3)
    Eh = None
    for a in [0, og.n_items - 20] + [int(x) for x in rng.integers(0, og.n_items - 20, 20)]:
        if Eh is None:
            Eh = E.cpu().numpy().astype(np.int64)
        assert np.array_equal(Eh[int(off[a]):int(off[a + 20])], og.generate(a, a + 20)), a


@pytest.mark.parametrize("tun,etype", [({}, 0), ({}, 1), ({"stage_factor": -1.0}, 0), ({"no_stage": 1}, 1),
                                       ({"tasks": 2}, 0)])
def test_parity_long_capped_runs(tun, etype):
    """Five hub rows whose every partner is capped (w_u w_v >= S for all v): their
    capped runs span two 2^16-wide segments and are written in one go; with 8-entry
    slots (stage_factor -1) they outgrow the slot and the emit pass regenerates them,
    and without staging the emit pass writes the runs itself.  Edges, counts and the
    loop-iteration total equal the oracle's (one draw per capped position)."""
    w = np.concatenate([np.full(5, 300000), np.full(100000, 10), np.full(3000, 1)]).astype(np.int32)
    Eg, cg, st = gpu_generate(w, 17, etype=etype, **tun)
    stats = oracle.Stats()
    Eo, co, g = oracle_generate(w, 17)
    oracle.Graph(w, 17).count_items(stats=stats)
    assert np.array_equal(cg, co)
    assert np.array_equal(Eg, Eo)
    assert st["iterations"] == stats.iterations
    assert int(co[0]) == 65535  # the first hub's first segment is one capped run
