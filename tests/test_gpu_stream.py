"""Out-of-core delivery through cl_generate_stream: the edge list is handed to
a sink piece by piece through a ring much smaller than the graph (the paper's
Section 5 network of 249 billion edges is far beyond one GPU's memory).  The
concatenated pieces must equal the oracle's edge list (small graph) and the
device-resident generation's (larger graph, sampled items against the
oracle); pieces arrive in edge order with consistent item ranges; splitting
(ranges larger than half the ring), stopping and the capacity error work."""
import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def collect(gen, ring_edges, etype=0, stop_after=None):
    pieces = []

    def sink(pairs, first, ib, ie):
        pieces.append((first, ib, ie, pairs.clone().numpy()))
        return stop_after is not None and len(pieces) >= stop_after

    m = gen.generate_stream(sink, ring_edges, etype)
    return m, pieces


def check_order(pieces, offsets):
    """Pieces come in edge order; items between two pieces (pieces without edges are
    not handed over) hold no edges."""
    nxt_edge, nxt_item = 0, 0
    for first, ib, ie, E in pieces:
        assert first == nxt_edge and ib >= nxt_item and offsets[ib] == offsets[nxt_item]
        assert len(E) == offsets[ie] - offsets[ib] > 0
        nxt_edge, nxt_item = first + len(E), ie
    assert offsets[nxt_item] == offsets[-1]


@pytest.mark.parametrize("tun", [{}, {"tasks": 3}, {"no_stage": 1}, {"max_pool_entries": 4096}, {"max_pool_entries": 30004}])
def test_stream_equals_oracle_small(tun):
    lib()
    from paper_1406_1215_gb300.generator import Generator

    w, seed = inputs.workload("pl_n1e5")
    g = Generator(cuda(w), seed, **tun)
    m, pieces = collect(g, ring_edges=2 * 4096)
    offsets = g.offsets.cpu().numpy()
    st = g.stats()
    g.close()
    assert st["error"] == 0
    Eo = oracle.Graph(w, seed).generate()
    assert m == len(Eo)
    assert len(pieces) > 40  # the graph is ~55 times half the ring
    check_order(pieces, offsets)
    E = np.concatenate([p[3] for p in pieces]).astype(np.int64)
    assert np.array_equal(E, Eo)


def test_stream_int64_and_stop():
    lib()
    from paper_1406_1215_gb300.generator import Generator

    w, seed = inputs.workload("pl_n1e5")
    Eo = oracle.Graph(w, seed).generate()
    g = Generator(cuda(w), seed)
    m, pieces = collect(g, ring_edges=2 * 10000, etype=1)
    assert m == len(Eo) and np.array_equal(np.concatenate([p[3] for p in pieces]), Eo)
    m2, pieces2 = collect(g, ring_edges=2 * 10000, etype=1, stop_after=3)
    assert len(pieces2) == 3 and m2 == sum(len(p[3]) for p in pieces2)
    assert np.array_equal(np.concatenate([p[3] for p in pieces2]), Eo[:m2])
    g.close()


def test_stream_capacity_error():
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    w, seed = inputs.workload("pl_n1e5")
    g = Generator(cuda(w), seed)
    with pytest.raises(P.ClError) as ei:
        collect(g, ring_edges=8)  # half a ring of 4 edges: the heaviest items hold more
    assert ei.value.status == P.CL_ERR_CAPACITY
    g.close()


def test_stream_large_graph_through_small_ring():
    """n = 10^7 (1.4e8 edges, 1.1 GB) through a ring of 2 x 2^21 edges (2 x 16 MB):
    every piece equals the device-resident generation's edges at the same place, and
    sampled items equal the oracle's."""
    lib()
    from paper_1406_1215_gb300.generator import Generator

    w, seed = inputs.workload("pl_n1e7")
    g = Generator(cuda(w), seed)
    ref = g.generate()  # device-resident count + scan + emit
    ref_off = g.offsets.clone()
    n_pieces, sampled = 0, []
    rng = np.random.default_rng(5)
    ring = 1 << 22

    def sink(pairs, first, ib, ie):
        nonlocal n_pieces
        n = pairs.shape[0]
        assert torch.equal(pairs.to("cuda", non_blocking=False), ref[first:first + n])
        if n_pieces % 7 == 0 and ie > ib:
            sampled.append(int(rng.integers(ib, ie)))
        n_pieces += 1
        return False

    m = g.generate_stream(sink, ring)
    assert m == ref.shape[0]
    assert n_pieces >= 60  # the edge list is over 60 times half the ring
    assert torch.equal(g.offsets, ref_off)
    o = oracle.Graph(w, seed)
    off = ref_off.cpu().numpy()
    R = ref.cpu().numpy().astype(np.int64)
    for it in sampled:
        assert np.array_equal(R[off[it]:off[it + 1]], o.generate(it, it + 1)), it
    g.close()
