"""Edge lists delivered to host memory (cl_generate_host) against the CPU
oracle, element by element: both pipelines (device staging + copy engines,
and kernels storing straight into mapped host memory), each overlapping the
host transfer of one item range with the sampling of the next, must give
exactly the edges of Algorithm 1 in canonical order, for any number of
ranges, both edge types, staged and unstaged plans and items that outgrow
their staging slots.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def oracle_edges(w, seed, heavy_w=8192.0):
    g = oracle.Graph(w, seed, heavy_w)
    return g.generate(counts=g.count_items())


def host_edges(w, seed, etype=0, chunks=0, copy_sms=0, slack=16, heavy_w=8192.0, direct=False, **tun):
    lib()
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(cuda(w), seed, heavy_w=heavy_w, **tun)
    dt = torch.int32 if etype == 0 else torch.int64
    m_dev = g.generate(etype).shape[0]  # the device path, for the size and the comparison
    out = torch.full((m_dev + slack, 2), -7, dtype=dt, pin_memory=True)
    m = g.generate_host(out, etype, chunks=chunks, copy_sms=copy_sms, direct=direct)
    st = g.stats()
    g.close()
    assert st["error"] == 0, st
    assert m == m_dev
    assert (out[m:] == -7).all()  # nothing written past the edge list
    return out[:m].numpy().astype(np.int64)


@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("chunks", [1, 3, 8, 64])
def test_host_output_matches_oracle(chunks, direct):
    w, seed = inputs.workload("pl_n1e5")
    E = host_edges(w, seed, chunks=chunks, direct=direct)
    assert np.array_equal(E, oracle_edges(w, seed))


@pytest.mark.parametrize("direct", [False, True])
def test_host_output_heavy_segments_int64(direct):
    # heavy rows cut into many 2^16 segments; wide ids
    w = inputs.powerlaw_degrees(300000, 2.1, 2, 20000, 31)
    E = host_edges(w, 5, etype=1, chunks=5, heavy_w=600.0, direct=direct)
    assert np.array_equal(E, oracle_edges(w, 5, heavy_w=600.0))


@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("tun", [{"no_stage": 1}, {"stage_factor": -1.0}, {"tasks": 7}, {"copy": 1}])
def test_host_output_paths(tun, direct):
    # unstaged plan (every edge regenerated), 8-entry slots (most items go through
    # the regeneration list of their range), fewer tasks than ranges, one copy SM
    w = inputs.powerlaw_degrees(40000, 2.2, 3, 3000, 33)
    tun = dict(tun)
    copy_sms = 1 if tun.pop("copy", None) else 0
    E = host_edges(w, 17, chunks=6, copy_sms=copy_sms, direct=direct, **tun)
    assert np.array_equal(E, oracle_edges(w, 17))


def test_host_output_capacity_and_arguments():
    P = lib()
    from paper_1406_1215_gb300.generator import Generator

    w = inputs.powerlaw_degrees(20000, 2.2, 3, 800, 34)
    g = Generator(cuda(w), 3)
    m = g.generate().shape[0]
    for direct in (False, True):
        small = torch.zeros((m // 2, 2), dtype=torch.int32, pin_memory=True)
        with pytest.raises(P.ClError) as e:
            g.generate_host(small, direct=direct)
        assert e.value.status == P.CL_ERR_CAPACITY
        g.stats()  # clear the device error word
    # pageable memory: fine through the copy engines; for direct stores accepted
    # only where the GPU addresses it (a coherent CPU-GPU link)
    pageable = torch.zeros((m, 2), dtype=torch.int32)
    assert g.generate_host(pageable) == m
    assert np.array_equal(pageable.numpy().astype(np.int64), oracle_edges(w, 3))
    pageable.zero_()
    mm = ctypes.c_int64(0)
    st = P.load_library().cl_generate_host(g.plan, 0, pageable.data_ptr(), m, None, g.counts.data_ptr(),
                                           g.offsets.data_ptr(), 0, 0, ctypes.byref(mm), None)
    assert st in (P.CL_OK, P.CL_ERR_INVALID_ARG)
    if st == P.CL_OK:
        assert mm.value == m
        assert np.array_equal(pageable.numpy().astype(np.int64), oracle_edges(w, 3))
    out = torch.zeros((m, 2), dtype=torch.int32, pin_memory=True)
    assert g.generate_host(out) == m  # usable after both errors
    assert np.array_equal(out.numpy().astype(np.int64), oracle_edges(w, 3))
    g.close()


def test_host_output_trivial_graphs():
    lib()
    from paper_1406_1215_gb300.generator import Generator

    for n in (1, 2, 3):
        w = np.full(n, 5, dtype=np.int32)
        g = Generator(cuda(w), 1)
        out = torch.zeros((4, 2), dtype=torch.int32, pin_memory=True)
        m = g.generate_host(out)
        E = oracle_edges(w, 1)
        assert m == len(E)
        assert np.array_equal(out[:m].numpy().astype(np.int64), E)
        g.close()
