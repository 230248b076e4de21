"""The C-ABI library loads and exports every entry point include/cl.h
declares; host-side argument checks answer without a GPU; the product
package never imports the oracle.  No compute call is made here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cl_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1406_1215_gb300 import build as B

    B.build()
    import paper_1406_1215_gb300 as P

    return P.load_library()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_host_side_argument_checks(L):
    import ctypes

    import paper_1406_1215_gb300 as P

    out = ctypes.c_void_p(123)
    assert L.cl_plan_create(None, 0, None, None, 0, None, ctypes.byref(out)) == 1
    assert out.value is None
    assert P.cl_status_string(2).startswith("weights are not sorted")
    g = (P.cl_graph * 1)(P.cl_graph(5, 7, 1234, 1, 8192.0))  # bad weight type
    assert L.cl_plan_create(g, 1, None, None, 0, None, ctypes.byref(out)) == 1
    g = (P.cl_graph * 1)(P.cl_graph(1 << 31, 0, 1234, 1, 8192.0))  # n too large for int32 ids
    assert L.cl_plan_create(g, 1, None, None, 0, None, ctypes.byref(out)) == 4
    g = (P.cl_graph * 1)(P.cl_graph(10, 0, 1234, 1, 8192.0))  # no scratch
    assert L.cl_plan_create(g, 1, None, None, 0, None, ctypes.byref(out)) == 6
    # scratch that is not 256-byte aligned is refused before it is touched
    sb = L.cl_plan_scratch_bytes(1)
    assert L.cl_plan_create(g, 1, None, ctypes.c_void_p(0x10000010), sb, None, ctypes.byref(out)) == 1
    assert out.value is None
    assert L.cl_diag_skip(None, None, None, None, -1, None, None, None) == 1
    m = ctypes.c_int64(5)
    assert L.cl_generate_host(None, 0, None, 0, None, None, None, 0, 0, ctypes.byref(m), None) == 1
    assert L.cl_generate_host(None, 0, None, 0, None, None, None, 65, 0, ctypes.byref(m), None) == 1
    assert L.cl_generate_stream(None, 0, None, None, 0, None, None, ctypes.cast(None, P.EDGE_SINK), None,
                                ctypes.byref(m), None) == 1
    T = ctypes.c_int32(7)
    assert L.cl_plan_tasks(None, ctypes.byref(T), None, None, None) == 1
    assert L.cl_plan_task_clock(None, None) == 1
    assert L.cl_diag_philox_rate(0, 0, None, None, None) == 1
    assert P.cl_status_string(11).startswith("the caller's edge sink")
    assert L.cl_plan_scratch_bytes(4) > L.cl_plan_scratch_bytes(1) > 0


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1406_1215_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "cl_oracle" not in text and "liboracle" not in text, f
