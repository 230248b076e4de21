"""GB300-native Chung-Lu random-network generator (Alam & Khan, Algorithm 1
with the cost model of Eq. 1-6 and the partition rule of Eq. 3).

The compute path is the CUDA library ``libcl.so`` (built from ``csrc/`` by
``build.py``) behind the C ABI declared in ``include/cl.h``.  This module is
a thin ctypes binding with the same names as the C entry points; torch is
used only for device memory and streams.  There is no CPU fallback: if the
library is missing or no GPU is visible, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcl.so")

CL_OK = 0
STATUS_NAMES = {
    0: "CL_OK", 1: "CL_ERR_INVALID_ARG", 2: "CL_ERR_UNSORTED", 3: "CL_ERR_NONFINITE", 4: "CL_ERR_RANGE",
    5: "CL_ERR_CAPACITY", 6: "CL_ERR_WORKSPACE", 7: "CL_ERR_TIMEOUT", 8: "CL_ERR_CUDA", 9: "CL_ERR_STATE",
    10: "CL_ERR_DEVICE", 11: "CL_ERR_STOPPED",
}
(CL_ERR_INVALID_ARG, CL_ERR_UNSORTED, CL_ERR_NONFINITE, CL_ERR_RANGE, CL_ERR_CAPACITY, CL_ERR_WORKSPACE,
 CL_ERR_TIMEOUT, CL_ERR_CUDA, CL_ERR_STATE, CL_ERR_DEVICE, CL_ERR_STOPPED) = range(1, 12)
CL_W_I32, CL_W_F64 = 0, 1
CL_E_I32, CL_E_I64 = 0, 1
CL_PART_UCP, CL_PART_CP, CL_PART_RRP = 0, 1, 2
HEAVY_W_DEFAULT = 8192.0


class ClError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({cl_status_string(status)})")


class cl_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("wtype", ctypes.c_int32), ("d_w", ctypes.c_void_p),
                ("seed", ctypes.c_uint64), ("heavy_w", ctypes.c_double)]


class cl_tuning(ctypes.Structure):
    _fields_ = [("tasks", ctypes.c_int32), ("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("no_stage", ctypes.c_int32), ("stage_factor", ctypes.c_double), ("partition", ctypes.c_int32),
                ("max_pool_entries", ctypes.c_int64)]


class cl_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("H", ctypes.c_int64), ("n_items", ctypes.c_int64),
                ("item_begin", ctypes.c_int64), ("S_i64", ctypes.c_int64), ("S", ctypes.c_double),
                ("status", ctypes.c_int32)]


class cl_calib_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("init_from_w", ctypes.c_int32)]


class cl_calib_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("max_rel_err", ctypes.c_double), ("S", ctypes.c_double)]


class cl_run_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("fallbacks", ctypes.c_int64), ("ties", ctypes.c_int64),
                ("error", ctypes.c_int32)]


# cl_edge_sink: int32 (*)(void* user, const void* h_edges, int64 first_edge, int64 n_edges,
#                        int64 item_begin, int64 item_end)
EDGE_SINK = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_int64)

_lib = None


def load_library(path: str | None = None):
    """Loads libcl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is not built; run paper_1406_1215_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, i32, i64, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "cl_status_string": ([i32], ctypes.c_char_p),
        "cl_plan_scratch_bytes": ([i32], sz),
        "cl_plan_create": ([P(cl_graph), i32, P(cl_tuning), vp, sz, vp, P(vp)], i32),
        "cl_plan_workspace_bytes": ([vp, P(sz)], i32),
        "cl_plan_build": ([vp, vp, sz, vp], i32),
        "cl_plan_items": ([vp, P(i64)], i32),
        "cl_plan_graph_info": ([vp, i32, P(cl_graph_info)], i32),
        "cl_plan_tasks": ([vp, P(i32), vp, vp, vp], i32),
        "cl_plan_task_clock": ([vp, vp], i32),
        "cl_plan_launch_info": ([vp, P(i32), P(i32)], i32),
        "cl_count": ([vp, vp, vp], i32),
        "cl_scan": ([vp, vp, vp, P(i64), vp], i32),
        "cl_emit": ([vp, vp, i32, vp, i64, i64, i64, vp], i32),
        "cl_generate_batch": ([vp, i32, vp, i64, vp, vp, vp, vp, vp], i32),
        "cl_generate": ([vp, i32, vp, i64, vp, vp, vp, vp], i32),
        "cl_generate_host": ([vp, i32, vp, i64, vp, vp, vp, i32, i32, P(i64), vp], i32),
        "cl_generate_stream": ([vp, i32, vp, vp, i64, vp, vp, EDGE_SINK, vp, P(i64), vp], i32),
        "cl_stats": ([vp, P(cl_run_stats), vp], i32),
        "cl_check": ([vp, vp], i32),
        "cl_plan_destroy": ([vp], None),
        "cl_diag_philox": ([vp, i64, u64, vp, vp], i32),
        "cl_diag_philox_curand": ([vp, i64, u64, vp, vp], i32),
        "cl_diag_neglog": ([vp, vp, i64, vp, vp, vp], i32),
        "cl_diag_skip": ([vp, vp, vp, vp, i64, vp, vp, vp], i32),
        "cl_diag_philox_rate": ([i64, u64, vp, P(ctypes.c_double), vp], i32),
        "cl_diag_neglog1m_f64": ([vp, vp, i64, vp, vp], i32),
        "cl_scan_noalloc": ([vp, i64, vp, vp], i32),
        "cl_expected_degree_workspace_bytes": ([i64], sz),
        "cl_expected_degree": ([vp, i64, ctypes.c_double, vp, vp, sz, vp], i32),
        "cl_expected_degree_adjoint": ([vp, vp, i64, ctypes.c_double, vp, vp, sz, vp], i32),
        "cl_calibrate_workspace_bytes": ([i64], sz),
        "cl_calibrate": ([vp, i64, vp, P(cl_calib_opts), P(cl_calib_report), vp, sz, vp], i32),
    }
    optional = {}
    for name, (args, res) in list(sig.items()) + list(optional.items()):
        if not hasattr(L, name):
            if name in optional:
                continue
            raise RuntimeError(f"{p} does not export {name}")
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor (or an int / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st: int, where: str):
    if st != CL_OK:
        raise ClError(st, where)


# ------------------------------------------------------------------ C ABI names
def cl_status_string(status: int) -> str:
    return load_library().cl_status_string(status).decode()


def cl_plan_scratch_bytes(G: int) -> int:
    return load_library().cl_plan_scratch_bytes(G)


def cl_plan_create(graphs, tuning: cl_tuning | None, d_scratch, scratch_bytes: int, stream=None):
    """graphs: sequence of cl_graph.  Returns the plan handle (int)."""
    arr = (cl_graph * len(graphs))(*graphs)
    out = ctypes.c_void_p()
    st = load_library().cl_plan_create(arr, len(graphs), ctypes.byref(tuning) if tuning else None,
                                       _ptr(d_scratch), scratch_bytes, _stream(stream), ctypes.byref(out))
    _check(st, "cl_plan_create")
    return out.value


def cl_plan_workspace_bytes(plan) -> int:
    b = ctypes.c_size_t()
    _check(load_library().cl_plan_workspace_bytes(plan, ctypes.byref(b)), "cl_plan_workspace_bytes")
    return b.value


def cl_plan_build(plan, d_ws, ws_bytes: int, stream=None):
    _check(load_library().cl_plan_build(plan, _ptr(d_ws), ws_bytes, _stream(stream)), "cl_plan_build")


def cl_plan_items(plan) -> int:
    n = ctypes.c_int64()
    _check(load_library().cl_plan_items(plan, ctypes.byref(n)), "cl_plan_items")
    return n.value


def cl_plan_tasks(plan, d_task_start=None, d_cost_prefix=None, stream=None) -> int:
    """Number of tasks T; copies the task table (T + 1 int64) and the item cost
    prefix (n_items int64, 1/16-edge units) into the given device arrays."""
    T = ctypes.c_int32()
    st = load_library().cl_plan_tasks(plan, ctypes.byref(T), _ptr(d_task_start), _ptr(d_cost_prefix),
                                      _stream(stream))
    _check(st, "cl_plan_tasks")
    return T.value


def cl_plan_task_clock(plan, d_task_ns):
    """Count passes record per-task global-timer stamps into d_task_ns (2 T uint64 /
    int64 device array), or stop doing so when it is None."""
    _check(load_library().cl_plan_task_clock(plan, _ptr(d_task_ns)), "cl_plan_task_clock")


def cl_plan_launch_info(plan):
    """(count-pass grid, threads per block)."""
    g, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().cl_plan_launch_info(plan, ctypes.byref(g), ctypes.byref(b)), "cl_plan_launch_info")
    return g.value, b.value


def cl_plan_graph_info(plan, g: int) -> cl_graph_info:
    info = cl_graph_info()
    _check(load_library().cl_plan_graph_info(plan, g, ctypes.byref(info)), "cl_plan_graph_info")
    return info


def cl_count(plan, d_counts, stream=None):
    _check(load_library().cl_count(plan, _ptr(d_counts), _stream(stream)), "cl_count")


def cl_scan(plan, d_counts, d_offsets, want_total: bool = False, stream=None):
    tot = ctypes.c_int64()
    st = load_library().cl_scan(plan, _ptr(d_counts), _ptr(d_offsets), ctypes.byref(tot) if want_total else None,
                                _stream(stream))
    _check(st, "cl_scan")
    return tot.value if want_total else None


def cl_emit(plan, d_offsets, etype: int, d_edges, capacity: int, item_begin: int, item_end: int, stream=None):
    st = load_library().cl_emit(plan, _ptr(d_offsets), etype, _ptr(d_edges), capacity, item_begin, item_end,
                                _stream(stream))
    _check(st, "cl_emit")


def cl_generate_batch(plan, etype: int, d_edges, capacity: int, d_graph_offsets, d_counts, d_offsets, d_status,
                      stream=None):
    st = load_library().cl_generate_batch(plan, etype, _ptr(d_edges), capacity, _ptr(d_graph_offsets),
                                          _ptr(d_counts), _ptr(d_offsets), _ptr(d_status), _stream(stream))
    _check(st, "cl_generate_batch")


def cl_generate(plan, etype: int, d_edges, capacity: int, d_counts, d_offsets, want_total: bool = True,
                stream=None):
    """count + scan + emit in one call; returns m when want_total (synchronizes), else None."""
    m = ctypes.c_int64(0)
    st = load_library().cl_generate(plan, etype, _ptr(d_edges), capacity, _ptr(d_counts), _ptr(d_offsets),
                                    ctypes.byref(m) if want_total else None, _stream(stream))
    _check(st, "cl_generate")
    return m.value if want_total else None


def cl_generate_host(plan, etype: int, h_edges, capacity: int, d_edges, d_counts, d_offsets, chunks: int = 0,
                     copy_sms: int = 0, stream=None) -> int:
    """Whole plan to host memory (h_edges: pinned tensor or address; d_edges: device
    staging buffer of the same capacity, or None for direct stores); returns m."""
    m = ctypes.c_int64(0)
    st = load_library().cl_generate_host(plan, etype, _ptr(h_edges), capacity, _ptr(d_edges), _ptr(d_counts),
                                         _ptr(d_offsets), chunks, copy_sms, ctypes.byref(m), _stream(stream))
    _check(st, "cl_generate_host")
    return m.value


def cl_generate_stream(plan, etype: int, h_ring, d_ring, ring_edges: int, d_counts, d_offsets, sink,
                       stream=None) -> int:
    """Whole plan delivered piece by piece to sink(h_edges_address, first_edge, n_edges,
    item_begin, item_end) -> bool (True stops) through a host ring and a device ring of
    ring_edges edges each; returns m (or the edges delivered before a stop)."""
    raised = []

    def _cb(user, h, first, n, ib, ie):
        try:
            return 1 if sink(h, first, n, ib, ie) else 0
        except BaseException as e:  # stops the generation; re-raised below
            raised.append(e)
            return 1

    cb = EDGE_SINK(_cb)
    m = ctypes.c_int64(0)
    st = load_library().cl_generate_stream(plan, etype, _ptr(h_ring), _ptr(d_ring), ring_edges, _ptr(d_counts),
                                           _ptr(d_offsets), cb, None, ctypes.byref(m), _stream(stream))
    if raised:
        raise raised[0]
    if st == CL_ERR_STOPPED:
        return m.value
    _check(st, "cl_generate_stream")
    return m.value


def cl_stats(plan, stream=None) -> dict:
    s = cl_run_stats()
    _check(load_library().cl_stats(plan, ctypes.byref(s), _stream(stream)), "cl_stats")
    return {"iterations": s.iterations, "fallbacks": s.fallbacks, "ties": s.ties, "error": s.error}


def cl_check(plan, stream=None) -> int:
    return load_library().cl_check(plan, _stream(stream))


def cl_plan_destroy(plan):
    if plan:
        load_library().cl_plan_destroy(plan)


def cl_expected_degree_workspace_bytes(n: int) -> int:
    return load_library().cl_expected_degree_workspace_bytes(n)


def cl_expected_degree(d_w, n: int, S: float, d_E, d_ws, ws_bytes: int, stream=None):
    _check(load_library().cl_expected_degree(_ptr(d_w), n, S, _ptr(d_E), _ptr(d_ws), ws_bytes, _stream(stream)),
           "cl_expected_degree")


def cl_expected_degree_adjoint(d_w, d_gE, n: int, S: float, d_gw, d_ws, ws_bytes: int, stream=None):
    _check(load_library().cl_expected_degree_adjoint(_ptr(d_w), _ptr(d_gE), n, S, _ptr(d_gw), _ptr(d_ws), ws_bytes,
                                                     _stream(stream)), "cl_expected_degree_adjoint")


def cl_calibrate_workspace_bytes(n: int) -> int:
    return load_library().cl_calibrate_workspace_bytes(n)


def cl_calibrate(d_target, n: int, d_w, opts: cl_calib_opts | None, d_ws, ws_bytes: int, stream=None):
    """Returns (status, report); status CL_ERR_RANGE means the tolerance was not reached."""
    rep = cl_calib_report()
    st = load_library().cl_calibrate(_ptr(d_target), n, _ptr(d_w), ctypes.byref(opts) if opts else None,
                                     ctypes.byref(rep), _ptr(d_ws), ws_bytes, _stream(stream))
    if st not in (CL_OK, 4):
        raise ClError(st, "cl_calibrate")
    return st, {"iterations": rep.iterations, "max_rel_err": rep.max_rel_err, "S": rep.S}


def _check_device_array(t, name: str, dtype, need: int):
    """For torch tensors passed as device arrays: dtype, length and device
    checked before the C call (a raw address is passed through unchecked)."""
    if t is None or isinstance(t, int):
        return
    import torch

    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must be a tensor on the current CUDA device")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() < need:
        raise ValueError(f"{name} must be contiguous with at least {need} elements")


def cl_scan_noalloc(d_counts, n: int, d_offsets, stream=None):
    """cl_scan without a plan, a workspace or any allocation (for callers that
    cannot allocate device memory); its scratch is a fixed array inside the
    library, so concurrent calls race.  n <= 2^28."""
    import torch

    if n < 0:
        raise ValueError("n must be >= 0")
    _check_device_array(d_counts, "d_counts", torch.int32, n)
    _check_device_array(d_offsets, "d_offsets", torch.int64, n + 1)
    _check(load_library().cl_scan_noalloc(_ptr(d_counts), n, _ptr(d_offsets), _stream(stream)), "cl_scan_noalloc")


def cl_diag_philox(d_ctr, count: int, seed: int, d_out, stream=None):
    _check(load_library().cl_diag_philox(_ptr(d_ctr), count, seed, _ptr(d_out), _stream(stream)), "cl_diag_philox")


def cl_diag_philox_curand(d_ctr, count: int, seed: int, d_out, stream=None):
    _check(load_library().cl_diag_philox_curand(_ptr(d_ctr), count, seed, _ptr(d_out), _stream(stream)),
           "cl_diag_philox_curand")


def cl_diag_neglog(d_A, d_B, count: int, d_ff, d_dd, stream=None):
    _check(load_library().cl_diag_neglog(_ptr(d_A), _ptr(d_B), count, _ptr(d_ff), _ptr(d_dd), _stream(stream)),
           "cl_diag_neglog")


def cl_diag_skip(d_a, d_Q, d_S, d_R, count: int, d_delta, d_tier, stream=None):
    st = load_library().cl_diag_skip(_ptr(d_a), _ptr(d_Q), _ptr(d_S), _ptr(d_R), count, _ptr(d_delta), _ptr(d_tier),
                                     _stream(stream))
    _check(st, "cl_diag_skip")


def cl_diag_neglog1m_f64(d_Q, d_S, count: int, d_ff, stream=None):
    _check(load_library().cl_diag_neglog1m_f64(_ptr(d_Q), _ptr(d_S), count, _ptr(d_ff), _stream(stream)),
           "cl_diag_neglog1m_f64")


def cl_diag_philox_rate(iters: int, seed: int, d_sink, stream=None) -> float:
    """Philox4x32-10 blocks per second on this GPU (synchronizing)."""
    r = ctypes.c_double()
    _check(load_library().cl_diag_philox_rate(iters, seed, _ptr(d_sink), ctypes.byref(r), _stream(stream)),
           "cl_diag_philox_rate")
    return r.value


from .generator import Generator, generate  # noqa: E402  (convenience layer over the C ABI)
