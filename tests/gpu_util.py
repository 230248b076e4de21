"""Shared helpers of the GPU tests: build-once, device tensors, and a spawn
pool that runs the CPU oracle over item ranges in parallel."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_built = False


def lib():
    """Builds (once) and loads the CUDA library; the tests call it through the C ABI."""
    global _built
    import paper_1406_1215_gb300 as P
    from paper_1406_1215_gb300 import build as B

    if not _built:
        B.build()
        _built = True
    P.load_library()
    return P


def cuda(x, dtype=None):
    import torch

    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ---------------------------------------------------------------- oracle pool
_W = None


def _init_worker(path, dtype, n):
    global _W
    _W = np.memmap(path, dtype=dtype, mode="r", shape=(n,))


def _count_range(args):
    import oracle

    seed, heavy_w, ib, ie = args
    g = oracle.Graph(np.asarray(_W), seed, heavy_w)
    st = oracle.Stats()
    c = g.count_items(ib, ie, st)
    return ib, c, st.as_dict()


def _edges_range(args):
    import oracle

    seed, heavy_w, ib, ie = args
    g = oracle.Graph(np.asarray(_W), seed, heavy_w)
    return ib, g.generate(ib, ie)


def oracle_parallel(w: np.ndarray, seed: int, heavy_w: float, ranges, what: str, tmpdir: str, procs: int | None = None):
    """Runs the oracle on item ranges in a spawn pool (the weights are shared
    through a read-only memory map).  what = 'count' or 'edges'."""
    path = os.path.join(tmpdir, f"w_{os.getpid()}_{id(w)}.bin")
    mm = np.memmap(path, dtype=w.dtype, mode="w+", shape=w.shape)
    mm[:] = w
    mm.flush()
    del mm
    procs = procs or min(16, os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    fn = _count_range if what == "count" else _edges_range
    with ctx.Pool(procs, initializer=_init_worker, initargs=(path, w.dtype, len(w))) as pool:
        out = pool.map(fn, [(seed, heavy_w, a, b) for a, b in ranges])
    os.remove(path)
    return out


def split_ranges(n_items: int, parts: int):
    b = np.linspace(0, n_items, parts + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(parts) if b[i + 1] > b[i]]
