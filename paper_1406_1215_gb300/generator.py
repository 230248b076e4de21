"""Convenience layer over the C ABI: owns the device buffers (torch tensors)
that the library needs and calls the entry points in order.  All arithmetic
runs in the CUDA library; this file only allocates and marshals.
"""
from __future__ import annotations

import torch

from . import (CL_E_I32, CL_W_F64, CL_W_I32, HEAVY_W_DEFAULT, cl_count, cl_emit, cl_generate,
               cl_generate_batch, cl_generate_host, cl_generate_stream,
               cl_graph, cl_plan_build, cl_plan_create, cl_plan_destroy, cl_plan_graph_info, cl_plan_items,
               cl_plan_scratch_bytes, cl_plan_workspace_bytes, cl_scan, cl_stats, cl_tuning)


def _wtype(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return CL_W_I32
    if t.dtype == torch.float64:
        return CL_W_F64
    raise TypeError("weights must be int32 or float64")


class Generator:
    """A plan over one or several graphs (sorted non-increasing weights on the
    GPU, one seed each) with its workspace and count / offset buffers."""

    def __init__(self, weights, seeds, heavy_w: float = HEAVY_W_DEFAULT, tasks: int = 0, block: int = 0,
                 blocks_per_sm: int = 0, no_stage: int = 0, stage_factor: float = 0.0, partition: int = 0,
                 max_pool_entries: int = 0, stream=None):
        if isinstance(weights, torch.Tensor):
            weights = [weights]
            seeds = [seeds]
        if len(weights) != len(seeds):
            raise ValueError("one seed per graph")
        for w in weights:
            if not w.is_cuda or not w.is_contiguous():
                raise ValueError("weights must be contiguous CUDA tensors")
        self.weights = list(weights)
        self.seeds = [int(s) for s in seeds]
        self.G = len(self.weights)
        self.device = self.weights[0].device
        self.stream = stream
        graphs = [cl_graph(w.numel(), _wtype(w), w.data_ptr(), s & (2**64 - 1), float(heavy_w))
                  for w, s in zip(self.weights, self.seeds)]
        tun = cl_tuning(tasks, block, blocks_per_sm, no_stage, stage_factor, partition, max_pool_entries)
        sb = cl_plan_scratch_bytes(self.G)
        scratch = torch.empty(sb, dtype=torch.uint8, device=self.device)
        self.plan = cl_plan_create(graphs, tun, scratch, sb, stream)
        del scratch
        wb = cl_plan_workspace_bytes(self.plan)
        self.workspace = torch.empty(wb, dtype=torch.uint8, device=self.device)
        cl_plan_build(self.plan, self.workspace, wb, stream)
        self.n_items = cl_plan_items(self.plan)
        self.counts = torch.empty(max(self.n_items, 1), dtype=torch.int32, device=self.device)
        self.offsets = torch.empty(self.n_items + 1, dtype=torch.int64, device=self.device)
        self.m = None

    def info(self, g: int = 0):
        i = cl_plan_graph_info(self.plan, g)
        return {"n": i.n, "H": i.H, "n_items": i.n_items, "item_begin": i.item_begin, "S_i64": i.S_i64,
                "S": i.S, "status": i.status}

    def count(self):
        cl_count(self.plan, self.counts, self.stream)

    def scan(self, want_total: bool = True):
        m = cl_scan(self.plan, self.counts, self.offsets, want_total, self.stream)
        if want_total:
            self.m = m
        return m

    def emit(self, edges: torch.Tensor | None = None, etype: int = CL_E_I32, item_begin: int = 0,
             item_end: int | None = None) -> torch.Tensor:
        item_end = self.n_items if item_end is None else item_end
        if edges is None:
            if self.m is None:
                self.scan(True)
            dt = torch.int32 if etype == CL_E_I32 else torch.int64
            edges = torch.empty((max(self.m, 1), 2), dtype=dt, device=self.device)
        cap = edges.shape[0] if edges.numel() else 0
        cl_emit(self.plan, self.offsets, etype, edges, cap, item_begin, item_end, self.stream)
        return edges

    def generate(self, etype: int = CL_E_I32) -> torch.Tensor:
        """count -> scan (reads m back) -> emit; returns an (m, 2) tensor."""
        self.count()
        m = self.scan(True)
        dt = torch.int32 if etype == CL_E_I32 else torch.int64
        edges = torch.empty((max(m, 1), 2), dtype=dt, device=self.device)
        self.emit(edges, etype)
        return edges[:m]

    def generate_into(self, edges: torch.Tensor, etype: int = CL_E_I32) -> int:
        """count + scan + emit in one library call into `edges` (a device (capacity, 2)
        tensor); returns m."""
        cap = edges.shape[0] if edges.numel() else 0
        self.m = cl_generate(self.plan, etype, edges, cap, self.counts, self.offsets, True, self.stream)
        return self.m

    def generate_host(self, out: torch.Tensor, etype: int = CL_E_I32, chunks: int = 0, copy_sms: int = 0,
                      staging: torch.Tensor | None = None, direct: bool = False) -> int:
        """count + scan + emit with the edge list delivered into `out`, a host
        tensor of (capacity, 2) pairs (page-locked for full speed); returns m.
        The host transfer of one item range overlaps the sampling of the next.
        staging: device buffer of out's shape for the copy-engine path (made
        here when omitted); direct=True stores straight into `out` instead."""
        if out.is_cuda:
            raise ValueError("out must be a host tensor")
        want = torch.int32 if etype == CL_E_I32 else torch.int64
        if out.dtype != want or out.dim() != 2 or out.shape[1] != 2 or not out.is_contiguous():
            raise ValueError("out must be a contiguous (capacity, 2) tensor of the edge type")
        if not direct and staging is None:
            staging = torch.empty(out.shape, dtype=want, device=self.device)
        if staging is not None and (staging.shape != out.shape or staging.dtype != want or not staging.is_cuda):
            raise ValueError("staging must be a device tensor shaped like out")
        self.m = cl_generate_host(self.plan, etype, out.data_ptr(), out.shape[0], None if direct else staging,
                                  self.counts, self.offsets, chunks, copy_sms, self.stream)
        return self.m

    def generate_stream(self, sink, ring_edges: int, etype: int = CL_E_I32, h_ring: torch.Tensor | None = None,
                        d_ring: torch.Tensor | None = None) -> int:
        """count + scan + emit delivered piece by piece: sink(pairs, first_edge, item_begin,
        item_end) gets a host tensor view (n, 2) of the ring -- valid only during the call --
        and returns True to stop.  The rings (ring_edges pairs, pinned on the host) are made
        here when omitted.  Returns m (or the edges delivered before a stop)."""
        dt = torch.int32 if etype == CL_E_I32 else torch.int64
        if h_ring is None:
            h_ring = torch.empty((ring_edges, 2), dtype=dt, pin_memory=True)
        if d_ring is None:
            d_ring = torch.empty((ring_edges, 2), dtype=dt, device=self.device)
        if h_ring.dtype != dt or h_ring.shape != (ring_edges, 2) or h_ring.is_cuda or not h_ring.is_contiguous():
            raise ValueError("h_ring must be a contiguous host (ring_edges, 2) tensor of the edge type")
        if d_ring.dtype != dt or d_ring.shape != (ring_edges, 2) or not d_ring.is_cuda:
            raise ValueError("d_ring must be a device (ring_edges, 2) tensor of the edge type")

        base, pair_bytes = h_ring.data_ptr(), 2 * h_ring.element_size()

        def cb(h, first, n, ib, ie):
            k = (h - base) // pair_bytes  # the piece sits in one half of the ring
            return sink(h_ring[k:k + n], first, ib, ie)

        self.m = cl_generate_stream(self.plan, etype, h_ring, d_ring, ring_edges, self.counts, self.offsets, cb,
                                    self.stream)
        return self.m

    def generate_batch(self, edges: torch.Tensor, graph_offsets: torch.Tensor, status: torch.Tensor,
                       etype: int = CL_E_I32):
        cap = edges.shape[0]
        cl_generate_batch(self.plan, etype, edges, cap, graph_offsets, self.counts, self.offsets, status,
                          self.stream)

    def stats(self) -> dict:
        return cl_stats(self.plan, self.stream)

    def close(self):
        if getattr(self, "plan", None):
            cl_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(weights: torch.Tensor, seed: int, heavy_w: float = HEAVY_W_DEFAULT, etype: int = CL_E_I32):
    """One graph: returns its (m, 2) edge list (u < v, canonical order)."""
    g = Generator(weights, seed, heavy_w)
    try:
        return g.generate(etype)
    finally:
        g.close()
