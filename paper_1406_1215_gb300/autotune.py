"""Autotuner for the launch knobs of a plan (cl_tuning: tasks, block,
blocks_per_sm).  Knobs never change the output, and the tuner checks that:
every candidate's full edge list (and its per-graph offsets) must equal the
first candidate's, element for element.  Candidates are timed with CUDA
events on the call the plan is used for: cl_generate_batch for a batch,
cl_generate (count + scan + emit) for one graph.  Results are cached as JSON
keyed by the GPU, its SM count and a size class of the plan.
"""
from __future__ import annotations

import json
import os

import torch

from . import cl_plan_launch_info
from .generator import Generator

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1406_1215_gb300", "tuning.json")


def default_candidates(resident_warps: int):
    """Task granularity (tasks per resident warp of the count pass), block size and
    blocks per SM: ten points around the defaults."""
    W = max(1, resident_warps)
    c = [{}]
    c += [{"tasks": m * W} for m in (1, 4, 16, 64, 256)]
    c += [{"block": 128}, {"block": 128, "blocks_per_sm": 4}, {"blocks_per_sm": 2}, {"blocks_per_sm": 2, "tasks": 16 * W}]
    return c


def _key(n_items: int, G: int) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    size_class = max(0, n_items.bit_length() - 16)
    return f"{p.name}|{p.multi_processor_count}|{'G1' if G == 1 else 'Gmany'}|items2^{size_class}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def _run(g: Generator, edges: torch.Tensor, goff: torch.Tensor, status: torch.Tensor) -> None:
    if g.G > 1:
        g.generate_batch(edges, goff, status)
    else:
        g.generate_into(edges)


def tune(weights, seeds, candidates=None, reps: int = 2, use_cache: bool = True, return_output: bool = False):
    """Returns (best knobs, timings) -- and, with return_output, the reference
    output (edges (m, 2) int32 and per-graph offsets (G + 1)) that every
    candidate reproduced.  weights/seeds as for Generator."""
    if isinstance(weights, torch.Tensor):
        weights, seeds = [weights], [seeds]
    n_items_hint = sum(int(w.numel()) for w in weights)
    key = _key(n_items_hint, len(weights))
    cache = _load() if use_cache else {}
    if use_cache and key in cache and not return_output:
        return cache[key]["best"], cache[key]["timings"]
    dev = weights[0].device
    probe = Generator(weights, seeds)
    grid, block = cl_plan_launch_info(probe.plan)
    probe.count()
    m = probe.scan(True)
    probe.close()
    candidates = candidates or default_candidates(grid * block // 32)
    G = len(weights)
    ref_edges, ref_goff = None, None
    edges = torch.empty((m + 1024, 2), dtype=torch.int32, device=dev)
    goff = torch.empty(G + 1, dtype=torch.int64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    timings = []
    for knobs in candidates:
        g = Generator(weights, seeds, **knobs)
        edges.fill_(-1)
        _run(g, edges, goff, status)
        torch.cuda.synchronize()
        if G > 1 and int(status.item()) != 0:
            g.close()
            raise RuntimeError(f"tuning {knobs}: status {int(status.item())}")
        if ref_edges is None:
            ref_edges, ref_goff = edges[:m].clone(), goff.clone()
        elif not (torch.equal(edges[:m], ref_edges) and (G == 1 or torch.equal(goff, ref_goff))):
            g.close()
            raise RuntimeError(f"tuning {knobs} changed the output")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            a.record()
            _run(g, edges, goff, status)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b) / 1e3)
        timings.append({"knobs": knobs, "seconds": best})
        g.close()
    del edges
    best = min(timings, key=lambda r: r["seconds"])["knobs"]
    if use_cache:
        cache[key] = {"best": best, "timings": timings}
        _save(cache)
    if return_output:
        if G == 1:
            ref_goff = torch.tensor([0, m], dtype=torch.int64, device=dev)
        return best, timings, (ref_edges, ref_goff)
    return best, timings
