"""The autotuner (launch knobs only): every candidate must reproduce the first
candidate's output element for element (the tuner checks that itself), and
that output must equal the CPU oracle's edge lists graph by graph -- so every
candidate's output equals the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def test_batch_tuning_candidates_equal_the_oracle():
    lib()
    from paper_1406_1215_gb300 import autotune

    work = inputs.batch_workload(40)
    views = [cuda(w) for w, _ in work]
    seeds = [s for _, s in work]
    best, timings, (edges, goff) = autotune.tune(views, seeds, reps=1, use_cache=False, return_output=True)
    assert len(timings) >= 8
    assert best in [t["knobs"] for t in timings]
    E = edges.cpu().numpy().astype(np.int64)
    go = goff.cpu().numpy()
    for g, (w, s) in enumerate(work):
        Eo = oracle.Graph(w, s).generate()
        assert np.array_equal(E[go[g]:go[g + 1]], Eo), g


def test_single_graph_tuning_equals_the_oracle():
    lib()
    from paper_1406_1215_gb300 import autotune

    w, seed = inputs.workload("pl_n1e5")
    best, timings, (edges, goff) = autotune.tune(cuda(w), seed, reps=1, use_cache=False, return_output=True)
    assert len(timings) >= 8
    Eo = oracle.Graph(w, seed).generate()
    assert np.array_equal(edges.cpu().numpy().astype(np.int64), Eo)
