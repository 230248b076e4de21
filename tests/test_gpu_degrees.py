"""Degree-distribution accuracy of generated graphs (the paper's Section 5
accuracy experiment, Fig. 4: generated against expected degrees), on the GPU
at sizes the oracle cannot reach.

For every node, d_u is a sum of independent Bernoulli(p_uv) (Algorithm 1 is an
exact sampler of the Chung-Lu model with the cap min(1, w_u w_v / S)), so for a
set B of nodes the sum of degrees has mean sum_{u in B} E_u and variance at
most 2 sum_{u in B} E_u (an edge with both ends in B counts twice).  Nodes are
binned by weight; every bin's z-score must be below 6 in magnitude.

With capping, E_u < w_u for heavy nodes (the paper's w_u - w_u^2/S is the
uncapped form), so generating with w = d misses the target degrees of the
heaviest nodes by many standard deviations; calibrated weights (cl_calibrate)
remove that bias.  Both effects are asserted.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1406_1215_gb300 import inputs
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def degrees(w: torch.Tensor, seed: int) -> torch.Tensor:
    from paper_1406_1215_gb300.generator import Generator

    g = Generator(w, seed)
    E = g.generate()
    st = g.stats()
    g.close()
    assert st["error"] == 0 and st["ties"] == 0
    n = w.numel()
    d = torch.bincount(E[:, 0].long(), minlength=n) + torch.bincount(E[:, 1].long(), minlength=n)
    del E
    return d.double()


def expected(w: np.ndarray, S: float) -> np.ndarray:
    """Capped expected degrees from the CPU oracle (O(n log n): sorted cap thresholds and
    suffix sums), independent of the GPU's own expected-degree kernel."""
    return oracle.expected_degree(np.asarray(w, dtype=np.float64), S)


def binned_z(key: np.ndarray, got: np.ndarray, want: np.ndarray, title: str):
    """z = (sum got - sum want) / sqrt(2 sum want) per log2 bin of key; prints the table."""
    b = np.floor(np.log2(key)).astype(np.int64)
    rows = []
    for k in np.unique(b):
        m = b == k
        sg, sw = float(got[m].sum()), float(want[m].sum())
        z = (sg - sw) / math.sqrt(2.0 * sw) if sw > 0 else 0.0
        rows.append((int(k), int(m.sum()), sg / m.sum(), sw / m.sum(), z))
    print(f"\n{title}\n  bin(log2)     nodes   mean deg   mean expected        z")
    for r in rows:
        print(f"  {r[0]:9d} {r[1]:9d} {r[2]:10.3f} {r[3]:15.3f} {r[4]:8.2f}")
    return rows


def test_power_law_degrees_match_capped_expectation():
    lib()
    w_np, seed = inputs.workload("pl_n1e7")
    w = cuda(w_np)
    S = float(w_np.astype(np.int64).sum())
    d = degrees(w, seed).cpu().numpy()
    E = expected(w_np, S)
    rows = binned_z(w_np.astype(np.float64), d, E, "pl_n1e7 (gamma 2.5 on [10, 1e4]): generated vs capped expectation")
    assert max(abs(r[4]) for r in rows) < 6.0
    assert abs(d.sum() / 2 - E.sum() / 2) < 6 * math.sqrt(E.sum())


def test_erdos_renyi_degree_histogram_is_binomial():
    lib()
    n, c = 10_000_000, 100
    w_np = inputs.constant_weights(n, c)
    d = degrees(cuda(w_np), 7).cpu().numpy().astype(np.int64)
    p = c * c / (n * c)  # every pair has p = c/n
    mean = (n - 1) * p
    assert abs(d.mean() - mean) < 6 * math.sqrt(2 * mean / n)
    # histogram against Binomial(n - 1, p) over the central range, chi-square per bin
    lgam = math.lgamma
    ks = np.arange(60, 141)
    pmf = np.exp([lgam(n) - lgam(k + 1) - lgam(n - k) + k * math.log(p) + (n - 1 - k) * math.log1p(-p) for k in ks])
    obs = np.bincount(d, minlength=ks[-1] + 1)[ks]
    expct = n * pmf
    chi2 = float(((obs - expct) ** 2 / expct).sum())
    dof = len(ks) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), chi2


def test_calibration_removes_the_cap_bias():
    lib()
    from paper_1406_1215_gb300.calibration import calibrate

    target = inputs.calibration_targets()
    t = cuda(target)
    w, rep = calibrate(t, tol=1e-9)
    assert rep["converged"], rep
    d_cal = degrees(w, 11).cpu().numpy()
    d_raw = degrees(t, 11).cpu().numpy()  # w = d: the uncapped reading of Section 3
    rows_cal = binned_z(target, d_cal, target, "calibrated weights: generated vs target degrees")
    rows_raw = binned_z(target, d_raw, target, "w = target degrees: generated vs target degrees")
    assert max(abs(r[4]) for r in rows_cal) < 6.0
    assert min(r[4] for r in rows_raw) < -6.0  # the heaviest bins fall short without calibration
