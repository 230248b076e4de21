"""The seeded input generators (no GPU): sorted non-increasing int32 weights on the
stated support, reproducible from the seed, distributed as the stated power law, and
batch parameters inside their stated ranges."""
import math

import numpy as np

from paper_1406_1215_gb300 import inputs


def test_powerlaw_sorted_in_range_and_reproducible():
    w = inputs.powerlaw_degrees(200_000, 2.5, 2, 1000, 7)
    assert w.dtype == np.int32 and len(w) == 200_000
    assert np.all(np.diff(w) <= 0)
    assert w.min() >= 2 and w.max() <= 1000
    assert np.array_equal(w, inputs.powerlaw_degrees(200_000, 2.5, 2, 1000, 7))
    assert not np.array_equal(w, inputs.powerlaw_degrees(200_000, 2.5, 2, 1000, 8))


def test_powerlaw_follows_its_law():
    """Chi-square of the value counts against d^-gamma / Z over the bins with at least
    50 expected draws (the rest pooled); the 1e-6 quantile bound keeps the test stable."""
    n, gamma, a, b = 1_000_000, 2.3, 3, 400
    w = inputs.powerlaw_degrees(n, gamma, a, b, 11)
    d = np.arange(a, b + 1)
    p = d.astype(np.float64) ** -gamma
    p /= p.sum()
    obs = np.array([np.count_nonzero(w == x) for x in d], dtype=np.float64)
    exp = n * p
    big = exp >= 50
    o = np.append(obs[big], obs[~big].sum())
    e = np.append(exp[big], exp[~big].sum())
    chi2 = float(((o - e) ** 2 / e).sum())
    k = len(o) - 1
    # Wilson-Hilferty: chi2_k quantile at z standard deviations
    z = 4.75  # upper 1e-6 tail
    bound = k * (1 - 2 / (9 * k) + z * math.sqrt(2 / (9 * k))) ** 3
    assert chi2 < bound, (chi2, bound, k)


def test_constant_weights_and_named_workloads():
    w = inputs.constant_weights(1000, 100)
    assert w.dtype == np.int32 and np.all(w == 100)
    w5, seed = inputs.workload("pl_n1e5")
    assert len(w5) == 100_000 and seed == 42 and w5.min() >= 2 and w5.max() <= 1000
    try:
        inputs.workload("no_such_workload")
        raise AssertionError("unknown workload accepted")
    except KeyError:
        pass


def test_batch_parameters_in_range():
    for g in range(0, 4096, 97):
        n, gamma, a, b = inputs.batch_graph_params(g)
        assert 1000 <= n < 1_000_000
        assert 2.1 <= gamma < 3.0
        assert a == 2 and b == max(2, math.isqrt(n))
        assert inputs.batch_graph_params(g) == (n, gamma, a, b)
    work = inputs.batch_workload(3)
    assert [s for _, s in work] == [0, 1, 2]
    for (w, _), g in zip(work, range(3)):
        n, _, a, b = inputs.batch_graph_params(g)
        assert len(w) == n and w.min() >= a and w.max() <= b and np.all(np.diff(w) <= 0)
