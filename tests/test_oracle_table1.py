"""The paper's Table 1 ER row as a pin of the oracle's expected-edge closed
form: an Erdos-Renyi network with 1M nodes and 200M edges is the Chung-Lu
model with every weight 400 (= 2m/n), whose exact E[m] = C(n, 2) * 400^2 / S
with S = 400 n must round to the printed 200M.  (Fixture: tests/golden/.)"""
import json
import math
import os

import numpy as np

import oracle
from paper_1406_1215_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table1_er_row_expected_edges():
    g = json.load(open(os.path.join(HERE, "golden", "table1_er.json")))
    n = g["nodes"]
    d = round(2 * g["edges"] / n)  # 400
    w = inputs.constant_weights(n, d)
    N, S, var = oracle.expected_edges_i32(w)
    Em = N / S
    assert S == d * n
    # the closed form written independently: every pair u < v has p = d^2 / (d n)
    assert N == n * (n - 1) // 2 * d * d
    assert abs(Em - g["edges"]) <= g["edges_rounding"]
    assert abs(var - Em * (1 - d / n)) <= 1e-6 * Em  # sum of p(1-p), p = d/n
    assert math.isclose(2 * Em / n, d - d / n, rel_tol=1e-12)
