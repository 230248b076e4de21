"""GPU primitives against independent references, through the C ABI.

* Philox4x32-10: the library's kernel = cuRAND's device Philox (called, an
  independent implementation) = the CPU oracle, on arbitrary counters.
* -ln(A/B): float-float and double-double values against the oracle's
  binary128 logarithm; float-float must stay within 2^-44 relative (the skip
  accepts only results farther than 2^-40 x from an integer) and
  double-double within 2^-98.
* The two-tier skip decision against the oracle's exact floor, including
  cases built to sit within an ulp of an integer.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from tests.gpu_util import cuda, lib

pytestmark = pytest.mark.gpu


def test_philox_matches_curand_device_and_oracle():
    P = lib()
    rng = np.random.default_rng(1)
    N = 1 << 20
    ctr = rng.integers(0, 2**32, (N, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:64] = 0
    ctr[:16, 0] = np.arange(16)
    for seed in (0, 42, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        d_ctr = cuda(ctr.view(np.int32))
        a = torch.empty(N * 4, dtype=torch.int32, device="cuda")
        b = torch.empty(N * 4, dtype=torch.int32, device="cuda")
        P.cl_diag_philox(d_ctr, N, seed, a)
        P.cl_diag_philox_curand(d_ctr, N, seed, b)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        got = a.cpu().numpy().view(np.uint32).reshape(N, 4)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for i in list(range(32)) + list(rng.integers(0, N, 200)):
            assert list(got[i]) == oracle.philox4x32_10(ctr[i].tolist(), key)


def _neglog_cases(rng):
    A, B = [], []
    two53 = 1 << 53
    # L_r: r = (2k+1)/2^53 over its whole range, dense near 0, 1/2 and 1
    k = rng.integers(0, 2**52, 60000, dtype=np.uint64)
    A += [2 * int(x) + 1 for x in k]
    B += [two53] * len(k)
    for edge in list(range(0, 2000)) + [2**52 - 1 - i for i in range(2000)] + [2**51 + i - 1000 for i in range(2000)]:
        A.append(2 * edge + 1)
        B.append(two53)
    # the leading word of the pair small (2^10 <= hi < 2^32: every shift of the 32-bit
    # reduction) and the rounding of J up to 1024
    for j in range(29, 53):
        for d in (0, 1, 2**8 - 1, 2**19 + 7):
            k = (1 << j) + d if (1 << j) + d < 2**52 else (1 << j) - 1 - d
            A.append(2 * k + 1)
            B.append(two53)
        kk = (1 << j) - 1  # all ones: J rounds up
        A.append(2 * kk + 1)
        B.append(two53)
    # L_p: A = S - Q for S up to 2^50, p from 1/S to 1 - 1/S
    for _ in range(60000):
        S = int(rng.integers(2, 2**int(rng.integers(2, 51))))
        mode = rng.integers(0, 4)
        if mode == 0:
            Q = int(rng.integers(1, min(S, 1000)))  # tiny p
        elif mode == 1:
            Q = S - int(rng.integers(1, min(S, 1000) + 0)) if S > 1 else 1  # p near 1
        elif mode == 2:
            Q = max(1, min(S - 1, S // 2 + int(rng.integers(-3, 4))))  # near 1/2
        else:
            Q = int(rng.integers(1, S))
        Q = max(1, min(S - 1, Q))
        A.append(S - Q)
        B.append(S)
    return np.array(A, dtype=np.uint64), np.array(B, dtype=np.uint64)


def test_neglog_ratio_accuracy_against_binary128():
    P = lib()
    rng = np.random.default_rng(2)
    A, B = _neglog_cases(rng)
    n = len(A)
    dff = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    ddd = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    P.cl_diag_neglog(cuda(A.view(np.int64)), cuda(B.view(np.int64)), n, dff, ddd)
    torch.cuda.synchronize()
    f = dff.cpu().numpy().reshape(n, 2).astype(np.float64)
    d = ddd.cpu().numpy().reshape(n, 2)
    worst_ff, worst_dd = 0.0, 0.0
    for i in range(n):
        hi, lo = oracle.neglog_ratio_quad(float(A[i]), float(B[i]))
        ref = hi
        # float-float value as an exact sum of two floats, compared in double pairs
        eff = abs((f[i, 0] - hi) + (f[i, 1] - lo)) / ref
        edd = abs((d[i, 0] - hi) + (d[i, 1] - lo)) / ref
        worst_ff = max(worst_ff, eff)
        worst_dd = max(worst_dd, edd)
    assert worst_ff <= 2.0**-44, math.log2(worst_ff)
    assert worst_dd <= 2.0**-98, math.log2(max(worst_dd, 1e-300))


def test_skip_two_tier_matches_oracle_exact_floor():
    P = lib()
    rng = np.random.default_rng(3)
    a, Q, S, R = [], [], [], []
    # random cases over all scales
    for _ in range(100000):
        s = int(rng.integers(2, 2**int(rng.integers(2, 45))))
        q = int(rng.integers(1, s))
        a.append(int(rng.integers(0, 2**52)))
        Q.append(q)
        S.append(s)
        R.append(int(rng.integers(1, 2**31)))
    # boundary cases: r on the grid point nearest (1-p)^k, from exact integers
    for _ in range(3000):
        s = int(rng.integers(3, 10**7))
        q = int(rng.integers(1, s))
        kmax = int(min(60, 36.0 / -math.log1p(-q / s)))
        if kmax < 1:
            continue
        kk = int(rng.integers(1, kmax + 1))
        t = ((s - q) ** kk * 2**53) // s**kk
        for x in ((t - 1) // 2 - 1, (t - 1) // 2, (t - 1) // 2 + 1):
            if 0 <= x < 2**52:
                a.append(x)
                Q.append(q)
                S.append(s)
                R.append(10**6)
    # the dyadic exact-integer case
    a.append(0), Q.append(1), S.append(2), R.append(1000)
    n = len(a)
    A_ = np.array(a, dtype=np.uint64)
    Q_ = np.array(Q, dtype=np.uint64)
    S_ = np.array(S, dtype=np.uint64)
    R_ = np.array(R, dtype=np.int64)
    delta = torch.empty(n, dtype=torch.int64, device="cuda")
    tier = torch.empty(n, dtype=torch.int32, device="cuda")
    P.cl_diag_skip(cuda(A_.view(np.int64)), cuda(Q_.view(np.int64)), cuda(S_.view(np.int64)), cuda(R_), n, delta, tier)
    torch.cuda.synchronize()
    dg = delta.cpu().numpy()
    tg = tier.cpu().numpy()
    bad = []
    for i in range(n):
        r = (2 * int(A_[i]) + 1) * 2.0**-53
        ref = oracle.skip(r, float(Q_[i]), float(S_[i]), int(R_[i]))
        if ref != dg[i]:
            bad.append((i, int(A_[i]), int(Q_[i]), int(S_[i]), int(R_[i]), int(dg[i]), ref, int(tg[i])))
    assert not bad, bad[:10]
    assert (tg == 1).sum() > 0  # the near-boundary cases reach the double-double tier
    assert tg[-1] == 2 and dg[-1] == 53  # x = 53 exactly: tie rule gives the exact floor


def test_neglog1m_from_doubles_against_binary128():
    """-ln(1 - Q/S) for double weights (float-float from the doubles, the sampler's
    tier 1) within 2^-44 relative of the oracle's binary128 value, over p from
    1e-15 to 1 - 1e-12, both sides of the series bound p = 2^-12, and S from 1 to 1e12
    (1e-30 to 1e30 just above the bound)."""
    P = lib()
    import oracle

    rng = np.random.default_rng(21)
    Q, S = [], []
    for _ in range(20000):
        s = 10.0 ** rng.uniform(0, 12)
        lp = rng.uniform(-15, 0)
        p = min(10.0 ** lp, 1 - 1e-12)
        q = s * p
        if 0 < q < s:
            Q.append(q)
            S.append(s)
    for _ in range(4000):  # just above the series bound, where S - Q's rounding matters most
        s = 10.0 ** rng.uniform(-30, 30)
        q = s * 2.0 ** -12 * (1 + rng.uniform(0, 0.01))
        if 0 < q < s:
            Q.append(q)
            S.append(s)
    for s in (1.0, 3.0, 7.8e9, 2.5e11):  # exactly at and around the series bound
        for p in (2.0 ** -12, 2.0 ** -12 * (1 - 2.0 ** -40), 2.0 ** -12 * (1 + 2.0 ** -40), 0.5, 1 - 2.0 ** -30):
            if 0 < s * p < s:
                Q.append(s * p)
                S.append(s)
    Qa, Sa = np.array(Q), np.array(S)
    n = len(Qa)
    out = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    P.cl_diag_neglog1m_f64(cuda(Qa), cuda(Sa), n, out)
    torch.cuda.synchronize()
    f = out.cpu().numpy().reshape(n, 2).astype(np.float64)
    worst = 0.0
    for i in range(n):
        hi, lo = oracle.neglog1m_quad(float(Qa[i]), float(Sa[i]))
        ref = hi + lo
        err = abs((f[i, 0] - hi) + (f[i, 1] - lo)) / ref
        worst = max(worst, err)
    assert worst < 2.0 ** -44, worst
