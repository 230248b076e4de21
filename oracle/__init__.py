"""CPU oracle for the Chung-Lu edge-skipping generator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_1406_1215_gb300``) never does.  The C source (``cl_oracle.c``) is a
plain single-threaded restatement of Algorithm 1 (Serial-CL / Create-Edges),
the cost model (Eq. 1, 2, 6) and the partition rule (Eq. 3) of Alam & Khan,
with closed forms used as pins.  It shares no code with the CUDA library.

Parity pins (what ties this oracle to something other than itself) live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cl_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

W_I32 = 0
W_F64 = 1
HEAVY_W_DEFAULT = 8192.0


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "cl_oracle.h"))
    ):
        return _SO
    cmd = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", _SO + ".tmp", _SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    subprocess.check_call(cmd)
    os.replace(_SO + ".tmp", _SO)
    return _SO


class _Graph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("wtype", ctypes.c_int32),
        ("w", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("heavy_w", ctypes.c_double),
        ("S_f64", ctypes.c_double),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("S_i64", ctypes.c_int64),
        ("S", ctypes.c_double),
        ("H", ctypes.c_int64),
        ("n_heavy_items", ctypes.c_int64),
        ("n_items", ctypes.c_int64),
        ("status", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int64),
        ("fallbacks", ctypes.c_int64),
        ("unresolved", ctypes.c_int64),
    ]

    def as_dict(self):
        return {"iterations": self.iterations, "fallbacks": self.fallbacks, "unresolved": self.unresolved}


_lib = None
_P = ctypes.POINTER


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, u32, u64, dbl, vp = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
        L.or_philox4x32_10.argtypes = [_P(u32), u32, u32]
        L.or_uniform53.argtypes = [u32, u32]
        L.or_uniform53.restype = dbl
        L.or_skip.argtypes = [dbl, dbl, dbl, i64, _P(Stats)]
        L.or_skip.restype = i64
        L.or_skip_x_quad.argtypes = [dbl, dbl, dbl, _P(dbl), _P(dbl)]
        L.or_neglog_ratio_quad.argtypes = [dbl, dbl, _P(dbl), _P(dbl)]
        L.or_neglog1m_quad.argtypes = [dbl, dbl, _P(dbl), _P(dbl)]
        L.or_analyze.argtypes = [_P(_Graph), _P(_Info)]
        L.or_analyze.restype = ctypes.c_int32
        L.or_item_bounds.argtypes = [_P(_Graph), _P(_Info), i64, _P(i64), _P(u32), _P(i64), _P(i64)]
        L.or_item_bounds.restype = ctypes.c_int32
        L.or_generate_item.argtypes = [_P(_Graph), _P(_Info), i64, vp, i64, _P(Stats)]
        L.or_generate_item.restype = i64
        L.or_count_items.argtypes = [_P(_Graph), _P(_Info), i64, i64, vp, _P(Stats)]
        L.or_generate_items.argtypes = [_P(_Graph), _P(_Info), i64, i64, vp, i64, _P(Stats)]
        L.or_generate_items.restype = i64
        L.or_item_costs.argtypes = [_P(_Graph), _P(_Info), vp]
        L.or_ucp_starts.argtypes = [vp, i64, i64, vp]
        L.or_calc_cost.argtypes = [vp, i64, i64, vp]
        L.or_expected_edges_i32.argtypes = [vp, i64, _P(u64), _P(u64), _P(i64), _P(dbl)]
        L.or_expected_edges_bruteforce_i32.argtypes = [vp, i64, _P(u64), _P(u64)]
        for name in ("or_expected_degree", "or_expected_degree_bruteforce"):
            getattr(L, name).argtypes = [vp, i64, dbl, vp]
        for name in ("or_expected_degree_adjoint", "or_expected_degree_adjoint_bruteforce",
                     "or_expected_degree_adjoint_pairwise"):
            getattr(L, name).argtypes = [vp, i64, dbl, vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    """Philox4x32-10 block for counter ``ctr`` (4 words) and key ``key`` (2 words)."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    lib().or_philox4x32_10(c, int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF)
    return [int(x) for x in c]


def uniform53(lo: int, hi: int) -> float:
    return lib().or_uniform53(lo, hi)


def skip(r: float, Q: float, S: float, R: int, stats: Stats | None = None) -> int:
    """min(floor(ln r / ln(1 - Q/S)), R): the skip of Algorithm 1."""
    return lib().or_skip(r, Q, S, R, ctypes.byref(stats) if stats is not None else None)


def skip_x_quad(r: float, Q: float, S: float):
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib().or_skip_x_quad(r, Q, S, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def neglog1m_quad(Q: float, S: float):
    """-ln(1 - Q/S) for doubles 0 < Q < S in binary128, as (hi, lo) doubles."""
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib().or_neglog1m_quad(Q, S, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def neglog_ratio_quad(A: float, B: float):
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib().or_neglog_ratio_quad(A, B, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


# ---------------------------------------------------------------- graphs
class Graph:
    """One Chung-Lu instance: sorted non-increasing weights, a seed and the
    heavy-row threshold (rows with w_u >= heavy_w are cut into 2^16-wide
    v-segments)."""

    def __init__(self, w: np.ndarray, seed: int, heavy_w: float = HEAVY_W_DEFAULT):
        if w.dtype == np.int32:
            self.w = np.ascontiguousarray(w)
            wtype, S_f64 = W_I32, 0.0
        elif w.dtype == np.float64:
            self.w = np.ascontiguousarray(w)
            wtype = W_F64
            S_f64 = math.fsum(self.w.tolist())  # correctly rounded sum of the weights
        else:
            raise TypeError("weights must be int32 or float64")
        self._g = _Graph(len(self.w), wtype, self.w.ctypes.data, seed & (2**64 - 1), float(heavy_w), S_f64)
        self._i = _Info()
        lib().or_analyze(ctypes.byref(self._g), ctypes.byref(self._i))
        self.n = len(self.w)
        self.seed = seed
        self.heavy_w = heavy_w

    @property
    def status(self):
        return self._i.status

    @property
    def S(self):
        return self._i.S_i64 if self._g.wtype == W_I32 else self._i.S

    @property
    def H(self):
        return self._i.H

    @property
    def n_items(self):
        return self._i.n_items

    @property
    def n_heavy_items(self):
        return self._i.n_heavy_items

    def item_bounds(self, item: int):
        u, j0, end = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        seg = ctypes.c_uint32()
        rc = lib().or_item_bounds(
            ctypes.byref(self._g), ctypes.byref(self._i), item, ctypes.byref(u), ctypes.byref(seg),
            ctypes.byref(j0), ctypes.byref(end))
        if rc != 0:
            raise IndexError(item)
        return u.value, seg.value, j0.value, end.value

    def generate_item(self, item: int, stats: Stats | None = None) -> np.ndarray:
        st = ctypes.byref(stats) if stats is not None else None
        c = lib().or_generate_item(ctypes.byref(self._g), ctypes.byref(self._i), item, None, 0, None)
        out = np.empty(max(c, 1), dtype=np.int64)
        c2 = lib().or_generate_item(ctypes.byref(self._g), ctypes.byref(self._i), item, _ptr(out), c, st)
        assert c2 == c
        return out[:c]

    def count_items(self, ib: int = 0, ie: int | None = None, stats: Stats | None = None) -> np.ndarray:
        ie = self.n_items if ie is None else ie
        out = np.empty(max(ie - ib, 1), dtype=np.int32)
        lib().or_count_items(ctypes.byref(self._g), ctypes.byref(self._i), ib, ie, _ptr(out),
                             ctypes.byref(stats) if stats is not None else None)
        return out[: ie - ib]

    def generate(self, ib: int = 0, ie: int | None = None, stats: Stats | None = None,
                 counts: np.ndarray | None = None) -> np.ndarray:
        """Edges of items [ib, ie) as an (m, 2) int64 array in canonical order."""
        ie = self.n_items if ie is None else ie
        if counts is None:
            counts = self.count_items(ib, ie)
        cap = int(counts.astype(np.int64).sum())
        out = np.empty((max(cap, 1), 2), dtype=np.int64)
        m = lib().or_generate_items(ctypes.byref(self._g), ctypes.byref(self._i), ib, ie, _ptr(out), cap,
                                    ctypes.byref(stats) if stats is not None else None)
        assert m == cap, (m, cap)
        return out[:m]

    def item_costs(self) -> np.ndarray:
        c = np.empty(max(self.n_items, 1), dtype=np.float64)
        lib().or_item_costs(ctypes.byref(self._g), ctypes.byref(self._i), _ptr(c))
        return c[: self.n_items]


def ucp_starts(c: np.ndarray, T: int) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(T + 1, dtype=np.int64)
    lib().or_ucp_starts(_ptr(c), len(c), T, _ptr(out))
    return out


def calc_cost(c: np.ndarray, P: int) -> np.ndarray:
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(max(len(c), 1), dtype=np.float64)
    lib().or_calc_cost(_ptr(c), len(c), P, _ptr(out))
    return out[: len(c)]


def expected_edges_i32(w: np.ndarray):
    """(N, S, Var): E[m] = N / S exactly (N as a Python int), Var[m] = sum p(1-p)."""
    w = np.ascontiguousarray(w, dtype=np.int32)
    hi, lo, S, var = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64(), ctypes.c_double()
    lib().or_expected_edges_i32(_ptr(w), len(w), ctypes.byref(hi), ctypes.byref(lo), ctypes.byref(S),
                                ctypes.byref(var))
    return (hi.value << 64) | lo.value, S.value, var.value


def expected_edges_bruteforce_i32(w: np.ndarray) -> int:
    w = np.ascontiguousarray(w, dtype=np.int32)
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    lib().or_expected_edges_bruteforce_i32(_ptr(w), len(w), ctypes.byref(hi), ctypes.byref(lo))
    return (hi.value << 64) | lo.value


def weight_sum_f64(w: np.ndarray) -> float:
    """S for double weights: the correctly rounded sum (math.fsum)."""
    return math.fsum(np.asarray(w, dtype=np.float64).tolist())


def expected_degree(w: np.ndarray, S: float | None = None, brute: bool = False) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    S = weight_sum_f64(w) if S is None else S
    E = np.empty(max(len(w), 1), dtype=np.float64)
    fn = lib().or_expected_degree_bruteforce if brute else lib().or_expected_degree
    fn(_ptr(w), len(w), S, _ptr(E))
    return E[: len(w)]


def expected_degree_adjoint(w: np.ndarray, gE: np.ndarray, S: float | None = None,
                            brute: bool = False, pairwise: bool = False) -> np.ndarray:
    """Gradient of sum_u gE_u E_u(w).  brute: O(n^3) term by term; pairwise: O(n^2)
    pair sums; default: O(n log n) with sorted cap thresholds and suffix sums."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    gE = np.ascontiguousarray(gE, dtype=np.float64)
    S = weight_sum_f64(w) if S is None else S
    g = np.empty(max(len(w), 1), dtype=np.float64)
    if brute:
        fn = lib().or_expected_degree_adjoint_bruteforce
    elif pairwise:
        fn = lib().or_expected_degree_adjoint_pairwise
    else:
        fn = lib().or_expected_degree_adjoint
    fn(_ptr(w), len(w), S, _ptr(gE), _ptr(g))
    return g[: len(w)]
