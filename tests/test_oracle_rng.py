"""Pins of the oracle's random stream (CPU only).

* Philox4x32-10 against NVIDIA cuRAND's host-side (CPU) Philox generator,
  an independent implementation; its sequence steps counter word 2 under a
  64-bit key (both key words non-zero).
* The uniform mapping r = (2k+1)/2^53: end points never reached, exactness,
  and uniformity.
"""
import numpy as np
import pytest

import oracle
from tests import _curand_host


def test_philox_matches_curand_host_generator():
    seed = 0x0123456789ABCDEF
    nblk = 4096
    words = _curand_host.philox_host_words(seed, 4 * nblk)
    if words is None:
        pytest.skip("cuRAND host library not loadable")
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(nblk):
        assert oracle.philox4x32_10((0, 0, i, 0), key) == words[4 * i: 4 * i + 4], i


def test_philox_matches_curand_with_offset_and_other_seeds():
    for seed in (0, 1, 42, 2**64 - 1, 0xDEADBEEF00000000):
        for off in (0, 3, 1000):
            words = _curand_host.philox_host_words(seed, 64, offset=4 * off)
            if words is None:
                pytest.skip("cuRAND host library not loadable")
            key = (seed & 0xFFFFFFFF, seed >> 32)
            for i in range(16):
                assert oracle.philox4x32_10((0, 0, off + i, 0), key) == words[4 * i: 4 * i + 4]


def test_philox_every_counter_word_and_key_word_matters():
    base = oracle.philox4x32_10((1, 2, 3, 4), (5, 6))
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        assert oracle.philox4x32_10(c, (5, 6)) != base
    assert oracle.philox4x32_10((1, 2, 3, 4), (4, 6)) != base
    assert oracle.philox4x32_10((1, 2, 3, 4), (5, 7)) != base


def test_uniform53_endpoints_and_grid():
    assert oracle.uniform53(0, 0) == 2.0**-53
    assert oracle.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0**-53
    # low 12 bits of the 64-bit word are dropped
    assert oracle.uniform53(0xFFF, 0) == 2.0**-53
    assert oracle.uniform53(0x1000, 0) == 3 * 2.0**-53
    # hi word is the high half
    assert oracle.uniform53(0, 1) == (2 * 2**20 + 1) * 2.0**-53


def test_uniform53_is_uniform():
    rng = np.random.default_rng(7)
    lo = rng.integers(0, 2**32, 20000, dtype=np.uint64)
    hi = rng.integers(0, 2**32, 20000, dtype=np.uint64)
    r = np.array([oracle.uniform53(int(a), int(b)) for a, b in zip(lo, hi)])
    assert r.min() > 0 and r.max() < 1
    hist, _ = np.histogram(r, bins=20, range=(0, 1))
    exp = len(r) / 20
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
