"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The block function is pinned to the generator's published known-answer
vectors (tests/golden/philox4x32_10_kat.txt): a wrong round permutation,
swapped high and low product halves, a missing key bump or a wrong multiplier
changes every one of them.  The statistics tests below check the properties
the method relies on: uniform output words, full avalanche of every counter
and key bit, and independence of the four output words.  On a GPU,
tests/test_gpu_philox.py compares the same vectors and a sweep of counters
with cuRAND's device Philox4_32_10, run as a library.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def kat_vectors():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            assert len(w) == 10
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors():
    rows = kat_vectors()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = [int(x) for x in oracle.philox4x32_10(ctr, key)]
        assert got == want, f"ctr={ctr} key={key}: {[hex(x) for x in got]} != {[hex(x) for x in want]}"


def _batch(ctrs, key):
    return np.array([oracle.philox4x32_10(c, key) for c in ctrs], dtype=np.uint64)


def test_output_bytes_uniform():
    from scipy.stats import chi2
    out = _batch([[i, 7, 3, 0] for i in range(6000)], [12345, 678])
    bytes_ = np.concatenate([(out >> s) & 0xFF for s in (0, 8, 16, 24)]).ravel()
    counts = np.bincount(bytes_.astype(np.int64), minlength=256)
    exp = len(bytes_) / 256
    stat = float(((counts - exp) ** 2 / exp).sum())
    assert chi2.sf(stat, 255) > 1e-4


def test_avalanche_counter_and_key_bits():
    rng = np.random.default_rng(0)
    base = rng.integers(0, 2**32, size=(60, 4), dtype=np.uint64)
    keys = rng.integers(0, 2**32, size=(60, 2), dtype=np.uint64)
    fr_ctr, fr_key = [], []
    for c, k in zip(base, keys):
        o0 = oracle.philox4x32_10(c, k)
        for word in range(4):
            for bit in range(0, 32, 3):
                c2 = c.copy()
                c2[word] ^= np.uint64(1 << bit)
                o1 = oracle.philox4x32_10(c2, k)
                fr_ctr.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(o0, o1)) / 128)
        for word in range(2):
            for bit in range(0, 32, 5):
                k2 = k.copy()
                k2[word] ^= np.uint64(1 << bit)
                o1 = oracle.philox4x32_10(c, k2)
                fr_key.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(o0, o1)) / 128)
    assert abs(np.mean(fr_ctr) - 0.5) < 0.01
    assert abs(np.mean(fr_key) - 0.5) < 0.01
    assert min(fr_ctr) > 0.25  # no counter bit leaves most of the output alone


def test_words_uncorrelated_and_distinct_streams():
    out = _batch([[i, 0, 3, 0] for i in range(5000)], [1, 0]).astype(np.float64) / 2**32
    C = np.corrcoef(out.T)
    assert np.all(np.abs(C - np.eye(4)) < 0.05)
    # different stream words give different draws for the same id
    a = oracle.philox4x32_10([5, 0, 1, 0], [1, 0])
    b = oracle.philox4x32_10([5, 0, 2, 0], [1, 0])
    assert not np.array_equal(a, b)


def test_distinct_counters_distinct_outputs():
    out = _batch([[i, 0, 0, 0] for i in range(4000)], [0, 0])
    as_int = [tuple(r) for r in out]
    assert len(set(as_int)) == len(as_int)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_uniform_mapping_exact(n):
    # u = (r >> 8) 2^-24 lies in [0, 1) and is exact in FP32
    r = oracle.philox4x32_10([n, 0, 3, 0], [9, 0])
    for w in r:
        u = (int(w) >> 8) / 2.0**24
        assert 0.0 <= u < 1.0
        assert float(np.float32(u)) == u
