"""Pins for the oracle's index stream (Algorithm 1, sampling step).

The paper only states that the s*b indices of an outer iteration are drawn
i.i.d. uniformly with replacement; the generator chosen here is
Philox4x64-10 (Salmon et al., SC'11).  Its oracle implementation is pinned
to numpy.random.Philox, an independent implementation of the same published
generator, and the row mapping floor(U m / 2^64) to Python big integers."""
import math

import numpy as np
import pytest

import oracle


def _numpy_block(ctr0, key):
    # numpy's Philox increments its 256-bit counter before each block, so the
    # block for counter (k,0,0,0) is produced from a start counter of k-1.
    start = (ctr0 - 1) % (1 << 256)
    words = [(start >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    bg = np.random.Philox(counter=np.array(words, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


@pytest.mark.parametrize("ctr0,key", [
    (0, (0, 0)), (1, (0, 0)), (7, (123, 9)), (2**40 + 3, (2**63 + 5, 77)),
    (2**64 - 1, (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF)), (12345, (42, 0)),
])
def test_philox_matches_numpy(ctr0, key):
    got = [int(v) for v in oracle.philox4x64_10([ctr0 % (1 << 64), 0, 0, 0], key)]
    assert got == _numpy_block(ctr0, key)


def test_philox_random_counters_and_keys():
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        k = (int(rng.integers(0, 2**63)), int(rng.integers(0, 2**63)))
        got = [int(v) for v in oracle.philox4x64_10([c, 0, 0, 0], k)]
        assert got == _numpy_block(c, k)


def test_draw_word_layout():
    # draw q takes word q mod 4 of block q div 4, key (seed, problem)
    seed, prob = 0xDEADBEEF12345678, 3
    for q in [0, 1, 2, 3, 4, 5, 1023, 4096 * 7 + 2]:
        blk = _numpy_block(q // 4, (seed, prob))
        assert oracle.draw_word(seed, prob, q) == blk[q % 4]


@pytest.mark.parametrize("m", [1, 2, 3, 8192, 1_048_576, 400_000, 2**31 - 1])
def test_row_mapping_bigint(m):
    seed, prob = 11, 0
    idx = oracle.sample_indices(seed, prob, 1000, 64, m)
    for i, v in enumerate(idx):
        U = oracle.draw_word(seed, prob, 1000 + i)
        assert v == (U * m) >> 64
        assert 0 <= v < m


def test_indices_uniform_chi_square():
    m, N = 64, 200_000
    idx = oracle.sample_indices(0, 0, 0, N, m)
    counts = np.bincount(idx, minlength=m)
    expected = N / m
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    # chi-square with 63 dof: mean 63, sd ~11.2; 5 sd bound
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    assert chi2 > 63 - 5 * math.sqrt(2 * 63)


def test_indices_are_a_function_of_draw_number():
    # the stream is counter-based: a slice equals the slice of a longer draw,
    # and distinct problems give distinct streams
    long = oracle.sample_indices(3, 1, 0, 1000, 977)
    assert np.array_equal(long[333:500], oracle.sample_indices(3, 1, 333, 167, 977))
    other = oracle.sample_indices(3, 2, 0, 1000, 977)
    assert not np.array_equal(long, other)
