"""Pins for the oracle's random-number spec: Philox, Lemire, signs, masks.

The mask must be m indices drawn uniformly without replacement (Sec. I-A and
Thm. B1); each index is kept with probability m/p (Lemma B2).  None of these
checks re-types the oracle's code: they test distributional facts and
published known answers."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _chi2_ok(counts, expected, alpha=1e-6):
    """Chi-square goodness of fit; True unless p-value < alpha."""
    from scipy.stats import chi2
    counts = np.asarray(counts, np.float64)
    expected = np.asarray(expected, np.float64)
    stat = float(np.sum((counts - expected) ** 2 / expected))
    dof = counts.size - 1
    return chi2.sf(stat, dof) > alpha, stat


def test_philox_known_answers():
    rows = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(f[0:4], f[4:6])
        assert [int(v) for v in out] == f[6:10]
        rows += 1
    assert rows == 3


def test_lemire_rejection_special_cases():
    # s = 1: every word maps to 0, nothing is rejected (2^32 mod 1 = 0).
    assert oracle.lemire_from_words(1, [0xFFFFFFFF]) == (0, 1)
    # s = 3: 2^32 mod 3 = 1, so the word 0 (low product 0 < 1) is rejected and
    # the next word is used.
    v, used = oracle.lemire_from_words(3, [0, 0xFFFFFFFF])
    assert used == 2 and v == 2
    # s = 2^31 + 1: threshold 2^31 - 1; word 2 gives low product 2 -> rejected,
    # word 1 gives low product 2^31 + 1 -> accepted with value 0.
    s = (1 << 31) + 1
    v, used = oracle.lemire_from_words(s, [2, 1])
    assert used == 2 and v == 0
    # high word maps to the top of the range
    v, used = oracle.lemire_from_words(1024, [0xFFFFFFFF])
    assert (v, used) == (1023, 1)
    # multiply-shift: value = floor(word * s / 2^32)
    for w in [0x12345678, 0x80000000, 0x7FFFFFFF, 0x00000001]:
        low = (w * 1000) & 0xFFFFFFFF
        if low >= (1 << 32) % 1000:
            assert oracle.lemire_from_words(1000, [w]) == ((w * 1000) >> 32, 1)
        else:  # 0x80000000 * 1000 = 0 mod 2^32 -> rejected
            assert oracle.lemire_from_words(1000, [w]) == (0, -1)
    # running out of words is reported
    assert oracle.lemire_from_words(3, [0]) == (0, -1)


def test_lemire_exact_uniformity_small_range():
    """Every value of [0,s) is hit by exactly floor(2^32/s) accepted words.

    Checked by counting accepted words in closed form per output value over a
    sample of words spread across the whole 32-bit range."""
    s = 7
    rng = np.random.default_rng(0)
    words = rng.integers(0, 1 << 32, size=200000, dtype=np.uint64)
    counts = np.zeros(s)
    for w in words[:20000]:
        v, used = oracle.lemire_from_words(s, [int(w), 0x55555555])
        assert 0 <= v < s
        counts[v] += 1
    ok, stat = _chi2_ok(counts, np.full(s, counts.sum() / s))
    assert ok, stat


def test_signs_are_pm1_and_balanced():
    D = oracle.signs(1 << 16, seed=12345)
    assert set(np.unique(D)) <= {-1.0, 1.0}
    # Binomial(65536, 1/2): 6 sigma band
    plus = int(np.sum(D > 0))
    assert abs(plus - 32768) < 6 * math.sqrt(65536 / 4)
    # different seeds give different D; same seed reproduces
    assert not np.array_equal(D, oracle.signs(1 << 16, seed=12346))
    assert np.array_equal(D, oracle.signs(1 << 16, seed=12345))
    # prefix property: D for a smaller p~ is the prefix of a larger one
    assert np.array_equal(oracle.signs(512, 12345), D[:512])


@pytest.mark.parametrize("pt,m", [(8, 1), (8, 3), (8, 8), (64, 8), (1024, 51), (4096, 205),
                                  (8192, 820), (2, 2)])
def test_mask_distinct_in_range(pt, m):
    for row in [0, 1, 7, 123456, (1 << 33) + 5]:
        om = oracle.mask(pt, m, seed=99, row=row)
        assert om.shape == (m,)
        assert om.min() >= 0 and om.max() < pt
        assert len(set(om.tolist())) == m
        if m == pt:
            assert sorted(om.tolist()) == list(range(pt))


def test_mask_rows_independent_and_reproducible():
    a = oracle.mask(1024, 51, 5, 10)
    assert np.array_equal(a, oracle.mask(1024, 51, 5, 10))
    assert not np.array_equal(a, oracle.mask(1024, 51, 5, 11))
    assert not np.array_equal(a, oracle.mask(1024, 51, 6, 10))
    # the first t draws of a row do not depend on m (prefix property of the stream)
    assert np.array_equal(oracle.mask(1024, 20, 5, 10), a[:20])


def test_mask_inclusion_probability_is_m_over_p():
    """Lemma B2: each coordinate is kept with probability m/p."""
    pt, m, rows = 64, 8, 12000
    counts = np.zeros(pt)
    for r in range(rows):
        counts[oracle.mask(pt, m, 2024, r)] += 1
    ok, stat = _chi2_ok(counts, np.full(pt, rows * m / pt))
    assert ok, stat


@pytest.mark.parametrize("m", [2, 3])
def test_mask_ordered_tuples_uniform(m):
    """Uniform without replacement: every ordered m-tuple of distinct indices
    of [0,8) is equally likely (the draw-order statement of Thm. B1's proof)."""
    pt = 8
    tuples = list(itertools.permutations(range(pt), m))
    index = {t: i for i, t in enumerate(tuples)}
    rows = 60 * len(tuples)
    counts = np.zeros(len(tuples))
    for r in range(rows):
        counts[index[tuple(oracle.mask(pt, m, 77, r).tolist())]] += 1
    ok, stat = _chi2_ok(counts, np.full(len(tuples), rows / len(tuples)))
    assert ok, stat


def test_mask_pair_frequency():
    """P(j and l both kept) = m(m-1)/(p(p-1)) (the alpha_2 count in Thm. B1)."""
    pt, m, rows = 16, 4, 20000
    pair = np.zeros((pt, pt))
    for r in range(rows):
        om = oracle.mask(pt, m, 31337, r)
        for a in om:
            for b in om:
                if a != b:
                    pair[a, b] += 1
    expected = rows * m * (m - 1) / (pt * (pt - 1))
    off = pair[~np.eye(pt, dtype=bool)]
    ok, stat = _chi2_ok(off, np.full(off.size, expected))
    assert ok, stat


def test_init_rows_distinct():
    rows = oracle.init_rows(2000, 5, 1)
    assert len(set(rows.tolist())) == 5 and rows.min() >= 0 and rows.max() < 2000
    assert np.array_equal(rows, oracle.init_rows(2000, 5, 1))


def test_stream_layout_matches_written_spec():
    """The oracle's word layout is the written spec: signs from word (j/32)%4
    of block (j/128, 0, 0, TAG_SIGN); mask words w from word w%4 of block
    (w/4, r_lo, r_hi, TAG_MASK), consumed by Lemire then Fisher-Yates."""
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    D = oracle.signs(512, seed)
    for j in [0, 1, 31, 32, 127, 128, 300, 511]:
        word = int(oracle.philox4x32_10([j // 128, 0, 0, oracle.TAG_SIGN], key)[(j // 32) % 4])
        assert D[j] == (-1.0 if (word >> (j % 32)) & 1 else 1.0)
    pt, m, row = 32, 10, (7 << 32) | 3
    words = []
    for b in range(16):
        words += [int(v) for v in oracle.philox4x32_10(
            [b, row & 0xFFFFFFFF, row >> 32, oracle.TAG_MASK], key)]
    a = list(range(pt))
    pos = 0
    expect = []
    for t in range(m):
        v, used = oracle.lemire_from_words(pt - t, words[pos:])
        pos += used
        k = t + v
        a[t], a[k] = a[k], a[t]
        expect.append(a[t])
    assert oracle.mask(pt, m, seed, row).tolist() == expect
