"""Pins for the oracle's K-means++ seeding on sparsified rows (Algorithm 1's
initialisation; Arthur & Vassilvitskii's D^2 sampling) and its 64-bit draw."""
import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")


def _tiny_rows():
    # n = 5 rows, m = 2 entries each, pt = 4; distinct rows, distances vary
    idx = np.array([[0, 1], [1, 2], [2, 3], [0, 3], [1, 3]], np.int32)
    val = np.array([[1.0, 2.0], [0.5, -1.0], [3.0, 0.25], [-2.0, 1.5], [0.75, 4.0]], np.float32)
    return idx, val


def _dense(idx, val, pt):
    D = np.zeros((idx.shape[0], pt))
    for i in range(idx.shape[0]):
        D[i, idx[i]] = val[i]
    return D


def _restricted(idx, val, cen):
    """Restricted squared distance of every row to the dense centre cen."""
    return ((val.astype(np.float64) - cen[idx]) ** 2).sum(1)


def test_draw_uniform_small_w():
    W = 7
    draws = np.array([oracle.kpp_draw(11, 0, r, W) for r in range(7000)])
    assert draws.min() >= 0 and draws.max() < W
    counts = np.bincount(draws, minlength=W)
    assert scipy_stats.chisquare(counts).pvalue > 1e-4


def test_draw_rejection_heavy_w():
    W = 2 ** 63 + 1  # (2^64 - W) mod W = 2^63 - 1: about half the words are rejected
    draws = [oracle.kpp_draw(3, 1, r, W) for r in range(2000)]
    assert all(0 <= d < W for d in draws)
    frac = np.array(draws, dtype=np.float64) / float(W)
    assert abs(frac.mean() - 0.5) < 0.05


def test_first_centre_uniform():
    idx, val = _tiny_rows()
    firsts = np.array([oracle.kmeanspp(idx, val, 4, 1, seed=5, r=r)[0][0] for r in range(3000)])
    counts = np.bincount(firsts, minlength=5)
    assert scipy_stats.chisquare(counts).pvalue > 1e-4


def test_second_centre_proportional_to_d2():
    idx, val = _tiny_rows()
    D = _dense(idx, val, 4)
    pairs = np.array([oracle.kmeanspp(idx, val, 4, 2, seed=9, r=r)[0] for r in range(6000)])
    for f in range(5):
        sel = pairs[pairs[:, 0] == f, 1]
        d2 = _restricted(idx, val, D[f])
        assert d2[f] == 0.0
        prob = d2 / d2.sum()
        counts = np.bincount(sel, minlength=5)
        assert counts[f] == 0
        keep = prob > 0
        exp = prob[keep] * counts.sum()
        assert scipy_stats.chisquare(counts[keep], exp).pvalue > 1e-4


def test_duplicates_never_chosen_and_permutation():
    idx, val = _tiny_rows()
    # K = n distinct rows: each row exactly once
    for r in range(50):
        rows, cen = oracle.kmeanspp(idx, val, 4, 5, seed=1, r=r)
        assert sorted(rows.tolist()) == [0, 1, 2, 3, 4]
        # centres are the dense scatters of the chosen rows
        assert np.array_equal(cen, _dense(idx, val, 4)[rows].astype(np.float32))
    # a duplicate of a chosen row has D^2 = 0 and is never picked while others remain
    idx2 = np.vstack([idx, idx[:1]])
    val2 = np.vstack([val, val[:1]])
    for r in range(200):
        rows, _ = oracle.kmeanspp(idx2, val2, 4, 2, seed=2, r=r)
        if rows[0] in (0, 5):
            assert rows[1] not in (0, 5)


def test_all_identical_rows_fall_back_to_uniform():
    idx = np.zeros((6, 2), np.int32)
    idx[:, 1] = 1
    val = np.ones((6, 2), np.float32)
    rows, _ = oracle.kmeanspp(idx, val, 4, 3, seed=4, r=0)
    assert all(0 <= x < 6 for x in rows)
