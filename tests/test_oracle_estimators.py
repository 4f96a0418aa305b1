"""Pins for the oracle's covariance and sample-mean estimators.

Exhaustive enumeration over every mask at p = 8 gives the exact expectation
over the sampling randomness; the paper fixes what that expectation must be:
E[C_emp-hat] = C_emp + (p-m)/(m-1) diag(C_emp) (Appendix C), E[C_n] = C_emp
(Sec. V, unbiasedness) and E[mean-hat] = mean (Sec. IV)."""
import itertools

import numpy as np
import pytest

import oracle


def _all_masks(pt, m):
    return list(itertools.combinations(range(pt), m))


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8])
def test_cov_unbiased_by_enumeration(m):
    pt = 8
    rng = np.random.default_rng(m)
    y = rng.standard_normal(pt)
    masks = _all_masks(pt, m)
    acc_n = np.zeros((pt, pt))
    acc_emp = np.zeros((pt, pt))
    P, M = float(pt), float(m)
    for om in masks:
        idx = np.array([om], np.int32)
        val = y[idx]
        G = oracle.gram(idx, val, pt)
        acc_emp += P * (P - 1) / (M * (M - 1)) * G
        acc_n += oracle.cov_finalize(G, 1, m)
    acc_n /= len(masks)
    acc_emp /= len(masks)
    C = np.outer(y, y)
    assert np.max(np.abs(acc_n - C)) < 1e-14 * max(1.0, np.max(np.abs(C))) * 10
    expect_emp = C + (P - M) / (M - 1) * np.diag(np.diag(C))
    assert np.max(np.abs(acc_emp - expect_emp)) < 1e-13
    # E[diag C_emp-hat] = (p-1)/(m-1) diag C_emp
    assert np.allclose(np.diag(acc_emp), (P - 1) / (M - 1) * np.diag(C), rtol=1e-13, atol=1e-14)


def test_cov_unbiased_multi_row_draw_order_irrelevant():
    """Several rows; masks enumerated as ordered tuples (draw order) at m=2."""
    pt, m = 8, 2
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((3, pt))
    tuples = list(itertools.permutations(range(pt), m))
    total = np.zeros((pt, pt))
    for i in range(3):
        acc = np.zeros((pt, pt))
        for om in tuples:
            idx = np.array([om], np.int32)
            acc += oracle.cov_finalize(oracle.gram(idx, Y[i][idx], pt), 1, m)
        total += acc / len(tuples)
    total /= 3
    assert np.max(np.abs(total - Y.T @ Y / 3)) < 1e-13


def test_cov_full_sampling_is_plain_gram():
    """m = p: no correction, C_n = (1/n) Y^T Y exactly (Sec. V)."""
    pt, n = 16, 25
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((n, pt))
    idx = np.stack([rng.permutation(pt) for _ in range(n)]).astype(np.int32)
    val = np.take_along_axis(Y, idx, axis=1)
    C = oracle.cov(idx, val, pt)
    assert np.max(np.abs(C - Y.T @ Y / n)) < 1e-13


def test_gram_brute_force_dense_scatter():
    pt, n, m = 32, 20, 5
    rng = np.random.default_rng(9)
    idx = np.stack([rng.choice(pt, m, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, m))
    W = np.zeros((n, pt))
    for i in range(n):
        W[i, idx[i]] = val[i]
    assert np.max(np.abs(oracle.gram(idx, val, pt) - W.T @ W)) < 1e-13


def test_cov_rejects_nothing_but_scales_correctly():
    """Off-diagonal factor p(p-1)/(m(m-1)), diagonal factor p/m (their product
    with 1 - (p-m)/(p-1))."""
    pt, m, n = 8, 3, 2
    G = np.arange(64, dtype=np.float64).reshape(8, 8)
    C = oracle.cov_finalize(G, n, m)
    off = pt * (pt - 1) / (m * (m - 1)) / n
    assert np.allclose(C[0, 1], off * G[0, 1], rtol=1e-15)
    assert np.allclose(C[3, 3], pt / m / n * G[3, 3], rtol=1e-14)


@pytest.mark.parametrize("m", [1, 3, 8])
def test_sample_mean_unbiased_by_enumeration(m):
    pt = 8
    y = np.random.default_rng(11).standard_normal(pt)
    acc = np.zeros(pt)
    masks = _all_masks(pt, m)
    for om in masks:
        idx = np.array([om], np.int32)
        acc += oracle.sample_mean(idx, y[idx], pt)
    assert np.max(np.abs(acc / len(masks) - y)) < 1e-14


def test_sampling_matrix_moments_by_enumeration():
    """Thm. B1: E[R R^T] = (m/p) I and E[R R^T x x^T R R^T] =
    m(m-1)/(p(p-1)) x x^T + m(p-m)/(p(p-1)) diag(x x^T), via the oracle Gram
    (one row, val = x[mask], so G = R R^T x x^T R R^T)."""
    pt, m = 8, 3
    x = np.random.default_rng(2).standard_normal(pt)
    acc = np.zeros((pt, pt))
    acc1 = np.zeros(pt)
    masks = _all_masks(pt, m)
    for om in masks:
        idx = np.array([om], np.int32)
        acc += oracle.gram(idx, x[idx], pt)
        acc1[list(om)] += 1
    acc /= len(masks)
    acc1 /= len(masks)
    assert np.allclose(acc1, m / pt, rtol=1e-15)
    P, M = float(pt), float(m)
    expect = M * (M - 1) / (P * (P - 1)) * np.outer(x, x) + \
        M * (P - M) / (P * (P - 1)) * np.diag(x * x)
    assert np.max(np.abs(acc - expect)) < 1e-14


@pytest.mark.parametrize("m", [2, 3, 5])
def test_cov_centred_unbiased_by_enumeration(m):
    """The centred estimate C_n - xbar xbar^T + B(C_n)/n, averaged over every
    pair of masks of two rows (independent masks per row, Sec. I-A), equals
    the centred second moment (1/n) Y^T Y - ybar ybar^T of the rows.
    Without the correction B the average would be off by the covariance of
    xbar; a wrong sign or a swapped diagonal/off-diagonal term fails here."""
    pt, n = 8, 2
    rng = np.random.default_rng(40 + m)
    Y = rng.standard_normal((n, pt)) + 0.7
    masks = _all_masks(pt, m)
    acc = np.zeros((pt, pt))
    for om0 in masks:
        for om1 in masks:
            idx = np.array([om0, om1], np.int32)
            val = np.take_along_axis(Y, idx, axis=1)
            G = oracle.gram(idx, val, pt)
            mean = oracle.sample_mean(idx, val, pt)
            acc += oracle.cov_centred(G, mean, n, m)
    acc /= len(masks) ** 2
    ybar = Y.mean(axis=0)
    expect = Y.T @ Y / n - np.outer(ybar, ybar)
    assert np.max(np.abs(acc - expect)) < 1e-13


def test_cov_centred_full_sampling_is_plain_centred_gram():
    """m = p: every row is kept whole, the correction vanishes and the
    estimate is the centred second moment itself."""
    pt, n = 16, 30
    rng = np.random.default_rng(12)
    Y = rng.standard_normal((n, pt)) - 1.5
    idx = np.stack([rng.permutation(pt) for _ in range(n)]).astype(np.int32)
    val = np.take_along_axis(Y, idx, axis=1)
    C = oracle.cov_centred(oracle.gram(idx, val, pt), oracle.sample_mean(idx, val, pt), n, pt)
    ybar = Y.mean(axis=0)
    assert np.max(np.abs(C - (Y.T @ Y / n - np.outer(ybar, ybar)))) < 1e-13


def test_cov_centred_needs_its_correction():
    """The plain plug-in C_n - xbar xbar^T is biased: its mask average misses
    the centred second moment by the covariance of xbar, B(C_emp)/n, which the
    correction term of the centred estimate removes (checked at p = 8)."""
    pt, n, m = 8, 2, 3
    rng = np.random.default_rng(77)
    Y = rng.standard_normal((n, pt)) + 0.3
    masks = _all_masks(pt, m)
    acc = np.zeros((pt, pt))
    for om0 in masks:
        for om1 in masks:
            idx = np.array([om0, om1], np.int32)
            val = np.take_along_axis(Y, idx, axis=1)
            xbar = oracle.sample_mean(idx, val, pt)
            acc += oracle.cov(idx, val, pt) - np.outer(xbar, xbar)
    acc /= len(masks) ** 2
    ybar = Y.mean(axis=0)
    target = Y.T @ Y / n - np.outer(ybar, ybar)
    Ce = Y.T @ Y / n
    P, M = float(pt), float(m)
    B = (P - M) / M * (np.diag(np.diag(Ce)) - (Ce - np.diag(np.diag(Ce))) / (P - 1))
    assert np.max(np.abs(acc - target)) > 1e-2
    assert np.max(np.abs(acc - (target - B / n))) < 1e-13
