"""Pins for the oracle's sparsified K-means (Sec. VI-B, Algorithm 1).

* m = p: J' reduces to the K-means objective on HDX and, HD being orthonormal,
  the iterations are Lloyd's on X after un-mixing (Sec. VI-A).
* Brute-force restricted distances on tiny inputs (Eq. (assignments)).
* Coordinate descent: J' never increases (Sec. VI-B, steps 1 and 2).
"""
import numpy as np
import pytest

import oracle
from paper_1511_00152_gb300 import synth


def lloyd(X, C0, iters):
    """Textbook Lloyd's iterations; empty clusters keep their centre."""
    C = C0.copy()
    labels = None
    for _ in range(iters):
        d = ((X[:, None, :] - C[None, :, :]) ** 2).sum(-1)
        labels = np.argmin(d, axis=1)
        for k in range(C.shape[0]):
            sel = labels == k
            if sel.any():
                C[k] = X[sel].mean(0)
    return labels, C


def test_full_sampling_reduces_to_lloyd():
    n, p, K, seed = 300, 16, 4, 21
    X, _, _ = synth.mixture(n, p, K, seed=5, heavy_frac=0.0)
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, pt, seed)
    rows = oracle.init_rows(n, K, seed)
    Y = oracle.precondition(X, seed)
    labels, mu, _ = oracle.kmeans(idx, val, Y[rows], pt, iters=6)
    ref_labels, ref_C = lloyd(X.astype(np.float64), X[rows].astype(np.float64), 6)
    # the oracle loop assigns then updates; the final labels are the ones the
    # last update used, which matches lloyd's last assignment
    assert np.array_equal(labels, ref_labels)
    assert np.max(np.abs(oracle.unmix(mu, p, seed) - ref_C)) < 1e-11


def test_assign_brute_force_and_ties():
    rng = np.random.default_rng(4)
    pt, m, n, K = 16, 5, 30, 6
    idx = np.stack([rng.choice(pt, m, replace=False) for _ in range(n)]).astype(np.int32)
    val = rng.standard_normal((n, m))
    mu = rng.standard_normal((K, pt))
    mu[3] = mu[1]  # exact duplicate centre: ties must resolve to k = 1
    labels, dist = oracle.kmeans_assign(idx, val, mu, pt)
    for i in range(n):
        d = [sum((val[i, t] - mu[k, idx[i, t]]) ** 2 for t in range(m)) for k in range(K)]
        best = int(np.argmin(d))  # numpy argmin returns the first minimum
        assert labels[i] == best and labels[i] != 3
        assert abs(dist[i] - d[best]) < 1e-12


def test_assign_uses_restricted_norm():
    """A centre with huge values on coordinates the row did not sample must
    not be penalised (Eq. (assignments) only sees Omega_i)."""
    pt = 8
    idx = np.array([[0, 1]], np.int32)
    val = np.array([[1.0, 1.0]])
    mu = np.zeros((2, pt))
    mu[0, :2] = 0.0
    mu[1, :2] = 1.0
    mu[1, 2:] = 1e6
    labels, dist = oracle.kmeans_assign(idx, val, mu, pt)
    assert labels[0] == 1 and dist[0] == 0.0


def test_update_unsampled_and_empty_keep_previous():
    pt, K = 8, 3
    idx = np.array([[0, 1], [1, 2]], np.int32)
    val = np.array([[2.0, 4.0], [6.0, 8.0]])
    labels = np.array([0, 0], np.int32)
    prev = np.arange(K * pt, dtype=np.float64).reshape(K, pt)
    mu, counts, nk = oracle.kmeans_update(idx, val, labels, prev, pt)
    assert mu[0, 0] == 2.0 and mu[0, 1] == 5.0 and mu[0, 2] == 8.0
    assert np.array_equal(mu[0, 3:], prev[0, 3:])
    assert np.array_equal(mu[1:], prev[1:])  # empty clusters unchanged
    assert counts[0, 1] == 2 and nk.tolist() == [2, 0, 0]


def test_objective_non_increasing_tiny_config():
    n, p, m, K, seed = 2000, 64, 8, 5, 1
    X = synth.lowrank_spiky(n, p, seed=seed)
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, m, seed)
    rows = oracle.init_rows(n, K, seed)
    Y = oracle.precondition(X[rows], seed)
    labels, mu, hist = oracle.kmeans(idx, val, Y, pt, iters=10)
    # J' after each update is <= J' before it; the history records J' at each
    # assignment, which can only go down
    assert all(b <= a * (1 + 1e-12) for a, b in zip(hist, hist[1:]))


def test_2pass_brute_force_and_uses_1pass_labels():
    """Algorithm 2: means under the 1-pass labels, labels against the 1-pass centres."""
    rng = np.random.default_rng(8)
    n, p, K = 60, 12, 4
    X = rng.standard_normal((n, p)).astype(np.float32)
    c1 = rng.integers(0, K - 1, n).astype(np.int32)  # cluster K-1 empty in pass 1
    mu1 = rng.standard_normal((K, p))
    c2, mu2, counts = oracle.kmeans_2pass(X, c1, mu1)
    Xd = X.astype(np.float64)
    d = ((Xd[:, None, :] - mu1[None]) ** 2).sum(-1)
    assert np.array_equal(c2, np.argmin(d, axis=1))
    for k in range(K):
        sel = c1 == k
        assert counts[k] == sel.sum()
        if sel.any():
            assert np.allclose(mu2[k], Xd[sel].mean(0), rtol=1e-14, atol=1e-14)
        else:
            assert np.array_equal(mu2[k], mu1[k])
    # the means follow the 1-pass labels, not the new ones
    assert not np.array_equal(c1, c2)


def test_2pass_fixed_point_of_converged_lloyd():
    """With m = p the 1-pass method is Lloyd's; at its fixed point the extra
    pass changes neither labels nor centres."""
    n, p, K, seed = 400, 16, 3, 4
    X, _, _ = synth.mixture(n, p, K, seed=6, heavy_frac=0.0)
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, pt, seed)
    rows = oracle.init_rows(n, K, seed)
    Y = oracle.precondition(X, seed)
    labels, mu, _ = oracle.kmeans(idx, val, Y[rows], pt, iters=30)
    # one more assign with the final centres gives the labels the centres came from
    labels, _ = oracle.kmeans_assign(idx, val, mu, pt)
    mu_x = oracle.unmix(mu, p, seed)
    c2, mu2, _ = oracle.kmeans_2pass(X, labels, mu_x)
    assert np.array_equal(c2, labels)
    assert np.max(np.abs(mu2 - mu_x)) < 1e-10


def test_compress_raw_is_gather_of_padded_rows():
    X = synth.uniform(20, 50, seed=2)
    idx, val = oracle.compress_raw(X, 9, 3, row0=77)
    Xp = np.zeros((20, 64))
    Xp[:, :50] = X
    for i in range(20):
        assert np.array_equal(idx[i], oracle.mask(64, 9, 3, 77 + i))
        assert np.array_equal(val[i], Xp[i, idx[i]])


def test_hk_identity_at_full_sampling_and_brute_force():
    """H_k = (pt/m)(1/n_k) sum_{i in I_k} R_i R_i^T (Eq. (Hkmk)): m = pt samples
    every coordinate, so H_k = I exactly."""
    n, p, K, seed = 500, 32, 3, 2
    X = synth.uniform(n, p, seed=1)
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, pt, seed)
    labels = (np.arange(n) % K).astype(np.int32)
    _mu, counts, nk = oracle.kmeans_update(idx, val, labels, np.zeros((K, pt)), pt)
    assert np.array_equal(oracle.kmeans_hk(counts, nk, pt, pt), np.zeros(K))
    # brute force on a tiny assignment, and an empty cluster
    counts = np.array([[3, 1, 0, 2], [0, 0, 0, 0]], np.int64)
    nk = np.array([3, 0], np.int64)
    h = 4 / 2 * counts[0] / 3
    dev = oracle.kmeans_hk(counts, nk, 4, 2)
    assert abs(dev[0] - np.abs(h - 1).max()) < 1e-15 and dev[1] == -1.0


def test_hk_within_matrix_bernstein_bound():
    """Sec. VI-B: P(||H_k - I|| <= t) >= 1 - p exp(-(n_k t^2 / 2) /
    ((p/m - 1) + (p/m + 1) t / 3)); the deviation must respect the t that
    makes that failure probability 1e-6."""
    n, p, m, K, seed = 40000, 64, 8, 2, 3
    X = synth.uniform(n, p, seed=4)
    pt = oracle.ptilde(p)
    idx, val = oracle.compress(X, m, seed)
    labels = (np.arange(n) % K).astype(np.int32)
    _mu, counts, nk = oracle.kmeans_update(idx, val, labels, np.zeros((K, pt)), pt)
    dev = oracle.kmeans_hk(counts, nk, pt, m)
    r = pt / m
    for k in range(K):
        lo, hi = 0.0, 10.0
        for _ in range(100):  # bisection for the t with failure probability 1e-6
            t = 0.5 * (lo + hi)
            d3 = pt * np.exp(-(nk[k] * t * t / 2) / ((r - 1) + (r + 1) * t / 3))
            lo, hi = (t, hi) if d3 > 1e-6 else (lo, t)
        assert 0.0 < dev[k] <= hi
