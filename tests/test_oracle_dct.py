"""Pins for the oracle's DCT preconditioner (Sec. III: H a DCT matrix, the
preconditioner of the paper's big-data runs of Sec. VII).

The oracle writes the orthonormal DCT-II out as its defining sum; these tests
fix it against what does not depend on that code: scipy.fft's DCT routines,
orthonormality, closed forms, the coherence sqrt(2/p) of the DCT (Sec. III's
eta = 1/2) and the tail bound that comes with it, and the inverse property
of the un-mixing map."""
import numpy as np
import pytest

import oracle

scipy_fft = pytest.importorskip("scipy.fft")


@pytest.mark.parametrize("p", [2, 6, 28, 50, 98, 784, 1000])
def test_dct_matches_scipy_orthonormal_dct(p):
    x = np.random.default_rng(p).standard_normal(p)
    assert np.max(np.abs(oracle.dct(x) - scipy_fft.dct(x, type=2, norm="ortho"))) < 1e-12
    assert np.max(np.abs(oracle.idct(x) - scipy_fft.dct(x, type=3, norm="ortho"))) < 1e-12


@pytest.mark.parametrize("p", [10, 24, 56])
def test_dct_matrix_is_orthonormal_and_idct_is_its_transpose(p):
    C = np.stack([oracle.dct(e) for e in np.eye(p)], axis=1)  # column l = H e_l
    assert np.max(np.abs(C.T @ C - np.eye(p))) < 1e-13
    Ct = np.stack([oracle.idct(e) for e in np.eye(p)], axis=1)
    assert np.max(np.abs(Ct - C.T)) < 1e-13
    x = np.random.default_rng(1).standard_normal(p)
    assert np.max(np.abs(oracle.idct(oracle.dct(x)) - x)) < 1e-13


def test_dct_closed_forms():
    p = 40
    # a constant vector has all its energy in coefficient 0
    y = oracle.dct(np.ones(p))
    assert abs(y[0] - np.sqrt(p)) < 1e-12 and np.max(np.abs(y[1:])) < 1e-12
    # the cosine of frequency k0 is sqrt(p/2) e_k0
    n = np.arange(p)
    for k0 in (1, 7, 39):
        y = oracle.dct(np.cos(np.pi * (2 * n + 1) * k0 / (2 * p)))
        e = np.zeros(p)
        e[k0] = np.sqrt(p / 2)
        assert np.max(np.abs(y - e)) < 1e-11


@pytest.mark.parametrize("p", [30, 784])
def test_dct_coherence_and_tail_bound(p):
    """Entries of the DCT are at most sqrt(2/p) in magnitude, which is what
    gives eta = 1/2 in Sec. III: for a fixed x and random signs D,
    P(|(H D x)_j| >= t ||x|| / sqrt(p)) <= 2 exp(-t^2 / 4) (Hoeffding)."""
    C = np.stack([oracle.dct(e) for e in np.eye(p)], axis=1) if p <= 64 else None
    if C is not None:
        assert abs(np.abs(C).max() - np.sqrt(2.0 / p)) < 1e-12
    rng = np.random.default_rng(5)
    x = np.zeros(p)
    x[: 3] = [5.0, -3.0, 1.0]  # a spiky sample
    xs = x / np.linalg.norm(x)
    hits = {2.0: 0, 3.0: 0}
    trials = 300
    for _ in range(trials):
        D = rng.choice([-1.0, 1.0], size=p)
        y = oracle.dct(D * xs) * np.sqrt(p)
        for t in hits:
            hits[t] += int(np.sum(np.abs(y) >= t))
    for t, h in hits.items():
        assert h / (trials * p) <= 2 * np.exp(-t * t / 4)


def test_dct_compress_precondition_unmix_consistent():
    """With the DCT flag: masks are m distinct indices of [0, p) by the
    written spec (the same stream as the Hadamard form, range p), val is the
    preconditioned row at them, and un-mixing inverts the preconditioner."""
    from paper_1511_00152_gb300 import synth
    n, p, m, seed = 40, 784, 39, 21
    X = synth.lowrank_spiky(n, p, seed=3)
    Y = oracle.precondition(X, seed, dct=True)
    assert Y.shape == (n, p)
    D = oracle.signs(p, seed)
    assert np.max(np.abs(Y[0] - oracle.dct(D * X[0].astype(np.float64)))) < 1e-12
    idx, val = oracle.compress(X, m, seed, row0=5, dct=True)
    for i in range(n):
        assert np.array_equal(idx[i], oracle.mask(p, m, seed, 5 + i))
        assert len(set(idx[i].tolist())) == m and idx[i].min() >= 0 and idx[i].max() < p
    assert np.max(np.abs(val - np.take_along_axis(Y, idx, axis=1))) < 1e-15
    back = oracle.unmix(Y, p, seed, dct=True)
    assert np.max(np.abs(back - X.astype(np.float64))) < 1e-10
    # the back-map of the second moment (Sec. V): (HD)^T C_emp(Y) (HD) = C_emp(X)
    CY = Y.T @ Y / n
    W = oracle.unmix(oracle.unmix(CY, p, seed, dct=True).T.copy(), p, seed, dct=True)
    CX = X.astype(np.float64).T @ X.astype(np.float64) / n
    assert np.max(np.abs(W - CX)) < 1e-9 * np.abs(CX).max()
