"""Pins for the oracle's preconditioner y = H D x (Sec. III, Eq. (ROS)) and
the un-mixing map mu = (HD)^T mu' (Eq. (mu-mu'))."""
import numpy as np
import pytest

import oracle
from paper_1511_00152_gb300 import synth


def sylvester(pt):
    """Orthonormal Sylvester-Hadamard matrix by repeated Kronecker products."""
    H = np.array([[1.0]])
    h2 = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)
    while H.shape[0] < pt:
        H = np.kron(h2, H)
    return H


@pytest.mark.parametrize("pt", [1, 2, 4, 8, 16, 32, 64])
def test_fwht_equals_explicit_matrix(pt):
    H = sylvester(pt)
    # entries are +-1/sqrt(p) (Sec. III)
    assert np.allclose(np.abs(H), 1.0 / np.sqrt(pt), atol=0, rtol=1e-15)
    for j in range(pt):
        e = np.zeros(pt)
        e[j] = 1.0
        assert np.max(np.abs(oracle.fwht(e) - H[:, j])) < 1e-14
    x = np.random.default_rng(pt).standard_normal(pt)
    assert np.max(np.abs(oracle.fwht(x) - H @ x)) < 1e-13


@pytest.mark.parametrize("pt", [128, 1024, 8192])
def test_fwht_orthonormal_and_involution(pt):
    x = np.random.default_rng(1).standard_normal(pt)
    y = oracle.fwht(x)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)
    assert np.max(np.abs(oracle.fwht(y) - x)) < 1e-12


def test_precondition_matches_H_D_with_padding():
    p, seed = 50, 4242
    pt = oracle.ptilde(p)
    assert pt == 64
    X = synth.uniform(7, p, seed=3)
    Y = oracle.precondition(X, seed)
    H = sylvester(pt)
    D = oracle.signs(pt, seed)
    Xp = np.zeros((7, pt))
    Xp[:, :p] = X.astype(np.float64)
    ref = (H @ (D[:, None] * Xp.T)).T
    assert np.max(np.abs(Y - ref)) < 1e-13
    # orthonormality of HD: norms preserved to 1e-12
    assert np.allclose(np.linalg.norm(Y, axis=1), np.linalg.norm(Xp, axis=1), rtol=1e-12, atol=0)


def test_compress_gathers_preconditioned_values():
    X = synth.lowrank_spiky(40, 100, seed=5)
    seed, m = 9, 12
    idx, val = oracle.compress(X, m, seed, row0=1000)
    Y = oracle.precondition(X, seed)
    for i in range(X.shape[0]):
        assert np.array_equal(idx[i], oracle.mask(128, m, seed, 1000 + i))
        assert np.array_equal(val[i], Y[i, idx[i]])


def test_unmix_inverts_precondition():
    p, seed = 37, 77
    X = synth.uniform(5, p, seed=8)
    Y = oracle.precondition(X, seed)
    Xr = oracle.unmix(Y, p, seed)
    assert np.max(np.abs(Xr - X.astype(np.float64))) < 1e-13


def test_covariance_backmap():
    """C_n estimates HD C_x (HD)^T; (HD)^T C_emp(Y) (HD) = C_emp(X) (Sec. V)."""
    p, seed = 64, 11
    X = synth.lowrank_spiky(300, p, seed=12).astype(np.float64)
    Y = oracle.precondition(X.astype(np.float32), seed)
    CY = Y.T @ Y / X.shape[0]
    CX = X.T @ X / X.shape[0]
    # (HD)^T A (HD) = D H A H D; un-mix the rows then the columns
    back = oracle.unmix(oracle.unmix(CY, p, seed).T.copy(), p, seed)
    assert np.max(np.abs(back - CX)) <= 1e-12 * np.max(np.abs(CX))
