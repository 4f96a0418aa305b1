"""Pins from the paper's theorems on the oracle's preconditioner and estimators.

* Sec. IV, proof of the sample-mean theorem: the per-sample error covariance
  Lambda = E[(p/m R R^T x - x)(p/m R R^T x - x)^T] has the closed form
  -(p-m)/(m(p-1)) x x^T + p(p-m)/(m(p-1)) diag(x x^T); checked exactly by
  enumerating every mask at p = 8.
* Sec. IV, the sample-mean theorem: ||mean-hat - mean||_inf <= t(delta_1),
  t from the Bernstein bound solved for t (the remark after the theorem);
  checked over seeded runs.
* Sec. III: with random signs D, E[(H D x)_j^2] = ||x||^2 / p; H D maps a
  single spike to a flat vector of entries +-1/sqrt(p).
* Appendix D, the pairwise-distance theorem: ||sqrt(p/m) R^T H D (x1 - x2)||
  lies in [0.40, 1.48] ||x1 - x2|| with high probability.
* Sec. V, the covariance theorem: ||C_n - C_emp||_2 <= t(delta_2) from its
  matrix Bernstein bound, on the model of the paper's own experiment.
"""
import itertools

import numpy as np
import pytest

import oracle


def _all_masks(pt, m):
    return list(itertools.combinations(range(pt), m))


@pytest.mark.parametrize("m", [1, 2, 5, 7, 8])
def test_sample_mean_error_covariance_by_enumeration(m):
    pt = 8
    x = np.random.default_rng(17).standard_normal(pt)
    acc = np.zeros((pt, pt))
    masks = _all_masks(pt, m)
    for om in masks:
        idx = np.array([om], np.int32)
        e = oracle.sample_mean(idx, x[idx], pt) - x
        acc += np.outer(e, e)
    acc /= len(masks)
    lam = (-(pt - m) / (m * (pt - 1)) * np.outer(x, x)
           + pt * (pt - m) / (m * (pt - 1)) * np.diag(x * x))
    assert np.max(np.abs(acc - lam)) <= 1e-13 * max(1.0, np.max(np.abs(lam)))


def test_sample_mean_linf_error_within_bernstein_bound():
    """Fixed data set x_i = xbar + noise (the setting of the paper's
    sample-mean experiment), masks drawn anew per run: the l_inf error of
    (p/m)(1/n) sum R_i R_i^T x_i stays below t(delta_1 = 1e-5) in every run,
    and is of the order the bound predicts (not far below it)."""
    p, m, n, runs = 128, 38, 1000, 200
    rng = np.random.default_rng(5)
    xbar = rng.standard_normal(p)
    X = (xbar + rng.standard_normal((n, p))).astype(np.float32)
    X64 = X.astype(np.float64)
    mean = X64.mean(axis=0)
    delta = 1e-5
    tau = max(p / m - 1.0, 1.0)
    xmax = np.abs(X64).max()
    maxrow2 = (X64 ** 2).sum(axis=0).max()  # ||X||_maxRow^2 with samples as columns
    L = np.log(2 * p / delta)
    a = tau / 3.0 * xmax * L
    t = (a + np.sqrt(a * a + 2.0 * (p / m - 1.0) * L * maxrow2)) / n
    errs = []
    for seed in range(runs):
        idx, val = oracle.compress_raw(X, m, seed + 1)
        errs.append(np.max(np.abs(oracle.sample_mean(idx, val, p) - mean)))
    errs = np.array(errs)
    assert errs.max() <= t
    assert errs.mean() >= 0.05 * t


def test_preconditioned_entry_second_moment():
    """E_D[(H D x)_j^2] = ||x||^2 / p for every coordinate j: the mean of
    y_j^2 over 4000 seeds (a sign pattern each) within 10%."""
    p, seeds = 64, 4000
    x = np.random.default_rng(3).standard_normal(p)
    acc = np.zeros(p)
    for seed in range(seeds):
        acc += oracle.precondition(x[None].astype(np.float32), seed)[0] ** 2
    target = float(np.sum(x.astype(np.float32).astype(np.float64) ** 2)) / p
    assert np.max(np.abs(acc / seeds - target)) <= 0.10 * target


@pytest.mark.parametrize("j", [0, 5, 777])
def test_preconditioning_spreads_a_spike_evenly(j):
    """H D e_j has every entry +-1/sqrt(p): any m sampled entries carry
    exactly m/p of the energy, so the rescaled sampled norm equals the norm
    whatever the mask; without preconditioning it is all or nothing."""
    p, m = 1024, 51
    x = np.zeros(p, np.float32)
    x[j] = 3.0
    for seed in range(20):
        _, val = oracle.compress(x[None], m, seed, row0=seed)
        ratio = np.sqrt(p / m) * np.linalg.norm(val) / 3.0
        assert abs(ratio - 1.0) < 1e-12
        _, raw = oracle.compress_raw(x[None], m, seed, row0=seed)
        r_raw = np.sqrt(p / m) * np.linalg.norm(raw) / 3.0
        assert min(abs(r_raw), abs(r_raw - np.sqrt(p / m))) < 1e-12


def test_pairwise_distance_ratio_in_band():
    """||sqrt(p/m) R^T H D d|| / ||d|| in [0.40, 1.48] for 300 seeded
    differences d (Gaussian, 5-sparse, one large spike on small noise) at
    p = 1024, m = 205; the unpreconditioned ablation leaves the band for the
    spiky ones."""
    p, m = 1024, 205
    rng = np.random.default_rng(9)
    diffs = []
    for _ in range(100):
        diffs.append(rng.standard_normal(p))
        s = np.zeros(p)
        s[rng.choice(p, 5, replace=False)] = rng.standard_normal(5) * 10
        diffs.append(s)
        k = np.full(p, 0.001) * rng.standard_normal(p)
        k[rng.integers(p)] = 50.0
        diffs.append(k)
    out_raw = 0
    for r, d in enumerate(diffs):
        d32 = d.astype(np.float32)
        nd = np.linalg.norm(d32.astype(np.float64))
        _, val = oracle.compress(d32[None], m, 77, row0=r)
        ratio = np.sqrt(p / m) * np.linalg.norm(val) / nd
        assert 0.40 <= ratio <= 1.48, (r, ratio)
        _, raw = oracle.compress_raw(d32[None], m, 77, row0=r)
        rr = np.sqrt(p / m) * np.linalg.norm(raw) / nd
        out_raw += not (0.40 <= rr <= 1.48)
    assert out_raw >= 90  # nearly every one-spike difference, without preconditioning


def _cov_bound(X64, m, rho, delta):
    """t with P{||C_n - C_emp||_2 <= t} >= 1 - delta from the covariance
    theorem of Sec. V (L and the bound on sigma^2 as stated there, the matrix
    Bernstein tail solved for t); X64 holds the samples as rows."""
    n, p = X64.shape
    Cemp = X64.T @ X64 / n
    maxcol2 = (X64 ** 2).sum(axis=1).max()  # ||X||_maxCol^2: largest sample norm
    xmax2 = np.abs(X64).max() ** 2
    fro2 = (X64 ** 2).sum()
    x4 = (X64 ** 4).sum(axis=0).max()
    a = p * (p - 1) / (m * (m - 1))
    L = ((a * rho + 1) * maxcol2 + p * (p - m) / (m * (m - 1)) * xmax2) / n
    s2 = ((a * rho - 1) * maxcol2 * np.linalg.norm(Cemp, 2)
          + p * (p - 1) * (p - m) / (m * (m - 1) ** 2) * rho * maxcol2 * np.max(np.diag(Cemp))
          + 2 * p * (p - 1) * (p - m) / (m * (m - 1) ** 2) * xmax2 * fro2 / n
          + p * (p - m) ** 2 / (m * (m - 1) ** 2) * x4 / n) / n
    lg = np.log(p / delta)
    return lg * L / 3 + np.sqrt((lg * L / 3) ** 2 + 2 * lg * s2), Cemp


def test_covariance_error_within_theorem_bound():
    """Sec. V covariance theorem on its own experiment's model (rank-5 data
    x_i = sum_j kappa_ij lambda_j u_j, lambda = (10, 8, 6, 4, 2)) at p = 256,
    gamma = 0.3: over seeded masks ||C_n - C_emp||_2 stays below the bound
    t(delta_2 = 0.01, rho = 1) and, as the paper reports, within an order of
    magnitude of it; the error falls like 1/sqrt(n) (4n samples: about half)."""
    p, k, m = 256, 5, 77
    lam = np.array([10.0, 8.0, 6.0, 4.0, 2.0])
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((p, k)))
    errs = {}
    for n in (2560, 10240):
        X = ((rng.standard_normal((n, k)) * lam) @ U.T).astype(np.float32)
        X64 = X.astype(np.float64)
        t, Cemp = _cov_bound(X64, m, 1.0, 0.01)
        e = []
        for seed in range(10):
            idx, val = oracle.compress_raw(X, m, seed + 1)
            e.append(np.linalg.norm(oracle.cov(idx, val, p) - Cemp, 2))
        e = np.array(e)
        assert e.max() <= t, (n, e.max(), t)
        assert t / 100 <= e.mean() <= t / 3, (n, e.mean(), t)
        errs[n] = e.mean()
    assert 0.35 <= errs[10240] / errs[2560] <= 0.7
