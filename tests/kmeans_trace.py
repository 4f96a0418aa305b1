"""Comparison of a K-means run with the oracle's, for runs whose assignments
may legitimately differ in near-ties (test helper, no test of its own).

A row whose oracle distances to its oracle label o and to another centre g
are within a relative 1e-4 of each other may go to g on the GPU (float32
sums in another order); from then on the two runs can diverge, but only
through the clusters such a row moved between.  `untouched` follows that
argument iteration by iteration: a row whose GPU label g differs from the
oracle's o must either involve a cluster touched earlier (g or o), or be a
near-tie between g and o under the oracle's distances; both clusters then
count as touched.  A cluster never touched has the same members in both runs
at every iteration, so its sums and centres must agree to rounding.  Every
check is an assertion: nothing is skipped, a comparison only narrows to the
untouched clusters.
"""
import numpy as np

import oracle


def restricted_distances(idx, val, mu, rows=None):
    """Restricted squared distances sum_t (val - mu_k[idx])^2 (float64) of the
    given rows (all if None) to every centre: len(rows) x K.  Used only to
    decide which rows are near-ties."""
    if rows is not None:
        idx, val = idx[rows], val[rows]
    n = idx.shape[0]
    K = mu.shape[0]
    d = np.zeros((n, K))
    for k in range(K):
        diff = val - mu[k][idx]
        d[:, k] = (diff * diff).sum(1)
    return d


def oracle_trace(idx, val, mu0, pt, iters):
    """The oracle's run: per iteration the labels and the centres they were
    chosen against; then the final centres, counts and nk."""
    mu = np.array(mu0, np.float64, copy=True)
    labels, mus = [], []
    counts = nk = None
    for _ in range(iters):
        lab, _d = oracle.kmeans_assign(idx, val, mu, pt)
        mus.append(mu)
        labels.append(lab)
        mu, counts, nk = oracle.kmeans_update(idx, val, lab, mu, pt)
    return dict(labels=labels, mus=mus, mu=mu, counts=counts, nk=nk, idx=idx, val=val)


def untouched(gpu_labels, trace, K, rel=1e-4):
    """Boolean mask of the clusters no differing assignment ever touched, and
    the number of (row, iteration) assignments that differed."""
    T = np.zeros(K, bool)
    nflip = 0
    for it, (g, o, mu) in enumerate(zip(gpu_labels, trace["labels"], trace["mus"])):
        g = np.asarray(g)
        f = np.nonzero(g != o)[0]
        nflip += len(f)
        if len(f) == 0:
            continue
        gf, of = g[f], o[f]
        assert np.all((gf >= 0) & (gf < K)), "label out of range"
        involved = T[gf] | T[of]
        D = trace["dists"][it][f] if "dists" in trace else \
            restricted_distances(trace["idx"], trace["val"], mu, f)
        j = np.arange(len(f))
        dg, do = D[j, gf], D[j, of]
        tie = (dg - do) <= rel * np.maximum(do, 1e-30)
        bad = ~(involved | tie)
        assert not np.any(bad), (
            f"iteration {it}: rows {f[bad][:5]} differ from the oracle outside the near-tie band")
        T[gf] = True
        T[of] = True
    return ~T, nflip


def check_against_trace(gpu_labels, mu, cnt, nk, trace, K, max_touched_frac=0.5, mu_rel=1e-5):
    """Final centres, counts and nk of a GPU run against the oracle's run,
    over the untouched clusters (at least 1 - max_touched_frac of them)."""
    keep, nflip = untouched(gpu_labels, trace, K)
    assert keep.sum() >= max(1, int(np.ceil((1.0 - max_touched_frac) * K))), (keep.sum(), K, nflip)
    muo = trace["mu"]
    scale = np.abs(muo).max() + 1e-30
    assert np.abs(np.asarray(mu, np.float64)[keep] - muo[keep]).max() <= mu_rel * scale
    if cnt is not None:
        assert np.array_equal(np.asarray(cnt)[keep], trace["counts"][keep])
    if nk is not None:
        assert np.array_equal(np.asarray(nk)[keep], trace["nk"][keep])
    return keep, nflip
