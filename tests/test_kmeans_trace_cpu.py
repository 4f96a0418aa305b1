"""The K-means run comparison used by the GPU parity tests (kmeans_trace),
checked on the CPU with runs made from the oracle itself: the oracle's own run
passes with every cluster compared, and a planted label error outside the
near-tie band, a planted error in a compared centre or count, each fail."""
import numpy as np
import pytest

import kmeans_trace
import oracle
from paper_1511_00152_gb300 import synth


def _setup(iters=6):
    n, p, m, K, seed = 600, 64, 8, 4, 3
    X = synth.mixture(n, p, K, seed=5)[0]
    oi, ov = oracle.compress(X, m, seed)
    mu0 = oracle.precondition(X[synth.init_rows(n, K, seed)], seed)
    tr = kmeans_trace.oracle_trace(oi, ov, mu0, oracle.ptilde(p), iters)
    return tr, K


def test_oracle_run_against_itself_compares_every_cluster():
    tr, K = _setup()
    keep, nflip = kmeans_trace.check_against_trace(tr["labels"], tr["mu"], tr["counts"], tr["nk"],
                                                   tr, K)
    assert nflip == 0 and keep.all()


def test_label_error_outside_the_band_fails():
    tr, K = _setup()
    labs = [lab.copy() for lab in tr["labels"]]
    D = kmeans_trace.restricted_distances(tr["idx"], tr["val"], tr["mus"][2])
    gaps = np.sort(D, axis=1)
    r = int(np.argmax(gaps[:, 1] - gaps[:, 0]))  # the clearest row of iteration 2
    labs[2][r] = (labs[2][r] + 1) % K
    with pytest.raises(AssertionError):
        kmeans_trace.untouched(labs, tr, K)


def test_near_tie_flip_narrows_the_comparison():
    tr, K = _setup()
    labs = [lab.copy() for lab in tr["labels"]]
    # make row 0 of the last iteration a near-tie by construction: move its
    # oracle distance to the second centre within the band, then flip it
    D = kmeans_trace.restricted_distances(tr["idx"], tr["val"], tr["mus"][-1])
    o = labs[-1][0]
    g = (o + 1) % K
    D[0, g] = D[0, o] * (1 + 1e-5)
    tr["dists"] = [None] * (len(labs) - 1) + [D]
    labs[-1][0] = g
    keep, nflip = kmeans_trace.untouched(labs, tr, K)
    assert nflip == 1 and not keep[o] and not keep[g] and keep.sum() == K - 2


def test_centre_or_count_error_in_a_compared_cluster_fails():
    tr, K = _setup()
    mu = tr["mu"].copy()
    mu[1, 5] += 1e-3 * np.abs(mu).max()
    with pytest.raises(AssertionError):
        kmeans_trace.check_against_trace(tr["labels"], mu, tr["counts"], tr["nk"], tr, K)
    cnt = tr["counts"].copy()
    cnt[2, 7] += 1
    with pytest.raises(AssertionError):
        kmeans_trace.check_against_trace(tr["labels"], tr["mu"], cnt, tr["nk"], tr, K)
