"""GPU parity of K-means++ seeding on the sparsified rows (sk_kmeanspp) and
of the objective J' (sk_kmeans_objective), against the oracle on the same
ELL rows (the oracle's own compression, values rounded to float32, or a
seeded synthetic ELL at full size).

  chosen rows      bit-exact (integer decisions taken in the same float32 /
                   integer arithmetic on both sides)
  centres          bit-exact (scatters of the chosen rows)
  J'               1e-12 relative (float64 sums of float32 distances)
"""
import numpy as np
import pytest

import oracle
from paper_1511_00152_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    from paper_1511_00152_gb300 import _lib
    return _lib


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("n,p,m,K", [(2000, 64, 8, 5), (5001, 1024, 51, 10), (777, 256, 13, 20),
                                     (300, 4096, 205, 8), (257, 128, 2, 3)])
def test_kmeanspp_matches_oracle(sk, n, p, m, K):
    seed = 13
    X, _, _ = synth.mixture(n, p, min(K, 10), seed=n + p)
    oi, ov = oracle.compress(X, m, seed)
    v32 = ov.astype(np.float32)
    ctx = sk.sk_init(p, m, seed)
    idx, val = _dev(oi), _dev(v32)
    for r in (0, 1, 7):
        mu, rows = sk.sk_kmeanspp(ctx, idx, val, K, restart=r)
        torch.cuda.synchronize()
        ro, co = oracle.kmeanspp(oi, v32, ctx.pt, K, seed, r)
        assert np.array_equal(rows.cpu().numpy(), ro), (r, rows.cpu().numpy(), ro)
        assert np.array_equal(mu.cpu().numpy(), co)
    assert sk.sk_device_status() == sk.SK_OK


def test_kmeanspp_full_size_synthetic_ell(sk):
    """The K-means workload's shape (n = 1,000,000, pt = 1024, m = 51, K = 10)
    on a seeded synthetic ELL (random indices and values)."""
    n, p, m, K, seed = 1_000_000, 1024, 51, 10, 20240611
    rng = np.random.default_rng(3)
    oi = rng.integers(0, p, (n, m)).astype(np.int32)
    v32 = (rng.standard_normal((n, m)) * 3.0).astype(np.float32)
    ctx = sk.sk_init(p, m, seed)
    mu, rows = sk.sk_kmeanspp(ctx, _dev(oi), _dev(v32), K, restart=2)
    torch.cuda.synchronize()
    ro, co = oracle.kmeanspp(oi, v32, ctx.pt, K, seed, 2)
    assert np.array_equal(rows.cpu().numpy(), ro)
    assert np.array_equal(mu.cpu().numpy(), co)


def test_objective_and_best_of_restarts(sk):
    from paper_1511_00152_gb300 import pipeline
    n, p, m, K, seed = 4000, 256, 26, 6, 21
    X, _, _ = synth.mixture(n, p, K, seed=5, heavy_frac=0.0)
    ctx = sk.sk_init(p, m, seed)
    idx, val = sk.sk_compress(ctx, _dev(X))
    dist = torch.rand(n, device="cuda", dtype=torch.float32)
    J = sk.sk_kmeans_objective(dist)
    torch.cuda.synchronize()
    ref = dist.double().sum().item()
    assert abs(J.item() - ref) <= 1e-12 * ref
    labels, mu, Jb, rb = pipeline.kmeans_best_of(ctx, idx, val, K, restarts=4, iters=8)
    # the best run's J' is the smallest of the four runs', re-run one by one
    st = pipeline.KMeansState(ctx, n, K, keep_dist=True)
    work = torch.empty(max(256, sk.sk_kmeanspp_workspace_bytes(ctx, n)), dtype=torch.uint8,
                       device="cuda")
    Js = []
    for r in range(4):
        mu0, _ = sk.sk_kmeanspp(ctx, idx, val, K, restart=r, work=work)
        st.run(idx, val, mu0, 8, use_graph=False)
        Js.append(sk.sk_kmeans_objective(st.dist).item())
    assert 0 <= rb < 4
    assert abs(Jb - min(Js)) <= 1e-6 * min(Js)
    assert int(np.argmin(Js)) == rb or abs(Js[rb] - min(Js)) <= 1e-6 * min(Js)
    nk = torch.bincount(labels.long(), minlength=K)
    assert nk.sum().item() == n
    assert sk.sk_device_status() == sk.SK_OK
