"""Full-size parity: the benchmark's workloads at their full sizes, in the
launch configuration bench.py times, checked on outputs the oracle can compute
one by one (sampled rows) and on properties that hold at any size.

K-means workload: n = 1,000,000, p = 1024, m = 51, K = 10.
PCA workload:     n = 1,048,576, p = 4096, m = 205, top-20.

The oracle only ever receives inputs drawn by the seeded generator (rows copied
back from the device generator) -- never a value computed by the CUDA path.
Tolerances are those of tests/test_gpu_parity.py; the split-BF16 Gram is
compared with the independent FP32 scatter Gram (rel. Frobenius <= 1e-5).
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


def _sample_rows(n, count, seed):
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([rng.choice(n, count - 2, replace=False), [0, n - 1]]))
    return rows


def _check_sampled_compress(sk, ctx, X, idx, val, m, seed, rows):
    Xs = X[torch.as_tensor(rows, device=X.device)].cpu().numpy()
    gi = idx[torch.as_tensor(rows, device=X.device)].cpu().numpy()
    gv = val[torch.as_tensor(rows, device=X.device)].cpu().numpy().astype(np.float64)
    for r, row in enumerate(rows):
        oi, ov = oracle.compress(Xs[r:r + 1], m, seed, row0=int(row))
        assert np.array_equal(gi[r], oi[0]), f"row {row}"
        nrm = np.linalg.norm(Xs[r].astype(np.float64))
        assert np.abs(gv[r] - ov[0]).max() <= 1e-5 * nrm, f"row {row}"
    return Xs


def test_kmeans_workload_full_size(sk):
    from paper_1511_00152_gb300 import pipeline
    n, p, m, K, seed = 1_000_000, 1024, 51, 10, 20240611
    ctx = sk.sk_init(p, m, seed)
    X, _, _ = synth.mixture_device(n, p, 10, seed)
    idx, val = sk.sk_compress(ctx, X)
    rows = _sample_rows(n, 256, 1)
    Xs = _check_sampled_compress(sk, ctx, X, idx, val, m, seed, rows)

    # first K-means pass from the seeded start: sampled labels vs the oracle
    init = synth.init_rows(n, K, seed)
    Xi = X[torch.as_tensor(init, device=X.device)].contiguous()
    mu0 = sk.sk_precondition(ctx, Xi)
    st = pipeline.KMeansState(ctx, n, K)
    st.mu.copy_(mu0)
    st.iteration(idx, val, first=True)
    torch.cuda.synchronize()
    mu_o = oracle.precondition(Xi.cpu().numpy(), seed)
    oi, ov = oracle.compress(Xs[:1], m, seed, row0=int(rows[0]))
    lab_g = st.labels[torch.as_tensor(rows, device=X.device)].cpu().numpy()
    for r, row in enumerate(rows):
        oi, ov = oracle.compress(Xs[r:r + 1], m, seed, row0=int(row))
        lo, _ = oracle.kmeans_assign(oi, ov, mu_o, ctx.pt)
        d = [float(np.sum((ov[0] - mu_o[k][oi[0]]) ** 2)) for k in range(K)]
        ds = sorted(d)
        if ds[1] - ds[0] > 1e-4 * ds[0]:
            assert lab_g[r] == lo[0], f"row {row}"
    # size-independent invariants of the sums (Eq. (mu_update_one))
    nk = st.nk.cpu().numpy()
    cnt = st.cnt.cpu().numpy()
    assert nk.sum() == n
    assert np.array_equal(cnt.sum(axis=1), m * nk)
    # the whole benchmark loop (20 iterations, graph) keeps the invariants
    st2 = pipeline.KMeansState(ctx, n, K)
    st2.run(idx, val, mu0, 20, use_graph=True)
    torch.cuda.synchronize()
    assert st2.nk.sum().item() == n
    assert np.array_equal(st2.cnt.cpu().numpy().sum(axis=1), m * st2.nk.cpu().numpy())
    assert sk.sk_device_status() == sk.SK_OK


def test_pca_workload_full_size(sk):
    n, p, m, k, seed = 1_048_576, 4096, 205, 20, 7
    ctx = sk.sk_init(p, m, seed)
    X = synth.lowrank_decay_device(n, p, seed)
    idx, val = sk.sk_compress(ctx, X)
    rows = _sample_rows(n, 64, 2)
    _check_sampled_compress(sk, ctx, X, idx, val, m, seed, rows)
    del X
    torch.cuda.empty_cache()
    pt = ctx.pt
    G3 = torch.zeros((pt, pt), dtype=torch.float64, device="cuda")
    G1 = torch.zeros_like(G3)
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G3)
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx, val, G1)
    torch.cuda.synchronize()
    U3, U1 = torch.triu(G3), torch.triu(G1)
    rel = (torch.linalg.norm(U3 - U1) / torch.linalg.norm(U1)).item()
    assert rel <= 1e-5, rel
    # trace(G) = sum of squared sampled values (holds at any size)
    tr = torch.diagonal(G1).sum().item()
    ssq = (val.double() ** 2).sum().item()
    # float shared-memory tile sums over long row ranges, then FP64: a small bias
    assert abs(tr - ssq) <= 1e-5 * ssq
    C = sk.sk_cov_finalize(ctx, G3, n)
    ev, U = sk.sk_cov_topk(ctx, C, k, iters=60)
    torch.cuda.synchronize()
    # eigenpair residuals and orthonormality of the returned subspace
    Cu = C @ U.T
    res = torch.linalg.norm(Cu - U.T * ev[None, :], dim=0) / ev.abs()
    assert res.max().item() <= 1e-6, res.max().item()
    I = U @ U.T
    assert torch.allclose(I, torch.eye(k, dtype=torch.float64, device="cuda"), atol=1e-10)
    assert torch.all(ev[:-1] >= ev[1:])
    assert sk.sk_device_status() == sk.SK_OK
