"""GPU parity for the paper's further rows: the no-preconditioning ablation
(Sec. VII), the second pass of the 2-pass sparsified K-means (Algorithm 2)
and the sample-mean estimator (Sec. IV), each against the FP64 oracle on the
same seeded inputs.

Tolerances (stated per result):
  ablation idx / val / Y / unmix   bit-exact (a gather of float32 values, no arithmetic)
  2-pass labels   identical where the oracle's best and second-best dense
                  distances differ by more than 1e-4 relative (near-tie band;
                  the kernel forms the distance in float32)
  2-pass counts   exact
  2-pass centres  |mu_gpu - mu_oracle| <= 1e-5 * max(1, max|x|)
                  (float32 sums over <= 1024 rows per CTA, then float64)
  sample mean     |mean_gpu - mean_oracle| <= 1e-5 * max|mean_oracle| + 1e-6 * rms(val)
                  (float32 ELL values vs the oracle's float64 transform,
                  float32 shared-memory partial sums)
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


def _padded(X, pad):
    n, p = X.shape
    Xw = np.zeros((n, p + pad), np.float32)
    Xw[:, :p] = X
    return _dev(Xw)[:, :p]


# ------------------------------------------------------------- ablation

@pytest.mark.parametrize("p,m,n,row0,pad", [
    (1000, 51, 3001, 0, 0),     # K-means workload dimension, ragged tail
    (50, 9, 777, 5, 0),         # p % 4 != 0: scalar loads
    (1024, 102, 1000, 2**33, 4),  # 64-bit row keys, padded ldx
    (4096, 205, 64, 0, 0),      # pt > 1024: multi-warp rows
    (3, 2, 100, 0, 0),          # pt = 4
    (1, 1, 17, 0, 0),           # pt = 1
])
def test_no_preconditioning_compress_is_gather(sk, p, m, n, row0, pad):
    seed = 99
    X = synth.uniform(n, p, seed=p + n)
    ctx = sk.sk_init_ex(p, m, seed, sk.SK_FLAG_NO_PRECONDITION)
    assert ctx.flags == sk.SK_FLAG_NO_PRECONDITION
    Xd = _padded(X, pad) if pad else _dev(X)
    idx, val = sk.sk_compress(ctx, Xd, row0=row0)
    torch.cuda.synchronize()
    oi, ov = oracle.compress_raw(X, m, seed, row0=row0)
    assert np.array_equal(idx.cpu().numpy(), oi)
    assert np.array_equal(val.cpu().numpy().astype(np.float64), ov)
    # the mask stream does not depend on the flag
    ctx2 = sk.sk_init(p, m, seed)
    idx2, _ = sk.sk_compress(ctx2, Xd, row0=row0)
    torch.cuda.synchronize()
    assert torch.equal(idx, idx2)


def test_no_preconditioning_precondition_and_unmix_are_pad_and_truncate(sk):
    p, m, n, seed = 1000, 51, 300, 3
    X = synth.uniform(n, p, seed=1)
    ctx = sk.sk_init_ex(p, m, seed, sk.SK_FLAG_NO_PRECONDITION)
    Y = sk.sk_precondition(ctx, _dev(X))
    torch.cuda.synchronize()
    Yh = Y.cpu().numpy()
    assert np.array_equal(Yh[:, :p], X) and not Yh[:, p:].any()
    back = sk.sk_unmix(ctx, Y)
    back64 = sk.sk_unmix(ctx, Y.double())
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), X)
    assert np.array_equal(back64.cpu().numpy(), X.astype(np.float64))


def test_init_ex_rejects_unknown_flags(sk):
    with pytest.raises(sk.SkError) as e:
        sk.sk_init_ex(100, 5, 1, 4)
    assert e.value.status == sk.SK_EINVAL


# ------------------------------------------------------------- 2-pass

def _check_2pass(sk, X, labels1, mu1, pad=0, chunks=1):
    n, p = X.shape
    K = mu1.shape[0]
    ctx = sk.sk_init(p, max(1, min(8, p)), 5)
    Xd = _padded(X, pad) if pad else _dev(X)
    mud = _dev(mu1.astype(np.float32))
    l1 = _dev(labels1.astype(np.int32))
    labels, dist = sk.sk_kmeans2_assign(ctx, Xd, mud,
                                       dist=torch.empty(n, dtype=torch.float32, device="cuda"))
    sums = torch.zeros((K, p), dtype=torch.float64, device="cuda")
    counts = torch.zeros(K, dtype=torch.int64, device="cuda")
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        sk.sk_kmeans2_sums(ctx, Xd[a:b], l1[a:b], K, sums, counts)
    mu2 = sk.sk_kmeans2_finalize(ctx, sums, counts, mud.clone())
    torch.cuda.synchronize()
    c2o, mu2o, cnto = oracle.kmeans_2pass(X, labels1, mu1.astype(np.float32).astype(np.float64))
    # labels outside the near-tie band
    Xd64 = X.astype(np.float64)
    m64 = mu1.astype(np.float32).astype(np.float64)
    d = ((Xd64 * Xd64).sum(1)[:, None] - 2 * Xd64 @ m64.T + (m64 * m64).sum(1)[None, :])
    ds = np.sort(d, axis=1)
    clear = (ds[:, 1] - ds[:, 0]) > 1e-4 * np.maximum(ds[:, 0], 1e-30) if K > 1 else np.ones(n, bool)
    lg = labels.cpu().numpy()
    assert np.array_equal(lg[clear], c2o[clear])
    assert clear.mean() > 0.9
    dg = dist.cpu().numpy().astype(np.float64)
    best = d[np.arange(n), lg]
    assert np.all(np.abs(dg - best) <= 1e-5 * np.maximum(best, 1.0) + 1e-4)
    assert np.array_equal(counts.cpu().numpy(), cnto)
    scale = max(1.0, float(np.abs(X).max()))
    assert np.abs(mu2.cpu().numpy().astype(np.float64) - mu2o).max() <= 1e-5 * scale


@pytest.mark.parametrize("n,p,K,pad,chunks", [
    (5003, 1000, 10, 0, 1),    # the K-means workload's p and K, ragged n
    (4000, 1024, 10, 0, 3),    # chunked sums
    (2999, 50, 3, 0, 1),       # scalar path (p % 4 != 0), KC = 4
    (2048, 256, 7, 4, 1),      # padded ldx, KC = 8
    (1500, 128, 16, 0, 1),     # KC = 16
    (1500, 128, 20, 0, 1),     # two register blocks of centres
    (1200, 2048, 40, 0, 1),    # centres exceed shared memory: read through L1/L2
    (3000, 1500, 60, 0, 1),    # two column blocks, two cluster launches (K > 48)
    (2000, 130, 20, 0, 1),     # scalar path with two register blocks
    (7, 33, 2, 0, 1),          # tiny, n < rows per warp group
])
def test_kmeans2_matches_oracle(sk, n, p, K, pad, chunks):
    X, _, _ = synth.mixture(n, p, K, seed=n + p + K, heavy_frac=0.0)
    rng = np.random.default_rng(K)
    rows = rng.choice(n, K, replace=False)
    mu1 = X[rows] + 0.1 * rng.standard_normal((K, p)).astype(np.float32)
    labels1 = rng.integers(0, K, n).astype(np.int32)
    if K > 2:
        labels1[labels1 == K - 1] = 0   # an empty 1-pass cluster keeps its centre
    _check_2pass(sk, X.astype(np.float32), labels1, mu1, pad=pad, chunks=chunks)


def test_kmeans2_skips_out_of_range_labels(sk):
    n, p, K = 1000, 64, 4
    X = synth.uniform(n, p, seed=3)
    l1 = np.random.default_rng(2).integers(-1, K + 1, n).astype(np.int32)
    ctx = sk.sk_init(p, 8, 1)
    sums = torch.zeros((K, p), dtype=torch.float64, device="cuda")
    counts = torch.zeros(K, dtype=torch.int64, device="cuda")
    sk.sk_kmeans2_sums(ctx, _dev(X), _dev(l1), K, sums, counts)
    torch.cuda.synchronize()
    for k in range(K):
        sel = l1 == k
        assert counts[k].item() == sel.sum()
        assert np.abs(sums[k].cpu().numpy() - X[sel].astype(np.float64).sum(0)).max() <= 1e-4


def test_kmeans2_after_one_pass_pipeline(sk):
    """Algorithm 2 end to end on the tiny workload: 1-pass sparsified K-means
    on the GPU, un-mix, then the second pass; checked against the oracle run
    on the same seeded X from the oracle's own 1-pass result."""
    from paper_1511_00152_gb300 import pipeline
    n, p, m, K, seed, iters = 4000, 64, 8, 5, 11, 6
    X, _, _ = synth.mixture(n, p, K, seed=4, heavy_frac=0.0)
    ctx = sk.sk_init(p, m, seed)
    Xd = _dev(X)
    idx, val = sk.sk_compress(ctx, Xd)
    rows = synth.init_rows(n, K, seed)
    mu0 = sk.sk_precondition(ctx, Xd[torch.as_tensor(rows, device="cuda")].contiguous())
    st = pipeline.KMeansState(ctx, n, K)
    st.run(idx, val, mu0, iters, use_graph=False)
    mu_x = sk.sk_unmix(ctx, st.mu)
    c2, mu2, counts = pipeline.kmeans_2pass(ctx, Xd, st.labels, mu_x, chunk_rows=1500)
    torch.cuda.synchronize()
    # oracle: its own 1-pass run from its own compression
    oi, ov = oracle.compress(X, m, seed)
    Y0 = oracle.precondition(X[rows], seed)
    lo, muo, _ = oracle.kmeans(oi, ov, Y0, ctx.pt, iters)
    mux_o = oracle.unmix(muo, p, seed)
    c2o, mu2o, cnto = oracle.kmeans_2pass(X, lo, mux_o)
    # well-separated mixture: the two runs agree on the 1-pass labels
    assert np.mean(st.labels.cpu().numpy() == lo) > 0.999
    assert np.mean(c2.cpu().numpy() == c2o) > 0.999
    assert np.abs(counts.cpu().numpy() - cnto).sum() <= 0.002 * n
    if np.array_equal(st.labels.cpu().numpy(), lo):
        assert np.abs(mu2.cpu().numpy() - mu2o).max() <= 1e-4


# ------------------------------------------------------------- sample mean

@pytest.mark.parametrize("n,p,m,chunks", [
    (20000, 1000, 51, 1),
    (20000, 1000, 51, 4),
    (5000, 64, 8, 1),
    (300, 4096, 205, 1),
    (9000, 3, 2, 2),
])
def test_sample_mean_matches_oracle(sk, n, p, m, chunks):
    seed = 17
    X = synth.lowrank_spiky(n, p, seed=2) + 1.5  # a mean worth estimating
    X = X.astype(np.float32)
    ctx = sk.sk_init(p, m, seed)
    Xd = _dev(X)
    sums = torch.zeros(ctx.pt, dtype=torch.float64, device="cuda")
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        idx, val = sk.sk_compress(ctx, Xd[a:b], row0=int(a))
        sk.sk_mean_accumulate(ctx, idx, val, sums)
    mean = sk.sk_mean_finalize(ctx, sums, n)
    mean_x = sk.sk_unmix(ctx, mean[None, :])
    torch.cuda.synchronize()
    oi, ov = oracle.compress(X, m, seed)
    mo = oracle.sample_mean(oi, ov, ctx.pt)
    tol = 1e-5 * np.abs(mo).max() + 1e-6 * np.sqrt(np.mean(ov * ov))
    assert np.abs(mean.cpu().numpy() - mo).max() <= tol
    mxo = oracle.unmix(mo[None, :], p, seed)
    assert np.abs(mean_x.cpu().numpy() - mxo).max() <= tol


def test_sample_mean_rejects_bad_args(sk):
    ctx = sk.sk_init(64, 8, 1)
    s = torch.zeros(ctx.pt, dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError):
        sk.sk_mean_finalize(ctx, s, 0)


def test_hk_deviation_matches_oracle(sk):
    """||H_k - I|| (Sec. VI-B) from the GPU's sums against the oracle's on the
    oracle's own rows and labels."""
    n, p, m, K, seed = 6000, 256, 13, 5, 4
    X = synth.uniform(n, p, seed=7)
    ctx = sk.sk_init(p, m, seed)
    oi, ov = oracle.compress(X, m, seed)
    labels = (np.arange(n) % (K - 1)).astype(np.int32)  # cluster K-1 empty
    _mu, counts_o, nk_o = oracle.kmeans_update(oi, ov, labels, np.zeros((K, ctx.pt)), ctx.pt)
    ref = oracle.kmeans_hk(counts_o, nk_o, ctx.pt, m)
    S = torch.zeros((K, ctx.pt), dtype=torch.float64, device="cuda")
    cnt = torch.zeros((K, ctx.pt), dtype=torch.int32, device="cuda")
    nk = torch.zeros(K, dtype=torch.int64, device="cuda")
    sk.sk_kmeans_update(ctx, _dev(oi), _dev(ov.astype(np.float32)), _dev(labels), K, S, cnt, nk)
    dev = sk.sk_kmeans_hk(ctx, cnt, nk)
    torch.cuda.synchronize()
    assert np.array_equal(cnt.cpu().numpy(), counts_o)
    assert np.abs(dev.cpu().numpy() - ref).max() <= 1e-14
    assert dev[K - 1].item() == -1.0


@pytest.mark.parametrize("p,m,n,mode", [(64, 8, 2000, 0), (256, 13, 3000, 2), (1000, 50, 1500, 2),
                                        (1024, 51, 4000, 0), (4096, 205, 300, 2)])
def test_cov_centred_matches_oracle(p, m, n, mode):
    """Centred covariance estimate (C_n - xbar xbar^T + B(C_n)/n) against the
    FP64 oracle on the same seeded rows, accumulated over two chunks:
    relative Frobenius <= 1e-6 (FP32 Gram) or 1e-5 (split-BF16 Gram)."""
    import oracle
    from paper_1511_00152_gb300 import _lib as sk
    X = synth.lowrank_spiky(n, p, seed=p + n) + 0.5
    seed = 19
    ctx = sk.sk_init(p, m, seed)
    idx, val = sk.sk_compress(ctx, torch.as_tensor(X, device="cuda"))
    G = torch.zeros((ctx.pt, ctx.pt), dtype=torch.float64, device="cuda")
    sums = torch.zeros(ctx.pt, dtype=torch.float64, device="cuda")
    h = n // 3
    for a, b in ((0, h), (h, n)):
        sk.sk_cov_accumulate(ctx, mode, idx[a:b].contiguous(), val[a:b].contiguous(), G)
        sk.sk_mean_accumulate(ctx, idx[a:b].contiguous(), val[a:b].contiguous(), sums)
    mean = sk.sk_mean_finalize(ctx, sums, n)
    C = sk.sk_cov_finalize_centred(ctx, G, mean, n)
    torch.cuda.synchronize()
    oi, ov = oracle.compress(X, m, seed)
    Co = oracle.cov_centred(oracle.gram(oi, ov, ctx.pt), oracle.sample_mean(oi, ov, ctx.pt), n, m)
    tol = 1e-6 if mode == 0 else 1e-5
    Cg = C.cpu().numpy()
    assert np.allclose(Cg, Cg.T)
    assert np.linalg.norm(Cg - Co) <= tol * np.linalg.norm(Co)
    # the pipeline helper gives the same estimate
    from paper_1511_00152_gb300 import pipeline
    C2, mean2 = pipeline.covariance_centred(ctx, idx, val, mode)
    torch.cuda.synchronize()
    assert np.linalg.norm(C2.cpu().numpy() - Co) <= tol * np.linalg.norm(Co)
    assert sk.sk_device_status() == sk.SK_OK
