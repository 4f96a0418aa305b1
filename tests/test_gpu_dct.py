"""The DCT preconditioner (SK_FLAG_DCT; Sec. III, H a DCT matrix) on the GPU
against the FP64 oracle, for p that are not powers of two and without zero
padding (pt = p), including the paper's MNIST shape p = 784.

Tolerances as for the Hadamard path: idx bit-exact; val and dense rows
<= 1e-5 ||x_r||; un-mixing <= 1e-5 ||row|| (float32) and 1e-12 (float64);
Gram relative Frobenius 1e-6 (FP32), 1e-5 (split-BF16); C_n likewise; the
K-means step as in tests/test_gpu_parity.py; top-k subspace sin <= 1e-6."""
import ctypes

import numpy as np
import pytest

import kmeans_trace
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


def _ctx(sk, p, m, seed):
    ctx = sk.sk_init_ex(p, m, seed, sk.SK_FLAG_DCT)
    assert ctx.pt == p
    return ctx


@pytest.mark.parametrize("p,m,n", [(784, 39, 3000), (1000, 50, 1001), (2, 1, 10), (6, 3, 77),
                                   (50, 7, 333), (98, 98, 20), (200, 10, 500), (4096, 205, 64),
                                   (8190, 409, 9), (3000, 150, 130)])
def test_dct_compress_parity(sk, p, m, n):
    X = synth.lowrank_spiky(n, p, seed=p + n)
    seed = 300 + p
    ctx = _ctx(sk, p, m, seed)
    idx, val = sk.sk_compress(ctx, _dev(X), row0=11)
    torch.cuda.synchronize()
    oi, ov = oracle.compress(X, m, seed, row0=11, dct=True)
    assert np.array_equal(idx.cpu().numpy(), oi)
    nrm = np.linalg.norm(X.astype(np.float64), axis=1)
    err = np.abs(val.cpu().numpy().astype(np.float64) - ov).max(axis=1)
    assert np.all(err <= 1e-5 * nrm), float((err / nrm).max())
    # dense preconditioned rows
    Y = sk.sk_precondition(ctx, _dev(X)).cpu().numpy().astype(np.float64)
    Yo = oracle.precondition(X, seed, dct=True)
    assert np.all(np.abs(Y - Yo).max(axis=1) <= 1e-5 * nrm)
    assert sk.sk_device_status() == sk.SK_OK


@pytest.mark.parametrize("p", [784, 1000, 8190])
def test_dct_unmix_parity(sk, p):
    ctx = _ctx(sk, p, 10, 5)
    M = np.random.default_rng(p).standard_normal((7, p))
    out = sk.sk_unmix(ctx, _dev(M.astype(np.float32))).cpu().numpy().astype(np.float64)
    ref = oracle.unmix(M.astype(np.float32).astype(np.float64), p, 5, dct=True)
    assert np.abs(out - ref).max() <= 1e-5 * np.linalg.norm(M, axis=1).max()
    out64 = sk.sk_unmix(ctx, _dev(M)).cpu().numpy()
    assert np.abs(out64 - oracle.unmix(M, p, 5, dct=True)).max() <= 1e-12 * np.linalg.norm(M, axis=1).max()
    # un-mixing inverts the preconditioner
    X = synth.lowrank_spiky(5, p, seed=1)
    back = sk.sk_unmix(ctx, sk.sk_precondition(ctx, _dev(X))).cpu().numpy()
    assert np.abs(back - X).max() <= 1e-5 * np.abs(X).max()


@pytest.mark.parametrize("p,m,n", [(784, 39, 3000), (1000, 100, 2000), (200, 20, 1500)])
def test_dct_covariance_parity(sk, p, m, n):
    X = synth.lowrank_spiky(n, p, seed=n)
    seed = 8
    ctx = _ctx(sk, p, m, seed)
    idx, val = sk.sk_compress(ctx, _dev(X))
    oi, ov = oracle.compress(X, m, seed, dct=True)
    Go = oracle.gram(oi, ov, p)
    Co = oracle.cov_finalize(Go, n, m)
    for mode, tol in ((sk.SK_GRAM_FP32, 1e-6), (sk.SK_GRAM_BF16X3, 1e-5)):
        G = torch.zeros((p, p), dtype=torch.float64, device="cuda")
        h = n // 2
        sk.sk_cov_accumulate(ctx, mode, idx[:h].contiguous(), val[:h].contiguous(), G)
        sk.sk_cov_accumulate(ctx, mode, idx[h:].contiguous(), val[h:].contiguous(), G)
        C = sk.sk_cov_finalize(ctx, G, n)
        torch.cuda.synchronize()
        rel = np.linalg.norm(np.triu(G.cpu().numpy()) - np.triu(Go)) / np.linalg.norm(np.triu(Go))
        assert rel <= tol, (mode, rel)
        assert np.linalg.norm(C.cpu().numpy() - Co) <= (tol + 1e-6) * np.linalg.norm(Co)
    # the sample mean and the centred estimate
    sums = torch.zeros(p, dtype=torch.float64, device="cuda")
    sk.sk_mean_accumulate(ctx, idx, val, sums)
    mean = sk.sk_mean_finalize(ctx, sums, n)
    meo = oracle.sample_mean(oi, ov, p)
    assert np.abs(mean.cpu().numpy() - meo).max() <= 1e-5 * np.abs(meo).max()
    G = torch.zeros((p, p), dtype=torch.float64, device="cuda")
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx, val, G)
    Cc = sk.sk_cov_finalize_centred(ctx, G, mean, n).cpu().numpy()
    Cco = oracle.cov_centred(Go, meo, n, m)
    assert np.linalg.norm(Cc - Cco) <= 1e-6 * np.linalg.norm(Cco)
    # top-k of C_n (even p: the panel kernel's 16-byte rows)
    ev, U = sk.sk_cov_topk(ctx, _dev(Co), 5, iters=200)
    wo, Vo = oracle.pca_topk(Co, 5)
    s = np.linalg.svd(Vo.T @ U.cpu().numpy().T, compute_uv=False)
    assert np.sqrt(max(0.0, 1 - s.min() ** 2)) <= 1e-6
    assert np.allclose(ev.cpu().numpy(), wo, rtol=1e-9, atol=1e-12)
    assert sk.sk_device_status() == sk.SK_OK


@pytest.mark.parametrize("p,m,n,K", [(784, 39, 4000, 10), (1000, 50, 2000, 5), (200, 13, 1500, 33)])
def test_dct_kmeans_step(sk, p, m, n, K):
    """One assignment + sums pass from the oracle's centres, and an
    incremental pass after it, at pt = p (not a power of two)."""
    X = synth.mixture(n, p, min(K, 10), seed=p + K)[0]
    seed = 23
    ctx = _ctx(sk, p, m, seed)
    idx, val = sk.sk_compress(ctx, _dev(X))
    oi, ov = oracle.compress(X, m, seed, dct=True)
    rows = synth.init_rows(n, K, seed)
    mu = oracle.precondition(X[rows], seed, dct=True)
    trace = kmeans_trace.oracle_trace(oi, ov, mu, p, 2)
    from paper_1511_00152_gb300 import pipeline
    st = pipeline.KMeansState(ctx, n, K, mode="incremental")
    hist = torch.empty((2, n), dtype=torch.int32, device="cuda")
    st.run(idx, val, _dev(mu.astype(np.float32)), iters=2, use_graph=False, history=hist)
    torch.cuda.synchronize()
    kmeans_trace.check_against_trace(list(hist.cpu().numpy()), st.mu.cpu().numpy(),
                                     st.cnt.cpu().numpy(), st.nk.cpu().numpy(), trace, K)
    um = sk.sk_unmix(ctx, st.mu).cpu().numpy()
    umo = oracle.unmix(trace["mu"], p, seed, dct=True)
    keep, _ = kmeans_trace.untouched(list(hist.cpu().numpy()), trace, K)
    assert np.abs(um[keep] - umo[keep]).max() <= 1e-5 * np.abs(umo).max()
    assert sk.sk_device_status() == sk.SK_OK


def test_dct_init_rejections(sk):
    lib = sk.load()
    h = ctypes.c_void_p(0)
    assert lib.sk_init_ex(ctypes.byref(h), 785, 10, 0, sk.SK_FLAG_DCT) == sk.SK_EUNSUPPORTED  # odd p
    assert lib.sk_init_ex(ctypes.byref(h), 34, 4, 0, sk.SK_FLAG_DCT) == sk.SK_EUNSUPPORTED  # 17
    assert lib.sk_init_ex(ctypes.byref(h), 784, 4, 0,
                          sk.SK_FLAG_DCT | sk.SK_FLAG_NO_PRECONDITION) == sk.SK_EINVAL
    assert lib.sk_init_ex(ctypes.byref(h), 784, 785, 0, sk.SK_FLAG_DCT) == sk.SK_EINVAL  # m > p
