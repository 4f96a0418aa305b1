"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (stated per result):
  idx      bit-exact
  val      |val_gpu - val_oracle| <= 1e-5 * ||x_r||_2       (FP32 transform)
  Y dense  same bound per row
  Gram     FP32 scatter: relative Frobenius <= 1e-6
  C_n      relative Frobenius <= 1e-6 (FP32 Gram)
  labels   identical where the oracle's best and second-best restricted
           distances differ by more than 1e-4 relative (near-tie band); over
           several iterations, every differing label is a near-tie or involves
           a cluster an earlier near-tie touched (tests/kmeans_trace.py)
  sums     cnt and nk exact; S within 1e-5 relative (float products summed in
           FP32 per CTA then FP64), per cluster no near-tie touched, and for
           every cluster under the oracle's labels
  centres  relative error <= 1e-5 (same clusters)
  top-k    max sin(principal angle) <= 1e-6
  unmix    |err| <= 1e-5 * ||row||
"""
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


def _check_compress(sk, X, m, seed, row0=0, ldx_pad=0):
    n, p = X.shape
    ctx = sk.sk_init(p, m, seed)
    if ldx_pad:
        Xw = np.zeros((n, p + ldx_pad), np.float32)
        Xw[:, :p] = X
        Xd = _dev(Xw)[:, :p]
    else:
        Xd = _dev(X)
    idx, val = sk.sk_compress(ctx, Xd, row0=row0)
    torch.cuda.synchronize()
    oi, ov = oracle.compress(X, m, seed, row0=row0)
    gi = idx.cpu().numpy()
    gv = val.cpu().numpy().astype(np.float64)
    assert np.array_equal(gi, oi), "mask indices differ"
    norms = np.linalg.norm(X.astype(np.float64), axis=1)
    err = np.abs(gv - ov).max(axis=1) if m else np.zeros(n)
    assert np.all(err <= 1e-5 * np.maximum(norms, 1e-30)), float((err / np.maximum(norms, 1e-30)).max())
    return ctx


@pytest.mark.parametrize("p,m,n", [
    (64, 8, 2000),      # tiny workload shape
    (50, 7, 333),       # zero padding to 64, ragged row count
    (1024, 51, 3000),   # K-means workload shape
    (1000, 50, 1000),   # padding to 1024
    (4096, 205, 300),   # PCA workload shape
    (2048, 102, 500),   # streaming workload shape
    (8192, 820, 40),    # largest pt, m = 10%
    (256, 13, 1000),
    (8, 3, 100),
    (1, 1, 10),
    (2, 2, 10),
    (16, 16, 50),       # m = pt: a permutation per row
    (128, 1, 77),
    (4, 4, 1),
    (700, 35, 5),
    (3001, 150, 64),    # pt = 4096, rows not 16-byte multiples: the one-kernel path
    (4000, 200, 129),   # pt = 4096 with padding: masks drawn by their own kernel
])
def test_compress_parity(sk, p, m, n):
    X = synth.lowrank_spiky(n, p, seed=p * 7 + n, sv=(10.0, 6.0, 4.0, 2.0, 1.0)[: max(1, min(5, p))])
    _check_compress(sk, X, m, seed=1234 + p)


def test_compress_row0_and_strided(sk):
    X = synth.mixture(777, 300, 4, seed=3)[0]
    _check_compress(sk, X, 15, seed=99, row0=(1 << 33) + 17, ldx_pad=13)
    _check_compress(sk, X, 15, seed=99, row0=5, ldx_pad=4)
    X2 = synth.mixture(150, 2500, 3, seed=5)[0]
    _check_compress(sk, X2, 120, seed=98, row0=(1 << 33) + 3, ldx_pad=4)


def test_compress_chunked_equals_single(sk):
    X = _dev(synth.uniform(5000, 1024, seed=4))
    ctx = sk.sk_init(1024, 51, 7)
    i1, v1 = sk.sk_compress(ctx, X)
    parts = [(0, 1234), (1234, 1235), (1235, 4000), (4000, 5000)]
    for a, b in parts:
        ia, va = sk.sk_compress(ctx, X[a:b].contiguous(), row0=a)
        assert torch.equal(ia, i1[a:b]) and torch.equal(va, v1[a:b])


@pytest.mark.parametrize("p", [64, 100, 1024, 4096, 8192])
def test_precondition_parity(sk, p):
    X = synth.lowrank_spiky(37, p, seed=p)
    ctx = sk.sk_init(p, 2, 55)
    Y = sk.sk_precondition(ctx, _dev(X)).cpu().numpy().astype(np.float64)
    Yo = oracle.precondition(X, 55)
    norms = np.linalg.norm(X.astype(np.float64), axis=1)
    assert np.all(np.abs(Y - Yo).max(axis=1) <= 1e-5 * norms)


def _near_tie_mask(idx, val, mu, pt, rel=1e-4):
    """Rows whose best and second-best oracle distances are within rel."""
    K = mu.shape[0]
    n, m = idx.shape
    d = np.zeros((n, K))
    for k in range(K):
        diff = val - mu[k][idx]
        d[:, k] = (diff * diff).sum(1)
    ds = np.sort(d, axis=1)
    if K == 1:
        return np.zeros(n, bool)
    return (ds[:, 1] - ds[:, 0]) <= rel * np.maximum(ds[:, 0], 1e-30)


@pytest.mark.parametrize("p,m,n,K", [(64, 8, 2000, 5), (1024, 51, 4000, 10), (2048, 102, 1500, 8),
                                     (256, 5, 3000, 50), (128, 13, 500, 1), (512, 26, 700, 70),
                                     (64, 8, 300, 200)])
def test_kmeans_step_teacher_forced(sk, p, m, n, K):
    """One fused assign+update pass from the oracle's centres (teacher forcing)."""
    X = synth.mixture(n, p, min(K, 10), seed=p + K)[0]
    seed = 17
    ctx = sk.sk_init(p, m, seed)
    pt = ctx.pt
    idx, val = sk.sk_compress(ctx, _dev(X))
    oi, ov = oracle.compress(X, m, seed)
    rows = synth.init_rows(n, K, seed)
    mu = oracle.precondition(X[rows], seed)
    trace = kmeans_trace.oracle_trace(oi, ov, mu, pt, 1)
    labels_o = trace["labels"][0]
    dist_o = kmeans_trace.restricted_distances(oi, ov, mu)[np.arange(n), labels_o]
    mu_new_o, counts_o, nk_o = trace["mu"], trace["counts"], trace["nk"]

    mu_d = _dev(mu.astype(np.float32))
    # assign alone
    lab_a, _ = sk.sk_kmeans_assign(ctx, idx, val, mu_d)
    # fused step
    S = torch.zeros((K, pt), dtype=torch.float64, device="cuda")
    cnt = torch.zeros((K, pt), dtype=torch.int32, device="cuda")
    nk = torch.zeros(K, dtype=torch.int64, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    dist = torch.empty(n, dtype=torch.float32, device="cuda")
    sk.sk_kmeans_reset(ctx, S, cnt, nk)
    sk.sk_kmeans_step(ctx, idx, val, mu_d, labels, S, cnt, nk, dist=dist)
    torch.cuda.synchronize()
    gl = labels.cpu().numpy()
    assert np.array_equal(gl, lab_a.cpu().numpy())
    tie = _near_tie_mask(oi, ov, mu, pt)
    assert np.array_equal(gl[~tie], labels_o[~tie])
    same = gl == labels_o
    assert np.allclose(dist.cpu().numpy()[same], dist_o[same], rtol=1e-4, atol=1e-6)
    # sums and centres over the clusters no near-tie row moved into or out of
    # (all of them unless a near-tie went the other way)
    sk.sk_kmeans_finalize(ctx, S, cnt, mu_d)
    keep, _ = kmeans_trace.check_against_trace([gl], mu_d.cpu().numpy(), cnt.cpu().numpy(),
                                               nk.cpu().numpy(), trace, K)
    So = np.where(counts_o > 0, mu_new_o * counts_o, 0.0)
    scale = np.abs(So).max() + 1e-30
    assert np.abs(S.cpu().numpy()[keep] - So[keep]).max() <= 1e-5 * scale
    # update alone under the oracle labels: every cluster, no tie can excuse a
    # difference here
    S2 = torch.zeros_like(S)
    c2 = torch.zeros_like(cnt)
    n2 = torch.zeros_like(nk)
    sk.sk_kmeans_update(ctx, idx, val, _dev(labels_o), K, S2, c2, n2)
    torch.cuda.synchronize()
    assert np.array_equal(c2.cpu().numpy(), counts_o)
    assert np.array_equal(n2.cpu().numpy(), nk_o)
    assert np.abs(S2.cpu().numpy() - So).max() <= 1e-5 * scale
    mu2 = _dev(mu.astype(np.float32))
    sk.sk_kmeans_finalize(ctx, S2, c2, mu2)
    assert np.abs(mu2.cpu().numpy() - mu_new_o).max() <= 1e-5 * (np.abs(mu_new_o).max() + 1e-30)


def test_kmeans_end_to_end_tiny(sk):
    """Tiny workload: n=2000, p=64, m=8, K=5, 10 iterations, eager and as one
    CUDA graph, each against the oracle's own run (labels per iteration,
    final centres, counts and un-mixed centres over the untouched clusters)."""
    from paper_1511_00152_gb300 import pipeline
    n, p, m, K, seed, iters = 2000, 64, 8, 5, 1, 10
    X = synth.lowrank_spiky(n, p, seed=seed)
    ctx = sk.sk_init(p, m, seed)
    Xd = _dev(X)
    idx, val = sk.sk_compress(ctx, Xd)
    rows = synth.init_rows(n, K, seed)
    mu0 = pipeline.initial_centres(ctx, Xd, rows)
    oi, ov = oracle.compress(X, m, seed)
    trace = kmeans_trace.oracle_trace(oi, ov, oracle.precondition(X[rows], seed), ctx.pt, iters)
    umo = oracle.unmix(trace["mu"], p, seed)
    for use_graph in (False, True):
        st = pipeline.KMeansState(ctx, n, K)
        hist = torch.empty((iters, n), dtype=torch.int32, device="cuda")
        labels, mu = st.run(idx, val, mu0, iters=iters, use_graph=use_graph, history=hist)
        torch.cuda.synchronize()
        gh = hist.cpu().numpy()
        assert np.array_equal(gh[-1], labels.cpu().numpy())
        keep, nflip = kmeans_trace.check_against_trace(list(gh), mu.cpu().numpy(),
                                                       st.cnt.cpu().numpy(), st.nk.cpu().numpy(),
                                                       trace, K)
        assert nflip <= n * iters // 100, nflip
        um = sk.sk_unmix(ctx, mu).cpu().numpy().astype(np.float64)
        assert np.abs(um[keep] - umo[keep]).max() <= 1e-5 * np.abs(umo).max()


@pytest.mark.parametrize("p,m,n", [(64, 8, 2000), (1024, 51, 3000), (300, 20, 1000), (4096, 205, 200),
                                   (256, 2, 500), (128, 128, 100)])
def test_gram_fp32_and_cov_parity(sk, p, m, n):
    X = synth.lowrank_spiky(n, p, seed=n + p)
    seed = 3
    ctx = sk.sk_init(p, m, seed)
    pt = ctx.pt
    idx, val = sk.sk_compress(ctx, _dev(X))
    oi, ov = oracle.compress(X, m, seed)
    Go = oracle.gram(oi, ov, pt)
    G = torch.empty((pt, pt), dtype=torch.float64, device="cuda")
    sk.sk_cov_reset(ctx, G)
    # two chunks accumulate into the same G
    h = n // 3
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx[:h].contiguous(), val[:h].contiguous(), G)
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_FP32, idx[h:].contiguous(), val[h:].contiguous(), G)
    C = sk.sk_cov_finalize(ctx, G, n)
    torch.cuda.synchronize()
    Gg = np.triu(G.cpu().numpy())
    Gu = np.triu(Go)
    assert np.linalg.norm(Gg - Gu) <= 1e-6 * np.linalg.norm(Gu)
    Co = oracle.cov_finalize(Go, n, m)
    Cg = C.cpu().numpy()
    assert np.allclose(Cg, Cg.T)
    assert np.linalg.norm(Cg - Co) <= 1e-6 * np.linalg.norm(Co)


def test_cov_finalize_exact_from_oracle_gram(sk):
    p, m, n = 256, 20, 50
    ctx = sk.sk_init(p, m, 1)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((p, p))
    Go = A + A.T
    C = sk.sk_cov_finalize(ctx, _dev(Go), n).cpu().numpy()
    Co = oracle.cov_finalize(Go, n, m)
    assert np.abs(C - Co).max() <= 1e-14 * np.abs(Co).max()


@pytest.mark.parametrize("pt,k", [(64, 5), (1024, 10), (256, 20)])
def test_topk_parity(sk, pt, k):
    """Top-k subspace of a symmetric matrix with a clear spectral gap."""
    rng = np.random.default_rng(pt + k)
    Q, _ = np.linalg.qr(rng.standard_normal((pt, pt)))
    lam = np.concatenate([np.linspace(10, 5, k), rng.uniform(-0.5, 1.0, pt - k)])
    C = (Q * lam) @ Q.T
    C = 0.5 * (C + C.T)
    ctx = sk.sk_init(pt, 2, 8)
    ev, U = sk.sk_cov_topk(ctx, _dev(C), k, iters=60)
    torch.cuda.synchronize()
    wo, Vo = oracle.pca_topk(C, k)
    assert np.allclose(ev.cpu().numpy(), wo, rtol=1e-9, atol=1e-9)
    Ug = U.cpu().numpy().T
    s = np.linalg.svd(Vo.T @ Ug, compute_uv=False)
    sin_max = np.sqrt(max(0.0, 1.0 - s.min() ** 2))
    assert sin_max <= 1e-6, sin_max


def test_pca_tiny_workload(sk):
    """Tiny workload: C_n from n=2000, p=64, m=8 and its top-5 subspace."""
    from paper_1511_00152_gb300 import pipeline
    n, p, m, seed = 2000, 64, 8, 1
    X = synth.lowrank_spiky(n, p, seed=seed)
    ctx = sk.sk_init(p, m, seed)
    idx, val = sk.sk_compress(ctx, _dev(X))
    C = pipeline.covariance(ctx, idx, val, sk.SK_GRAM_FP32)
    ev, Up, U = pipeline.pca(ctx, C, 5, iters=200)
    torch.cuda.synchronize()
    oi, ov = oracle.compress(X, m, seed)
    Co = oracle.cov(oi, ov, ctx.pt)
    wo, Vo = oracle.pca_topk(Co, 5)
    assert np.allclose(ev.cpu().numpy(), wo, rtol=1e-5)
    s = np.linalg.svd(Vo.T @ Up.cpu().numpy().T, compute_uv=False)
    assert np.sqrt(max(0.0, 1 - s.min() ** 2)) <= 1e-4
    Uo = oracle.unmix(Vo.T.copy(), p, seed)
    s2 = np.linalg.svd(Uo @ U.cpu().numpy().T, compute_uv=False)
    assert np.sqrt(max(0.0, 1 - s2.min() ** 2)) <= 1e-4


def test_unmix_parity(sk):
    p = 1000
    ctx = sk.sk_init(p, 10, 21)
    M = np.random.default_rng(1).standard_normal((7, ctx.pt))
    out = sk.sk_unmix(ctx, _dev(M.astype(np.float32))).cpu().numpy().astype(np.float64)
    ref = oracle.unmix(M.astype(np.float32).astype(np.float64), p, 21)
    assert np.abs(out - ref).max() <= 1e-5 * np.linalg.norm(M, axis=1).max()
    out64 = sk.sk_unmix(ctx, _dev(M)).cpu().numpy()
    assert np.abs(out64 - oracle.unmix(M, p, 21)).max() <= 1e-12 * np.abs(M).max()


def test_invalid_arguments_rejected_before_launch(sk):
    import ctypes
    lib = sk.load()
    h = ctypes.c_void_p(0)
    assert lib.sk_init(ctypes.byref(h), 0, 1, 0) == sk.SK_EINVAL
    assert lib.sk_init(ctypes.byref(h), 10000, 1, 0) == sk.SK_EUNSUPPORTED
    assert lib.sk_init(ctypes.byref(h), 64, 65, 0) == sk.SK_EINVAL
    assert lib.sk_init(ctypes.byref(h), 64, 0, 0) == sk.SK_EINVAL
    ctx = sk.sk_init(64, 1, 0)
    nul = ctypes.c_void_p(0)
    assert lib.sk_compress(ctx.handle, nul, 10, 64, 0, nul, nul, nul) == sk.SK_EINVAL
    assert lib.sk_compress(ctx.handle, nul, -1, 64, 0, nul, nul, nul) == sk.SK_EINVAL
    assert lib.sk_compress(ctx.handle, nul, 0, 64, 0, nul, nul, nul) == sk.SK_OK  # n = 0 no-op
    assert lib.sk_compress(ctx.handle, nul, 5, 10, 0, nul, nul, nul) == sk.SK_EINVAL  # ldx < p
    G = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    # m = 1: covariance needs m >= 2 (Thm. B1)
    assert lib.sk_cov_finalize(ctx.handle, sk._ptr(G), 10, sk._ptr(G), nul) == sk.SK_EINVAL
    ctx2 = sk.sk_init(64, 4, 0)
    assert lib.sk_cov_finalize(ctx2.handle, sk._ptr(G), 10, sk._ptr(G), nul) == sk.SK_EINVAL  # overlap
    assert lib.sk_cov_accumulate(ctx2.handle, 7, nul, nul, 5, nul, nul, 0, nul) == sk.SK_EINVAL
    ctx3 = sk.sk_init(256, 4, 0)
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    # tensor-core mode without its workspace: rejected before any launch
    assert lib.sk_cov_accumulate(ctx3.handle, sk.SK_GRAM_BF16X3, sk._ptr(d), sk._ptr(d), 4,
                                 sk._ptr(G), nul, 0, nul) == sk.SK_EINVAL
    assert "workspace" in sk.sk_last_error()
    assert lib.sk_kmeans_assign(ctx2.handle, nul, nul, 5, nul, 0, nul, nul, nul) == sk.SK_EINVAL
    assert lib.sk_cov_topk(ctx2.handle, sk._ptr(G), 0, 10, nul, nul, nul, nul) == sk.SK_EINVAL
    assert "must be" in sk.sk_last_error() or sk.sk_last_error() != ""
    assert sk.sk_device_status() == sk.SK_OK


def _sums_of_labels(labs, oi, v32, K, pt, m):
    """Eq. (mu_update_one) written out with numpy over the input rows."""
    labs = np.asarray(labs).astype(np.int64)
    lk = np.repeat(labs, m)
    counts = np.zeros((K, pt), np.int64)
    S = np.zeros((K, pt))
    np.add.at(counts, (lk, oi.ravel()), 1)
    np.add.at(S, (lk, oi.ravel()), v32.astype(np.float64).ravel())
    return counts, S, np.bincount(labs, minlength=K)


def _loop_inputs(sk, p, m, n, K, dseed, seed, iters):
    from paper_1511_00152_gb300 import pipeline
    X = synth.mixture(n, p, min(K, 10), seed=dseed)[0]
    ctx = sk.sk_init(p, m, seed)
    Xd = _dev(X)
    # the ELL rows are the oracle's (rounded to float32), so the expected sums
    # and the oracle's run below start from inputs, never from a GPU result
    oi, ov = oracle.compress(X, m, seed)
    v32 = ov.astype(np.float32)
    rows = synth.init_rows(n, K, seed)
    mu0 = pipeline.initial_centres(ctx, Xd, rows)
    trace = kmeans_trace.oracle_trace(oi, v32.astype(np.float64), oracle.precondition(X[rows], seed),
                                      ctx.pt, iters)
    return ctx, oi, v32, _dev(oi), _dev(v32), mu0, trace


@pytest.mark.parametrize("p,m,n,K", [(64, 8, 2000, 5), (1024, 51, 20000, 10), (256, 5, 5000, 50)])
def test_kmeans_incremental_sums_match_recomputed(sk, p, m, n, K):
    """sk_kmeans_step_delta keeps S, cnt, nk equal to the sums of
    Eq. (mu_update_one) for the current labels: counts exactly, sums to FP64
    rounding; incremental and full-rebuild loops both follow the oracle's run."""
    from paper_1511_00152_gb300 import pipeline
    iters = 8
    ctx, oi, v32, idx, val, mu0, trace = _loop_inputs(sk, p, m, n, K, p + n, 29, iters)
    runs = {}
    for mode in ("incremental", "full"):
        st = pipeline.KMeansState(ctx, n, K, mode=mode)
        hist = torch.empty((iters, n), dtype=torch.int32, device="cuda")
        st.run(idx, val, mu0, iters=iters, use_graph=False, history=hist)
        torch.cuda.synchronize()
        runs[mode] = st
        kmeans_trace.check_against_trace(list(hist.cpu().numpy()), st.mu.cpu().numpy(),
                                         st.cnt.cpu().numpy(), st.nk.cpu().numpy(), trace, K)
    a = runs["incremental"]
    # the running sums describe the final labels exactly
    counts_o, So, nk_o = _sums_of_labels(a.labels.cpu().numpy(), oi, v32, K, ctx.pt, m)
    assert np.array_equal(a.cnt.cpu().numpy(), counts_o)
    assert np.array_equal(a.nk.cpu().numpy(), nk_o)
    # the first pass sums per-CTA float partials, later passes add FP64 deltas
    assert np.abs(a.S.cpu().numpy() - So).max() <= 1e-5 * (np.abs(So).max() + 1e-30)
    assert int(a.changed.item()) > 0


@pytest.mark.parametrize("p,m,n,K", [(64, 8, 2000, 5), (1024, 51, 20000, 10), (256, 5, 5000, 50)])
def test_kmeans_auto_pass_matches_full(sk, p, m, n, K):
    """sk_kmeans_step_auto (full rebuild while many labels change, then
    incremental, chosen on the device) follows the oracle's run, eagerly and
    in a graph, and its sums describe the final labels exactly (counts) or
    to FP64 rounding (S)."""
    from paper_1511_00152_gb300 import pipeline
    iters = 8
    ctx, oi, v32, idx, val, mu0, trace = _loop_inputs(sk, p, m, n, K, p + n + 1, 31, iters)
    a = pipeline.KMeansState(ctx, n, K, mode="auto")
    a.mu.copy_(mu0)
    modes, moved, hist_a = [], [], []
    for it in range(iters):
        a.iteration(idx, val, first=(it == 0))
        modes.append(int(a.state[1].item()))
        moved.append(int(a.state[0].item()))
        assert int(a.state[2].item()) == 0  # the scratch counter is left at zero
        hist_a.append(a.labels.cpu().numpy().copy())
        if it > 0:
            # the count of changed rows matches the labels
            assert moved[-1] == int((hist_a[-1] != hist_a[-2]).sum())
    # each later pass is a rebuild exactly when the previous one moved more
    # than n / 12 rows
    for it in range(1, iters):
        assert modes[it] == (1 if moved[it - 1] > n // 12 else 2), (modes, moved)
    g = pipeline.KMeansState(ctx, n, K, mode="auto")
    hist_g = torch.empty((iters, n), dtype=torch.int32, device="cuda")
    g.run(idx, val, mu0, iters=iters, use_graph=True, history=hist_g)
    torch.cuda.synchronize()
    assert modes[0] == 1  # the first pass always rebuilds
    assert set(modes) <= {1, 2}
    for st, hist in ((a, hist_a), (g, list(hist_g.cpu().numpy()))):
        kmeans_trace.check_against_trace(hist, st.mu.cpu().numpy(), st.cnt.cpu().numpy(),
                                         st.nk.cpu().numpy(), trace, K)
        counts_o, So, nk_o = _sums_of_labels(st.labels.cpu().numpy(), oi, v32, K, ctx.pt, m)
        assert np.array_equal(st.cnt.cpu().numpy(), counts_o)
        assert np.array_equal(st.nk.cpu().numpy(), nk_o)
        assert np.abs(st.S.cpu().numpy() - So).max() <= 1e-5 * (np.abs(So).max() + 1e-30)
    # state[0] is the last pass's count of changed rows
    assert 0 <= int(a.state[0].item()) <= n
    assert sk.sk_device_status() == sk.SK_OK
