"""Full-size parity: the benchmark's workloads at their full sizes, in the
launch configuration bench.py times, checked against the FP64 oracle.

K-means workload: n = 1,000,000, p = 1024, m = 51, K = 10, 20 iterations.
  The oracle compresses every row (idx bit-exact, val <= 1e-5 ||x_r|| for all
  10^6 rows) and runs its own 20 iterations from the same seeded start; the
  GPU's CUDA-graph loop (with its labels recorded each iteration) must follow
  it: a differing label is a near-tie or involves a cluster an earlier
  near-tie touched, and the untouched clusters' centres, counts and sizes
  agree (tests/kmeans_trace.py).
PCA workload: n = 1,048,576, p = 4096, m = 205, top-20.
  * every row's idx bit-exact and val <= 1e-5 ||x_r||;
  * over all rows (four FP32 accumulation segments per tile of the
    tensor-core Gram, then the FP64 reduction), the Gram restricted to a
    seeded set J of 256 coordinates against the oracle's Gram of the same
    entries: relative Frobenius <= 1e-5 split-BF16, <= 1e-2 BF16;
  * on the first 70,000 rows, the whole Gram and C_n element by element
    (split-BF16 1e-5, BF16 1e-2, FP32 1e-6), and the GPU's top-20 of its C_n
    against the oracle's LAPACK top-20 of the oracle's C_n: principal angles
    within the Davis-Kahan bound ||C_oracle U - U L||_2 / (min L -
    lambda_21(C_oracle)) for the GPU's Ritz pairs (U, L), each Ritz value
    within its residual of an oracle eigenvalue;
  * at full size, the top-20 eigen-residuals <= 1e-6 and orthonormality.

The oracle only ever receives inputs drawn by the seeded generator (rows copied
back from the device generator) -- never a value computed by the CUDA path.
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


def _compress_all_checked(ctx, X, idx, val, m, seed, chunk, on_chunk=None):
    """Oracle compress of every row, chunk by chunk: idx bit-exact, val within
    1e-5 of the row norm; on_chunk(r0, oi, ov) sees each chunk's ELL."""
    n = X.shape[0]
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        Xc = X[r0:r1].cpu().numpy()
        oi, ov = oracle.compress(Xc, m, seed, row0=r0)
        assert np.array_equal(idx[r0:r1].cpu().numpy(), oi), f"idx differs in rows {r0}..{r1}"
        err = np.abs(val[r0:r1].cpu().numpy().astype(np.float64) - ov).max(axis=1)
        nrm = np.linalg.norm(Xc.astype(np.float64), axis=1)
        assert np.all(err <= 1e-5 * nrm), f"val differs in rows {r0}..{r1}"
        if on_chunk is not None:
            on_chunk(r0, oi, ov)


def test_kmeans_workload_full_size(sk):
    from paper_1511_00152_gb300 import pipeline
    n, p, m, K, seed, iters = 1_000_000, 1024, 51, 10, 20240611, 20
    ctx = sk.sk_init(p, m, seed)
    X, _, _ = synth.mixture_device(n, p, 10, seed)
    idx, val = sk.sk_compress(ctx, X)
    oi = np.empty((n, m), np.int32)
    ov = np.empty((n, m), np.float64)

    def keep_chunk(r0, ci, cv):
        oi[r0:r0 + len(ci)] = ci
        ov[r0:r0 + len(ci)] = cv

    _compress_all_checked(ctx, X, idx, val, m, seed, 1 << 17, keep_chunk)
    init = synth.init_rows(n, K, seed)
    Xi = X[torch.as_tensor(init, device=X.device)].contiguous()
    mu0 = sk.sk_precondition(ctx, Xi)
    st = pipeline.KMeansState(ctx, n, K)
    hist = torch.empty((iters, n), dtype=torch.int32, device="cuda")
    st.run(idx, val, mu0, iters, use_graph=True, history=hist)
    torch.cuda.synchronize()
    trace = kmeans_trace.oracle_trace(oi, ov, oracle.precondition(Xi.cpu().numpy(), seed),
                                      ctx.pt, iters)
    keep, nflip = kmeans_trace.check_against_trace(
        list(hist.cpu().numpy()), st.mu.cpu().numpy(), st.cnt.cpu().numpy(), st.nk.cpu().numpy(),
        trace, K, max_touched_frac=0.6)
    assert nflip <= n * iters // 1000, nflip
    # size-independent invariants of the sums (Eq. (mu_update_one))
    nk = st.nk.cpu().numpy()
    assert nk.sum() == n
    assert np.array_equal(st.cnt.cpu().numpy().sum(axis=1), m * nk)
    assert sk.sk_device_status() == sk.SK_OK


def _sym_from_upper(G):
    U = np.triu(G)
    return U + U.T - np.diag(np.diag(U))


def _restricted(oi, ov, pos, width):
    """The entries of each row whose coordinate is in J, relabelled to
    0..|J|-1 and padded with zero values (which add nothing to a Gram)."""
    P = pos[oi]
    sel = P >= 0
    c = max(1, int(sel.sum(axis=1).max()))
    order = np.argsort(~sel, axis=1, kind="stable")[:, :c]
    rows = np.arange(oi.shape[0])[:, None]
    take = sel[rows, order]
    return (np.where(take, P[rows, order], 0).astype(np.int32),
            np.where(take, ov[rows, order], 0.0))


def test_pca_workload_full_size(sk):
    n, p, m, k, seed = 1_048_576, 4096, 205, 20, 7
    n0 = 70_000
    ctx = sk.sk_init(p, m, seed)
    pt = ctx.pt
    X = synth.lowrank_decay_device(n, p, seed)
    idx, val = sk.sk_compress(ctx, X)
    J = np.sort(np.random.default_rng(3).choice(pt, 256, replace=False))
    pos = -np.ones(pt, np.int64)
    pos[J] = np.arange(J.size)
    GJ = np.zeros((J.size, J.size))
    pre = {}

    def per_chunk(r0, ci, cv):
        ri, rv = _restricted(ci, cv, pos, J.size)
        oracle.gram(ri, rv, J.size, G=GJ)
        if r0 < n0:
            pre[r0] = (ci[: n0 - r0], cv[: n0 - r0])

    _compress_all_checked(ctx, X, idx, val, m, seed, 1 << 15, per_chunk)
    del X
    torch.cuda.empty_cache()
    GJo = _sym_from_upper(GJ)
    # all rows: the Gram restricted to J
    Gs = {}
    for mode, tol in ((sk.SK_GRAM_BF16X3, 1e-5), (sk.SK_GRAM_BF16, 1e-2)):
        G = torch.zeros((pt, pt), dtype=torch.float64, device="cuda")
        sk.sk_cov_accumulate(ctx, mode, idx, val, G)
        torch.cuda.synchronize()
        Gg = _sym_from_upper(G.cpu().numpy())
        rel = np.linalg.norm(Gg[np.ix_(J, J)] - GJo) / np.linalg.norm(GJo)
        assert rel <= tol, (mode, rel)
        Gs[mode] = G
    # full size: eigen-residuals and orthonormality of the top-20
    C = sk.sk_cov_finalize(ctx, Gs[sk.SK_GRAM_BF16X3], n)
    del Gs
    ev, U = sk.sk_cov_topk(ctx, C, k, iters=60)
    torch.cuda.synchronize()
    Cu = C @ U.T
    res = torch.linalg.norm(Cu - U.T * ev[None, :], dim=0) / ev.abs()
    assert res.max().item() <= 1e-6, res.max().item()
    I = U @ U.T
    assert torch.allclose(I, torch.eye(k, dtype=torch.float64, device="cuda"), atol=1e-10)
    assert torch.all(ev[:-1] >= ev[1:])
    del C, Cu, U
    torch.cuda.empty_cache()

    # the first n0 rows: the whole Gram, C_n and the top-20 subspace
    oi0 = np.concatenate([pre[r][0] for r in sorted(pre)])
    ov0 = np.concatenate([pre[r][1] for r in sorted(pre)])
    assert oi0.shape[0] == n0
    Go = oracle.gram(oi0, ov0, pt)
    Gou = np.triu(Go)
    Co = oracle.cov_finalize(Go, n0, m)
    for mode, tol in ((sk.SK_GRAM_BF16X3, 1e-5), (sk.SK_GRAM_BF16, 1e-2), (sk.SK_GRAM_FP32, 1e-6)):
        G = torch.zeros((pt, pt), dtype=torch.float64, device="cuda")
        sk.sk_cov_accumulate(ctx, mode, idx[:n0].contiguous(), val[:n0].contiguous(), G)
        Cg = sk.sk_cov_finalize(ctx, G, n0)
        torch.cuda.synchronize()
        rel = np.linalg.norm(np.triu(G.cpu().numpy()) - Gou) / np.linalg.norm(Gou)
        assert rel <= tol, (mode, rel)
        relc = np.linalg.norm(Cg.cpu().numpy() - Co) / np.linalg.norm(Co)
        assert relc <= tol + 1e-6, (mode, relc)
        if mode == sk.SK_GRAM_BF16X3:
            evg, Ug = sk.sk_cov_topk(ctx, Cg, k, iters=200)
            torch.cuda.synchronize()
            Cgh = Cg.cpu().numpy()
            evg = evg.cpu().numpy()
            Ug = Ug.cpu().numpy().T  # pt x k
    wo, Vo = oracle.pca_topk(Co, 2 * k)
    # Davis-Kahan sin-theta theorem for the GPU's Ritz pairs (U orthonormal,
    # Ritz values in [min evg, max evg]) against the oracle's C_n: the sines
    # of the principal angles to the oracle's top-k subspace are at most
    # ||Co U - U diag(evg)||_2 / (min evg - lambda_{k+1}(Co))
    assert np.abs(Ug.T @ Ug - np.eye(k)).max() <= 1e-10
    Ro = Co @ Ug - Ug * evg[None, :]
    delta = evg.min() - wo[k]
    assert delta > 0, (evg.min(), wo[k])
    bound = np.linalg.norm(Ro, 2) / delta
    s = np.linalg.svd(Vo[:, :k].T @ Ug, compute_uv=False)
    sin_max = float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))
    print(f"top-{k} on {n0} rows: sin {sin_max:.3e} bound {bound:.3e} "
          f"(||Cg - Co||_F {np.linalg.norm(Cgh - Co):.3e}, gap {delta:.3e}, "
          f"lambda_1 {wo[0]:.3e})")
    assert sin_max <= bound + 1e-12
    # each Ritz value lies within its residual of an eigenvalue of Co
    # (Krylov-Weinstein)
    for i in range(k):
        assert np.abs(wo - evg[i]).min() <= np.linalg.norm(Ro[:, i]) + 1e-14 * wo[0], i
    assert sk.sk_device_status() == sk.SK_OK
