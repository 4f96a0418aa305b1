"""Many data sets, one launch per stage (sk_batch_*): every data set's
result equals the single-data-set call on the same inputs.

  idx, val         bit-exact (same kernel code per data set)
  Gram G           1e-12 relative Frobenius (the same products; only the
                   order of the float64 atomic adds differs)
  labels           identical (same per-row arithmetic), teacher forced
  cnt, nk          exact
  S, centres       1e-6 relative (float partial sums in another order)
"""
import numpy as np
import pytest

from paper_1511_00152_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SETS = [  # (n, p, m, K, seed)
    (3000, 256, 13, 5, 1),
    (1777, 1000, 51, 10, 2),
    (500, 2048, 102, 8, 3),
    (2100, 4096, 82, 20, 4),
    (64, 8192, 819, 50, 5),
    (4097, 512, 26, 33, 6),
]


@pytest.fixture(scope="module")
def run():
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import pipeline
    ds = []
    for (n, p, m, K, seed) in SETS:
        X, _, _ = synth.mixture_device(n, p, min(K, 10), seed)
        ds.append(dict(X=X, m=m, K=K, seed=seed))
    br = pipeline.BatchRun(ds, mode=sk.SK_GRAM_BF16)
    br.compress_and_cov()
    br.init_centres()
    torch.cuda.synchronize()
    return sk, br


def test_batch_compress_and_gram_match_single(run):
    sk, br = run
    for e in br.ds:
        ctx = e["ctx"]
        idx, val = sk.sk_compress(ctx, e["X"])
        G = torch.zeros_like(e["G"])
        sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16, idx, val, G)
        torch.cuda.synchronize()
        assert torch.equal(idx, e["idx"])
        assert torch.equal(val, e["val"])
        U1, U2 = torch.triu(G), torch.triu(e["G"])
        rel = (torch.linalg.norm(U1 - U2) / torch.linalg.norm(U1)).item()
        assert rel <= 1e-12, rel
    assert sk.sk_device_status() == sk.SK_OK


def test_batch_kmeans_pass_matches_single(run):
    sk, br = run
    mus = [e["mu"].clone() for e in br.ds]
    sk.sk_batch_kmeans_reset(br.batch)
    sk.sk_batch_kmeans_step(br.batch, incremental=False)
    torch.cuda.synchronize()
    for e, mu in zip(br.ds, mus):
        ctx, n, K = e["ctx"], e["n"], e["K"]
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        S = torch.zeros_like(e["S"])
        cnt = torch.zeros_like(e["cnt"])
        nk = torch.zeros_like(e["nk"])
        sk.sk_kmeans_step(ctx, e["idx"], e["val"], mu, lab, S, cnt, nk)
        torch.cuda.synchronize()
        assert torch.equal(lab, e["labels"])
        assert torch.equal(cnt, e["cnt"]) and torch.equal(nk, e["nk"])
        sc = S.abs().max().item() + 1e-30
        assert (S - e["S"]).abs().max().item() <= 1e-6 * sc
    # finalize, then an incremental pass against the single-data-set delta
    sk.sk_batch_kmeans_finalize(br.batch)
    torch.cuda.synchronize()
    ref = []
    for e in br.ds:
        st = dict(mu=e["mu"].clone(), labels=e["labels"].clone(), S=e["S"].clone(),
                  cnt=e["cnt"].clone(), nk=e["nk"].clone())
        sk.sk_kmeans_step_delta(e["ctx"], e["idx"], e["val"], st["mu"], st["labels"], st["S"],
                                st["cnt"], st["nk"])
        ref.append(st)
    sk.sk_batch_kmeans_step(br.batch, incremental=True)
    torch.cuda.synchronize()
    for e, st in zip(br.ds, ref):
        assert torch.equal(st["labels"], e["labels"])
        assert torch.equal(st["cnt"], e["cnt"]) and torch.equal(st["nk"], e["nk"])
    assert sk.sk_device_status() == sk.SK_OK


def test_batch_graph_loop_matches_eager(run):
    sk, br = run
    br.init_centres()
    br.kmeans(6, use_graph=False)
    torch.cuda.synchronize()
    eager = [(e["labels"].clone(), e["mu"].clone()) for e in br.ds]
    br.init_centres()
    br.kmeans(6, use_graph=True)
    torch.cuda.synchronize()
    for e, (l0, m0) in zip(br.ds, eager):
        assert float((e["labels"] == l0).float().mean()) >= 0.999
        assert torch.allclose(e["mu"], m0, rtol=1e-5, atol=1e-6)
        nk = e["nk"].cpu().numpy()
        assert nk.sum() == e["n"]
        assert np.array_equal(e["cnt"].cpu().numpy().sum(axis=1), e["ctx"].m * nk)
    assert sk.sk_device_status() == sk.SK_OK


def test_batch_autotune_keeps_results(run):
    sk, br = run
    br.compress_and_cov()
    torch.cuda.synchronize()
    idx0 = [e["idx"].clone() for e in br.ds]
    G0 = [e["G"].clone() for e in br.ds]
    u, t = br.autotune()
    assert u in (32, 128) and t in (256, 128)
    br.compress_and_cov()
    torch.cuda.synchronize()
    for e, i0, g0 in zip(br.ds, idx0, G0):
        assert torch.equal(e["idx"], i0)
        U0, U1 = torch.triu(g0), torch.triu(e["G"])
        assert (torch.linalg.norm(U1 - U0) / torch.linalg.norm(U0)).item() <= 1e-5
    br.init_centres()
    br.kmeans(3, use_graph=True)
    torch.cuda.synchronize()
    for e in br.ds:
        assert e["nk"].sum().item() == e["n"]
    assert sk.sk_device_status() == sk.SK_OK


def test_single_handle_autotuners():
    from paper_1511_00152_gb300 import _lib as sk
    n, p, m, seed = 20000, 1024, 51, 9
    X, _, _ = synth.mixture_device(n, p, 10, seed)
    ctx = sk.sk_init(p, m, seed)
    idx, val = sk.sk_compress(ctx, X)
    G0 = torch.zeros((ctx.pt, ctx.pt), dtype=torch.float64, device="cuda")
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G0)
    c = sk.sk_autotune_compress(ctx, X, torch.empty_like(idx), torch.empty_like(val))
    assert c in (0, 1)
    tn, sm = sk.sk_autotune_gram(ctx, sk.SK_GRAM_BF16X3, idx, val, torch.empty_like(G0))
    assert tn in (128, 256) and sm in (1, 2)
    idx2, val2 = sk.sk_compress(ctx, X)
    G = torch.zeros_like(G0)
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx2, val2, G)
    torch.cuda.synchronize()
    assert torch.equal(idx, idx2) and torch.equal(val, val2)
    U0, U1 = torch.triu(G0), torch.triu(G)
    assert (torch.linalg.norm(U1 - U0) / torch.linalg.norm(U0)).item() <= 1e-6
    assert sk.sk_device_status() == sk.SK_OK


def test_batch_matches_oracle():
    """Every data set of a split-BF16 batch (ragged p, m, K and n in one
    launch per stage) against the FP64 oracle on its own rows: idx bit-exact,
    val <= 1e-5 ||x_r||; the Gram and C_n to 1e-5 relative Frobenius; the
    first K-means pass from the seeded start against the oracle's assignment
    and sums (counts and sizes exact, centres 1e-5, over the clusters no
    near-tie row touched; tests/kmeans_trace.py)."""
    import kmeans_trace
    import oracle
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import pipeline
    sets = [(2500, 256, 13, 5, 21), (1300, 1000, 51, 10, 22), (700, 4096, 205, 20, 23),
            (333, 2048, 41, 7, 24)]
    ds = []
    for (n, p, m, K, seed) in sets:
        X, _, _ = synth.mixture_device(n, p, min(K, 10), seed)
        ds.append(dict(X=X, m=m, K=K, seed=seed))
    br = pipeline.BatchRun(ds, mode=sk.SK_GRAM_BF16X3)
    br.compress_and_cov()
    br.init_centres()
    sk.sk_batch_kmeans_reset(br.batch)
    sk.sk_batch_kmeans_step(br.batch, incremental=False)
    sk.sk_batch_kmeans_finalize(br.batch)
    torch.cuda.synchronize()
    for e, (n, p, m, K, seed) in zip(br.ds, sets):
        X = e["X"].cpu().numpy()
        oi, ov = oracle.compress(X, m, seed)
        assert np.array_equal(e["idx"].cpu().numpy(), oi)
        nrm = np.linalg.norm(X.astype(np.float64), axis=1)
        assert np.all(np.abs(e["val"].cpu().numpy() - ov).max(axis=1) <= 1e-5 * nrm)
        pt = e["ctx"].pt
        Go = oracle.gram(oi, ov, pt)
        Gg = e["G"].cpu().numpy()
        assert np.linalg.norm(np.triu(Gg) - np.triu(Go)) <= 1e-5 * np.linalg.norm(np.triu(Go))
        C = sk.sk_cov_finalize(e["ctx"], e["G"], n).cpu().numpy()
        Co = oracle.cov_finalize(Go, n, m)
        assert np.linalg.norm(C - Co) <= 1e-5 * np.linalg.norm(Co)
        mu0 = oracle.precondition(e["Xsel"].cpu().numpy(), seed)
        trace = kmeans_trace.oracle_trace(oi, ov, mu0, pt, 1)
        kmeans_trace.check_against_trace([e["labels"].cpu().numpy()], e["mu"].cpu().numpy(),
                                         e["cnt"].cpu().numpy(), e["nk"].cpu().numpy(), trace, K)
    assert sk.sk_device_status() == sk.SK_OK
