"""Streaming request loop: continuous admission, memory budget, and the same
result for a data stream alone and in the mix.  Counts are exact; the Gram
differs only by the order of its FP64 atomic additions (relative 1e-12); the
centre sums S add per-CTA float partials whose within-CTA atomic order varies
(relative 1e-7)."""
import numpy as np
import pytest

from paper_1511_00152_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P, M, K = 2048, 102, 8


def _chunks(stream_id, total_rows, seed):
    rng = np.random.default_rng(seed)
    out, r0 = [], 0
    while r0 < total_rows:
        n = int(min(total_rows - r0, np.exp(rng.uniform(np.log(4096), np.log(16384)))))
        out.append((r0, n))
        r0 += n
    return out


def _requests(serving, stream_seeds, rows):
    reqs = []
    for sid, sseed in enumerate(stream_seeds):
        for (r0, n) in _chunks(sid, rows, sseed):
            reqs.append(serving.Request(
                stream_id=sid, row0=r0, n=n,
                make_x=(lambda s, n=n, r0=r0, sseed=sseed:
                        synth.lowrank_mixture_chunk_device(n, P, sseed, r0))))
    return reqs


def _centres(sk, ctx, sseed):
    X0 = synth.lowrank_mixture_chunk_device(K, P, sseed, 10**9)
    return sk.sk_precondition(ctx, X0)


def _state(st):
    torch.cuda.synchronize()
    return (st.G.cpu().numpy(), st.S.cpu().numpy(), st.cnt.cpu().numpy(), st.nk.cpu().numpy(),
            st.rows)


def test_alone_equals_mix_and_budget_respected():
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import serving
    seeds = [11, 22, 33]
    rows = 60000
    seed = 5
    # alone: one stream at a time through a one-slot server
    alone = {}
    for sid, sseed in enumerate(seeds):
        srv = serving.Server(P, M, seed, slots=1, max_rows=16384, mem_budget_bytes=1 << 30)
        srv.open_stream(sid, _centres(sk, srv.ctx, sseed))
        srv.run([r for r in _requests(serving, seeds, rows) if r.stream_id == sid])
        alone[sid] = _state(srv.streams[sid])
    # in the mix: all streams' chunks interleaved over four slots, with a
    # memory budget that holds at most two chunks in flight
    budget = 2 * 16384 * P * 4
    srv = serving.Server(P, M, seed, slots=4, max_rows=16384, mem_budget_bytes=budget)
    for sid, sseed in enumerate(seeds):
        srv.open_stream(sid, _centres(sk, srv.ctx, sseed))
    reqs = _requests(serving, seeds, rows)
    rng = np.random.default_rng(0)
    for r in reqs:
        r.arrival = float(rng.uniform(0, 1))
    done = srv.run(reqs)
    assert len(done) == len(reqs)
    assert srv.peak_bytes <= budget
    lat = serving.Server.latency_percentiles(done)
    assert lat["p50"] > 0 and lat["p99"] >= lat["p50"]
    for sid in range(len(seeds)):
        Ga, Sa, ca, na, ra = alone[sid]
        Gm, Sm, cm, nm, rm = _state(srv.streams[sid])
        assert ra == rm == rows
        assert np.array_equal(ca, cm) and np.array_equal(na, nm)
        assert na.sum() == rows
        Gu_a, Gu_m = np.triu(Ga), np.triu(Gm)
        assert np.linalg.norm(Gu_a - Gu_m) <= 1e-12 * np.linalg.norm(Gu_a)
        assert np.abs(Sa - Sm).max() <= 1e-7 * np.abs(Sa).max()


def test_stream_equals_one_batch():
    """A stream served in chunks gives the Gram of one call over all its rows
    (up to FP32 partial-sum grouping) and the same counts."""
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import serving
    seed, sseed, rows = 9, 44, 40000
    srv = serving.Server(P, M, seed, slots=3, max_rows=16384, mode=sk.SK_GRAM_BF16X3)
    srv.open_stream(0, _centres(sk, srv.ctx, sseed))
    reqs = [r for r in _requests(serving, [sseed], rows)]
    srv.run(reqs)
    G, S, cnt, nk, _ = _state(srv.streams[0])
    X = torch.cat([synth.lowrank_mixture_chunk_device(n, P, sseed, r0)
                   for (r0, n) in _chunks(0, rows, sseed)])
    ctx = srv.ctx
    idx, val = sk.sk_compress(ctx, X)
    G1 = torch.zeros((ctx.pt, ctx.pt), dtype=torch.float64, device="cuda")
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G1)
    mu = srv.streams[0].mu
    lab, _ = sk.sk_kmeans_assign(ctx, idx, val, mu)
    S1 = torch.zeros_like(srv.streams[0].S)
    c1 = torch.zeros_like(srv.streams[0].cnt)
    n1 = torch.zeros_like(srv.streams[0].nk)
    sk.sk_kmeans_update(ctx, idx, val, lab, K, S1, c1, n1)
    torch.cuda.synchronize()
    Gu, G1u = np.triu(G), np.triu(G1.cpu().numpy())
    assert np.linalg.norm(Gu - G1u) <= 1e-5 * np.linalg.norm(G1u)
    assert np.array_equal(cnt, c1.cpu().numpy()) and np.array_equal(nk, n1.cpu().numpy())
    C = srv.streams[0].covariance()
    assert torch.allclose(C, C.T)


def test_served_stream_matches_oracle():
    """A stream served in the mix (three slots, its chunks interleaved with
    another stream's, uneven chunk sizes and row offsets) against the FP64
    oracle on the same rows: the split-BF16 Gram to 1e-5 relative Frobenius,
    C_n likewise; the K-means sums against the oracle's assignment to the
    stream's centres (counts and sizes exact, S to 1e-5, over the clusters no
    near-tie row touched; tests/kmeans_trace.py)."""
    import kmeans_trace
    import oracle
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import serving
    seed, seeds, rows = 13, [55, 66], 30000
    srv = serving.Server(P, M, seed, slots=3, max_rows=16384, mode=sk.SK_GRAM_BF16X3)
    X0s = {}
    for sid, sseed in enumerate(seeds):
        X0s[sid] = synth.lowrank_mixture_chunk_device(K, P, sseed, 10**9)
        srv.open_stream(sid, sk.sk_precondition(srv.ctx, X0s[sid]))
    reqs = _requests(serving, seeds, rows)
    rng = np.random.default_rng(1)
    lab_g = torch.full((rows,), -1, dtype=torch.int32, device="cuda")
    for r in reqs:
        r.arrival = float(rng.uniform(0, 1))
        if r.stream_id == 0:
            r.labels_out = lab_g[r.row0:r.row0 + r.n]
    srv.run(reqs)
    G, S, cnt, nk, nrows = _state(srv.streams[0])
    assert nrows == rows
    # the oracle's run of stream 0: its chunks' rows (drawn again from the
    # seeded generator), compressed at their global row offsets
    oi_parts, ov_parts = [], []
    for (r0, n) in _chunks(0, rows, seeds[0]):
        Xc = synth.lowrank_mixture_chunk_device(n, P, seeds[0], r0).cpu().numpy()
        ci, cv = oracle.compress(Xc, M, seed, row0=r0)
        oi_parts.append(ci)
        ov_parts.append(cv)
    oi, ov = np.concatenate(oi_parts), np.concatenate(ov_parts)
    pt = srv.ctx.pt
    Go = oracle.gram(oi, ov, pt)
    rel = np.linalg.norm(np.triu(G) - np.triu(Go)) / np.linalg.norm(np.triu(Go))
    assert rel <= 1e-5, rel
    C = srv.streams[0].covariance().cpu().numpy()
    Co = oracle.cov_finalize(Go, rows, M)
    assert np.linalg.norm(C - Co) <= 1e-5 * np.linalg.norm(Co)
    mu_o = oracle.precondition(X0s[0].cpu().numpy(), seed)
    trace = kmeans_trace.oracle_trace(oi, ov, mu_o, pt, 1)
    keep, _ = kmeans_trace.untouched([lab_g.cpu().numpy()], trace, K)
    assert keep.sum() >= K // 2
    assert np.array_equal(cnt[keep], trace["counts"][keep])
    assert np.array_equal(nk[keep], trace["nk"][keep])
    So = np.where(trace["counts"] > 0, trace["mu"] * trace["counts"], 0.0)
    assert np.abs(S[keep] - So[keep]).max() <= 1e-5 * np.abs(So).max()
    assert sk.sk_device_status() == sk.SK_OK
