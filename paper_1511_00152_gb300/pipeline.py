"""Host-side drivers of the paper's algorithms over the C ABI.

Only control flow lives here (loops, buffer management, CUDA-graph capture);
every arithmetic step is a libsk.so kernel reached through ``_lib``.
"""
from __future__ import annotations

import torch

from . import _lib as sk


class KMeansState:
    """Device buffers of one sparsified K-means run (Algorithm 1 loop)."""

    def __init__(self, ctx: sk.Ctx, n: int, K: int, device="cuda", keep_dist: bool = False,
                 mode: str = "auto"):
        self.ctx, self.n, self.K = ctx, n, K
        self.mu = torch.empty((K, ctx.pt), dtype=torch.float32, device=device)
        self.labels = torch.empty(n, dtype=torch.int32, device=device)
        # each row's winning restricted distance, written only when asked for
        self.dist = torch.empty(n, dtype=torch.float32, device=device) if keep_dist else None
        self.S = torch.empty((K, ctx.pt), dtype=torch.float64, device=device)
        self.cnt = torch.empty((K, ctx.pt), dtype=torch.int32, device=device)
        self.nk = torch.empty(K, dtype=torch.int64, device=device)
        self.changed = torch.zeros(1, dtype=torch.int64, device=device)
        # how passes after the first update the sums: "auto" (full rebuild
        # while many labels change, incremental after; chosen on the device),
        # "incremental" or "full"
        self.mode = mode
        self.state = torch.zeros(3, dtype=torch.int64, device=device)
        self.graph = None
        self._graph_args = None

    def iteration(self, idx, val, first: bool = True, stream=None):
        """One assign + update pass (Eqs. (assignments), (mu_update_two)).

        The first pass builds the sums from scratch; later passes rebuild them
        or update them from the rows whose label changed (same sums)."""
        ctx = self.ctx
        if self.mode == "auto":
            sk.sk_kmeans_step_auto(ctx, idx, val, self.mu, self.labels, self.S, self.cnt, self.nk,
                                   self.state, first, dist=self.dist, stream=stream)
        elif first or self.mode == "full":
            sk.sk_kmeans_reset(ctx, self.S, self.cnt, self.nk, stream=stream)
            sk.sk_kmeans_step(ctx, idx, val, self.mu, self.labels, self.S, self.cnt, self.nk,
                              dist=self.dist, stream=stream)
        else:
            sk.sk_kmeans_step_delta(ctx, idx, val, self.mu, self.labels, self.S, self.cnt,
                                    self.nk, dist=self.dist, changed=self.changed, stream=stream)
        sk.sk_kmeans_finalize(ctx, self.S, self.cnt, self.mu, stream=stream)

    def run(self, idx, val, mu0, iters: int, use_graph: bool = True, history=None):
        """iters iterations from the preconditioned-domain centres mu0 (K x pt).

        With use_graph, the loop is captured once as a CUDA graph and replayed
        (the same kernels, one launch for the whole loop).  history (device
        int32 iters x n, optional) receives each iteration's labels."""
        self.mu.copy_(mu0)
        if history is not None and tuple(history.shape) != (iters, self.n):
            raise ValueError("history must be iters x n")
        if not use_graph or iters == 0:
            for it in range(iters):
                self.iteration(idx, val, first=(it == 0))
                if history is not None:
                    history[it].copy_(self.labels)
            return self.labels, self.mu
        key = (idx.data_ptr(), val.data_ptr(), idx.shape[0], iters,
               None if history is None else history.data_ptr())
        if self.graph is None or self._graph_args != key:
            # warm the launch configuration outside capture, then capture
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                saved = self.mu.clone()
                self.iteration(idx, val, first=True, stream=s)
                self.iteration(idx, val, first=False, stream=s)
                self.mu.copy_(saved)
            torch.cuda.current_stream().wait_stream(s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                for it in range(iters):
                    self.iteration(idx, val, first=(it == 0))
                    if history is not None:
                        history[it].copy_(self.labels)
            self.graph, self._graph_args = g, key
            self.mu.copy_(mu0)
        self.graph.replay()
        return self.labels, self.mu


def kmeans_best_of(ctx: sk.Ctx, idx, val, K: int, restarts: int, iters: int,
                   use_graph: bool = True):
    """Sparsified K-means from K-means++ starts, best of `restarts` runs by the
    objective J' (Algorithm 1 with K-means++ seeding; Sec. VII keeps the run
    with the smallest objective).  The seeding, the iterations and J' run in
    the library; the host only compares the R objective values.
    Returns (labels, centres mu' [K x pt], J', best restart)."""
    n = idx.shape[0]
    st = KMeansState(ctx, n, K, device=idx.device, keep_dist=True)
    work = torch.empty(max(256, sk.sk_kmeanspp_workspace_bytes(ctx, n)), dtype=torch.uint8,
                       device=idx.device)
    mu0 = torch.empty((K, ctx.pt), dtype=torch.float32, device=idx.device)
    rows = torch.empty(K, dtype=torch.int64, device=idx.device)
    J = torch.empty(1, dtype=torch.float64, device=idx.device)
    best = None
    for r in range(restarts):
        sk.sk_kmeanspp(ctx, idx, val, K, restart=r, mu=mu0, rows=rows, work=work)
        st.run(idx, val, mu0, iters, use_graph=use_graph)
        # J' at the last assignment (the distances of the final labels)
        sk.sk_kmeans_objective(st.dist, J=J)
        j = float(J.item())
        if best is None or j < best[2]:
            best = (st.labels.clone(), st.mu.clone(), j, r)
    return best


def kmeans_2pass(ctx: sk.Ctx, X, labels1, mu_x, chunk_rows: int | None = None):
    """Second pass of Algorithm 2 over the raw rows X (n x p): labels against
    the un-mixed 1-pass centres mu_x (K x p) and the means of X under the
    1-pass labels.  Returns (labels2, mu2 [K x p], counts [K]).  With
    chunk_rows the pass streams X in row chunks (out-of-core input)."""
    n = X.shape[0]
    K = mu_x.shape[0]
    labels2 = torch.empty(n, dtype=torch.int32, device=X.device)
    sums = torch.zeros((K, ctx.p), dtype=torch.float64, device=X.device)
    counts = torch.zeros(K, dtype=torch.int64, device=X.device)
    step = chunk_rows or max(n, 1)
    for a in range(0, n, step):
        b = min(n, a + step)
        sk.sk_kmeans2_assign(ctx, X[a:b], mu_x, labels=labels2[a:b])
        sk.sk_kmeans2_sums(ctx, X[a:b], labels1[a:b], K, sums, counts)
    mu2 = sk.sk_kmeans2_finalize(ctx, sums, counts, mu_x.clone())
    return labels2, mu2, counts


def sample_mean(ctx: sk.Ctx, idx, val, n_total: int | None = None, sums=None):
    """Sample-mean estimator (Sec. IV) of the ELL rows: (mean in the
    preconditioned domain [pt], mean un-mixed to the data domain [p])."""
    if sums is None:
        sums = torch.zeros(ctx.pt, dtype=torch.float64, device=idx.device)
        sk.sk_mean_accumulate(ctx, idx, val, sums)
    mean = sk.sk_mean_finalize(ctx, sums, n_total or idx.shape[0])
    return mean, sk.sk_unmix(ctx, mean[None, :])[0]


def initial_centres(ctx: sk.Ctx, X, rows) -> torch.Tensor:
    """Preconditioned rows X[rows] (dense y = H D x) as starting centres."""
    sel = X[torch.as_tensor(rows, device=X.device, dtype=torch.long)].contiguous()
    return sk.sk_precondition(ctx, sel)


def covariance(ctx: sk.Ctx, idx, val, mode: int, G=None, C=None, work=None):
    """C_n from one batch of ELL rows (Sec. V)."""
    if G is None:
        G = torch.empty((ctx.pt, ctx.pt), dtype=torch.float64, device=idx.device)
    sk.sk_cov_reset(ctx, G)
    sk.sk_cov_accumulate(ctx, mode, idx, val, G, work=work)
    return sk.sk_cov_finalize(ctx, G, idx.shape[0], C=C)


def covariance_centred(ctx: sk.Ctx, idx, val, mode: int, G=None, C=None, work=None):
    """Centred covariance estimate of one batch of ELL rows: C_n (Sec. V) and
    the sample mean (Sec. IV) of the same rows, combined with the correction
    that makes C_n - xbar xbar^T unbiased.  Returns (C, mean)."""
    n = idx.shape[0]
    if G is None:
        G = torch.empty((ctx.pt, ctx.pt), dtype=torch.float64, device=idx.device)
    sk.sk_cov_reset(ctx, G)
    sk.sk_cov_accumulate(ctx, mode, idx, val, G, work=work)
    sums = torch.zeros(ctx.pt, dtype=torch.float64, device=idx.device)
    sk.sk_mean_accumulate(ctx, idx, val, sums)
    mean = sk.sk_mean_finalize(ctx, sums, n)
    return sk.sk_cov_finalize_centred(ctx, G, mean, n, C=C), mean


class HostStreamer:
    """Compress host rows and add them to the Gram while they stream to the
    device (Algorithm 1's one pass over X, Sec. V's G = sum of w w^T).

    Xh is pinned host memory (n x p float32).  The rows go to the device in
    chunks on a copy stream, into a ring of `nbuf` device chunk buffers; the
    caller's stream compresses each chunk into its rows of the ELL output and
    adds it to G as soon as it has landed, so the copy of the next chunks
    overlaps this work.  The masks are keyed by the global row number (row0 of
    each chunk), so idx / val are those of one sk_compress call over all n
    rows; G equals the one-call Gram up to float64 summation order.

    Stream order: the compute of chunk c waits for the copy of chunk c; the
    copy into a ring buffer waits for the compute of the chunk that used it
    before, in this call or an earlier one (so a call may be enqueued while
    the previous one still runs: its first copies then overlap the caller's
    work that follows the previous call).  Each wait is issued after the
    record it waits for and before that event is recorded again, so no wait
    depends on work queued after it.
    """

    def __init__(self, ctx: sk.Ctx, chunk_rows: int, mode: int, nbuf: int = 3,
                 device="cuda"):
        if chunk_rows < 1 or nbuf < 1:
            raise ValueError("chunk_rows and nbuf must be positive")
        self.ctx, self.mode, self.chunk = ctx, mode, int(chunk_rows)
        self.bufs = [torch.empty((self.chunk, ctx.p), dtype=torch.float32, device=device)
                     for _ in range(nbuf)]
        self.copy_stream = torch.cuda.Stream(device=device)
        self.copied = [torch.cuda.Event() for _ in range(nbuf)]
        self.used = [torch.cuda.Event() for _ in range(nbuf)]
        self.used_recorded = [False] * nbuf
        need = sk.sk_cov_workspace_bytes(ctx, mode, self.chunk)
        self.work = torch.empty(max(1, need), dtype=torch.uint8, device=device)

    def run(self, Xh, idx, val, G, reset: bool = True):
        """Streams Xh through compress and the Gram update; returns G."""
        if Xh.is_cuda or not Xh.is_pinned():
            raise ValueError("Xh must be pinned host memory")
        n = Xh.shape[0]
        stream = torch.cuda.current_stream()
        nb, ch = len(self.bufs), self.chunk
        nch = (n + ch - 1) // ch
        if reset:
            sk.sk_cov_reset(self.ctx, G)

        def issue(c):
            r0, r1, b = c * ch, min(n, (c + 1) * ch), c % nb
            with torch.cuda.stream(self.copy_stream):
                if self.used_recorded[b]:
                    self.copy_stream.wait_event(self.used[b])
                self.bufs[b][: r1 - r0].copy_(Xh[r0:r1], non_blocking=True)
                self.copied[b].record(self.copy_stream)

        for c in range(min(nb, nch)):
            issue(c)
        for c in range(nch):
            r0, r1, b = c * ch, min(n, (c + 1) * ch), c % nb
            stream.wait_event(self.copied[b])
            sk.sk_compress(self.ctx, self.bufs[b][: r1 - r0], row0=r0, idx=idx[r0:r1],
                           val=val[r0:r1])
            sk.sk_cov_accumulate(self.ctx, self.mode, idx[r0:r1], val[r0:r1], G, work=self.work)
            self.used[b].record(stream)
            self.used_recorded[b] = True
            if c + nb < nch:
                issue(c + nb)
        return G


def pca(ctx: sk.Ctx, C, k: int, iters: int = 40):
    """Top-k eigenpairs of C_n and the eigenvectors un-mixed to the data domain
    (U = (HD)^T U', Sec. V).  Returns (evals, U' [k x pt], U [k x p])."""
    evals, Up = sk.sk_cov_topk(ctx, C, k, iters)
    return evals, Up, sk.sk_unmix(ctx, Up)


class BatchRun:
    """Many independent data sets through the hot path with one launch per
    stage (sk_batch_*): compress, Gram, and each K-means pass cover every data
    set; the K-means loop is captured once as a CUDA graph.

    datasets: list of dicts with X (device n x p float32), m, K, seed (and
    optionally flags).  Buffers are allocated here with torch."""

    def __init__(self, datasets, mode: int = sk.SK_GRAM_BF16, device="cuda"):
        self.mode = mode
        self.ds = []
        items = []
        for d in datasets:
            X = d["X"]
            n, p = X.shape
            ctx = sk.sk_init_ex(p, d["m"], d["seed"], d.get("flags", 0))
            pt, m, K = ctx.pt, ctx.m, d["K"]
            e = dict(ctx=ctx, X=X, n=n, K=K, seed=d["seed"])
            e["idx"] = torch.empty((n, m), dtype=torch.int32, device=device)
            e["val"] = torch.empty((n, m), dtype=torch.float32, device=device)
            e["G"] = torch.empty((pt, pt), dtype=torch.float64, device=device)
            wb = sk.sk_cov_workspace_bytes(ctx, mode, n)
            e["work"] = torch.empty(max(wb, 256), dtype=torch.uint8, device=device)
            e["mu"] = torch.empty((K, pt), dtype=torch.float32, device=device)
            # transposed centres (used when the table does not fit shared memory)
            e["mu_t"] = torch.empty((pt, 2 * ((K + 1) // 2)), dtype=torch.float32, device=device)
            e["labels"] = torch.empty(n, dtype=torch.int32, device=device)
            e["S"] = torch.empty((K, pt), dtype=torch.float64, device=device)
            e["cnt"] = torch.empty((K, pt), dtype=torch.int32, device=device)
            e["nk"] = torch.empty(K, dtype=torch.int64, device=device)
            e["changed"] = torch.zeros(1, dtype=torch.int64, device=device)
            # the seeded start rows, selected once (input preparation)
            rows = torch.as_tensor(synth_init_rows(n, K, d["seed"]), device=device)
            e["Xsel"] = X.index_select(0, rows).contiguous()
            self.ds.append(e)
            items.append(sk.SkBatchItem(
                p=p, m=m, seed=int(d["seed"]) & (2**64 - 1), flags=d.get("flags", 0),
                X=X.data_ptr(), n=n, ldx=X.stride(0) if n > 1 else p, row0=0,
                idx=e["idx"].data_ptr(), val=e["val"].data_ptr(), G=e["G"].data_ptr(),
                gram_work=e["work"].data_ptr(), gram_work_bytes=e["work"].numel(), K=K,
                mu=e["mu"].data_ptr(), mu_t=e["mu_t"].data_ptr(), labels=e["labels"].data_ptr(),
                S=e["S"].data_ptr(),
                cnt=e["cnt"].data_ptr(), nk=e["nk"].data_ptr(), changed=e["changed"].data_ptr()))
        self.batch = sk.sk_batch_create(items, mode, keep=self.ds)
        self.table = torch.empty(max(256, sk.sk_batch_workspace_bytes(self.batch)),
                                 dtype=torch.uint8, device=device)
        sk.sk_batch_upload(self.batch, self.table)
        self.graph = None
        self._graph_iters = None

    def autotune(self):
        """Library autotuner: compress task size and Gram tile width for this
        batch (runs both stages once; call before capture)."""
        self.tuning = sk.sk_batch_autotune(self.batch, self.table)
        self.graph = None  # the plan's tables moved: recapture
        return self.tuning

    def compress_and_cov(self, stream=None):
        """Compress every data set, then its Gram (one launch each stage)."""
        sk.sk_batch_compress(self.batch, stream=stream)
        sk.sk_batch_cov_reset(self.batch, stream=stream)
        sk.sk_batch_cov_accumulate(self.batch, stream=stream)

    def init_centres(self, stream=None):
        """Seeded start: the preconditioned K seeded rows of each data set."""
        for e in self.ds:
            sk.sk_precondition(e["ctx"], e["Xsel"], Y=e["mu"], stream=stream)

    def _loop(self, iters, stream=None):
        sk.sk_batch_kmeans_reset(self.batch, stream=stream)
        for it in range(iters):
            sk.sk_batch_kmeans_step(self.batch, incremental=it > 0, stream=stream)
            sk.sk_batch_kmeans_finalize(self.batch, stream=stream)

    def kmeans(self, iters: int, use_graph: bool = True):
        """iters passes over every data set from the current centres."""
        if not use_graph:
            self._loop(iters)
            return
        if self.graph is None or self._graph_iters != iters:
            saved = [e["mu"].clone() for e in self.ds]
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                self._loop(min(iters, 2), stream=s)
            torch.cuda.current_stream().wait_stream(s)
            for e, m0 in zip(self.ds, saved):
                e["mu"].copy_(m0)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._loop(iters)
            self.graph, self._graph_iters = g, iters
        self.graph.replay()


def synth_init_rows(n, K, seed):
    from . import synth
    return synth.init_rows(n, K, seed)
