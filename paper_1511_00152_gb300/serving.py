"""Streaming request loop with continuous admission (the paper's one-pass,
out-of-core setting, Sec. VII "Out-of-core", as a serving loop).

A *data stream* is one logical data set that arrives in row chunks of uneven
size.  Its state stays resident on the device: the running Gram G (for C_n,
Sec. V) and the K-means sums S, cnt, n_k of Eq. (mu_update_one) against the
stream's centres.  Because masks are keyed by the global row (row0 + i), a
chunk's contribution does not depend on which other chunks ran before, after
or at the same time -- only on floating-point summation order.

A *request* is one chunk of one stream.  The server keeps a fixed number of
slots (each with its own CUDA stream and ELL/workspace buffers sized for the
largest chunk).  Requests that arrive while others are on the GPU are admitted
as soon as a slot is free and the bytes of in-flight chunks stay within the
memory budget; admitted requests run concurrently on their slots' streams.
Latency is measured per request from arrival to completion with CUDA events.

Everything here is control flow; the arithmetic is libsk.so's kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import torch

from . import _lib as sk


@dataclasses.dataclass
class Request:
    stream_id: int
    row0: int                 # global index of the chunk's first row in its stream
    n: int                    # rows in the chunk
    make_x: object = None     # callable(torch.cuda.Stream) -> device tensor n x p (generated)
    x: object = None          # or a device / pinned host tensor n x p
    arrival: float = 0.0      # seconds, relative to the start of run()
    labels_out: object = None  # optional device int32 tensor (n): the rows' K-means labels
    # filled by the server
    admitted: float = -1.0
    done_event: object = None
    start_event: object = None
    latency_ms: float = -1.0
    bytes: int = 0


class StreamState:
    """Device-resident running sums of one data stream."""

    def __init__(self, ctx: sk.Ctx, mu: torch.Tensor, mode: int):
        dev = mu.device
        self.ctx, self.mode = ctx, mode
        self.K = mu.shape[0]
        self.mu = mu.contiguous()
        self.G = torch.empty((ctx.pt, ctx.pt), dtype=torch.float64, device=dev)
        self.S = torch.empty((self.K, ctx.pt), dtype=torch.float64, device=dev)
        self.cnt = torch.empty((self.K, ctx.pt), dtype=torch.int32, device=dev)
        self.nk = torch.empty(self.K, dtype=torch.int64, device=dev)
        sk.sk_cov_reset(ctx, self.G)
        sk.sk_kmeans_reset(ctx, self.S, self.cnt, self.nk)
        self.rows = 0

    def covariance(self):
        """C_n of every row seen so far (Sec. V)."""
        return sk.sk_cov_finalize(self.ctx, self.G, self.rows)

    def centres(self):
        """One-pass centre update mu'_kj = S/cnt (Eq. (mu_update_two)), un-mixed."""
        mu = self.mu.clone()
        sk.sk_kmeans_finalize(self.ctx, self.S, self.cnt, mu)
        return mu, sk.sk_unmix(self.ctx, mu)


class _Slot:
    def __init__(self, ctx: sk.Ctx, max_rows: int, mode: int, device):
        self.stream = torch.cuda.Stream(device=device)
        m = ctx.m
        self.idx = torch.empty((max_rows, m), dtype=torch.int32, device=device)
        self.val = torch.empty((max_rows, m), dtype=torch.float32, device=device)
        self.labels = torch.empty(max_rows, dtype=torch.int32, device=device)
        wb = sk.sk_cov_workspace_bytes(ctx, mode, max_rows)
        self.work = torch.empty(max(wb, 1), dtype=torch.uint8, device=device)
        self.req = None
        self.x = None


class Server:
    """Continuous-admission request loop over a fixed set of slots."""

    def __init__(self, p: int, m: int, seed: int, slots: int = 4, max_rows: int = 65536,
                 mem_budget_bytes: int = 8 << 30, mode: int = sk.SK_GRAM_BF16,
                 device="cuda"):
        self.ctx = sk.sk_init(p, m, seed)
        self.p, self.m, self.mode = p, m, mode
        self.device = torch.device(device)
        self.max_rows = max_rows
        self.budget = int(mem_budget_bytes)
        self.slots = [_Slot(self.ctx, max_rows, mode, self.device) for _ in range(slots)]
        self.streams: dict[int, StreamState] = {}
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.completed: list[Request] = []

    def request_bytes(self, n: int) -> int:
        """Device bytes a chunk of n rows holds while in flight (its X)."""
        return n * self.p * 4

    def open_stream(self, stream_id: int, mu: torch.Tensor) -> StreamState:
        st = StreamState(self.ctx, mu, self.mode)
        self.streams[stream_id] = st
        return st

    # ---------------------------------------------------------------- work
    def _launch(self, slot: _Slot, req: Request):
        st = self.streams[req.stream_id]
        s = slot.stream
        n = req.n
        with torch.cuda.stream(s):
            req.start_event = torch.cuda.Event(enable_timing=True)
            req.start_event.record(s)
            if req.make_x is not None:
                x = req.make_x(s)
            elif req.x.is_cuda:
                x = req.x
            else:
                x = req.x.to(self.device, non_blocking=True)
            slot.x = x
            idx, val = slot.idx[:n], slot.val[:n]
            sk.sk_compress(self.ctx, x, row0=req.row0, idx=idx, val=val, stream=s)
            sk.sk_cov_accumulate(self.ctx, self.mode, idx, val, st.G, work=slot.work, stream=s)
            labels = slot.labels[:n] if req.labels_out is None else req.labels_out
            sk.sk_kmeans_assign(self.ctx, idx, val, st.mu, labels=labels, stream=s)
            sk.sk_kmeans_update(self.ctx, idx, val, labels, st.K, st.S, st.cnt, st.nk,
                                stream=s)
            req.done_event = torch.cuda.Event(enable_timing=True)
            req.done_event.record(s)
        st.rows += n
        slot.req = req

    def run(self, requests, realtime: bool = False):
        """Serve the requests (sorted by arrival).  With realtime, a request is
        not admitted before its arrival time and its latency_ms runs from its
        arrival (queueing included) to the end of its device work.  Otherwise
        arrivals only order the queue and latency_ms is the request's device
        time alone (start to end of its work on its slot's stream).  Returns
        the completed requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in pending:
            r.bytes = self.request_bytes(r.n)
            if r.n > self.max_rows:
                raise ValueError(f"chunk of {r.n} rows exceeds the slot size {self.max_rows}")
            if r.bytes > self.budget:
                raise ValueError("chunk larger than the memory budget")
        # stream states were reset on the caller's stream; slots start after that
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_arrival = {}
        active = 0
        while pending or active:
            now = time.perf_counter() - t0
            progressed = False
            # retire finished work (non-blocking)
            for slot in self.slots:
                r = slot.req
                if r is not None and r.done_event.query():
                    progressed = True
                    r.latency_ms = r.start_event.elapsed_time(r.done_event) + \
                        max(0.0, (r.admitted - host_arrival[id(r)]) * 1e3)
                    self.in_flight_bytes -= r.bytes
                    slot.req, slot.x = None, None
                    self.completed.append(r)
                    active -= 1
            # admit as slots and memory free up
            for slot in self.slots:
                if slot.req is not None or not pending:
                    continue
                r = pending[0]
                if realtime and r.arrival > now:
                    break
                if self.in_flight_bytes + r.bytes > self.budget:
                    break
                pending.popleft()
                host_arrival[id(r)] = r.arrival if realtime else now
                r.admitted = now
                self.in_flight_bytes += r.bytes
                self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
                self._launch(slot, r)
                active += 1
                progressed = True
            if not progressed:
                # nothing retired or admitted (all slots busy, the next request
                # not yet arrived, or the budget full): yield before polling again
                time.sleep(0 if active else 1e-4)
        torch.cuda.synchronize()
        return self.completed

    @staticmethod
    def latency_percentiles(reqs, qs=(50, 99)):
        import numpy as np
        lat = np.array([r.latency_ms for r in reqs], dtype=np.float64)
        return {f"p{q}": float(np.percentile(lat, q)) for q in qs}
