"""Thin ctypes binding of libsk.so (include/sk.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Tensors are
torch CUDA tensors (PyTorch provides the device memory and the stream);
outputs the caller does not pass are allocated with torch.  All arithmetic
runs in the library's CUDA kernels.  There is no fallback: if libsk.so is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsk.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sk.h")

SK_OK, SK_EINVAL, SK_ENOMEM, SK_ECUDA, SK_ETIMEOUT, SK_EUNSUPPORTED = range(6)
SK_GRAM_FP32, SK_GRAM_BF16, SK_GRAM_BF16X3 = 0, 1, 2
SK_FLAG_NO_PRECONDITION = 1
SK_FLAG_DCT = 2
STATUS_NAMES = {0: "SK_OK", 1: "SK_EINVAL", 2: "SK_ENOMEM", 3: "SK_ECUDA",
                4: "SK_ETIMEOUT", 5: "SK_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class SkError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libsk.so (building it first only if explicitly asked by build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libsk.so not built at {p}; run paper_1511_00152_gb300.build.build()")
        lib = ctypes.CDLL(p)
        i64, i32, u64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p
        st = ctypes.c_int
        sigs = {
            "sk_init": (st, [ctypes.POINTER(vp), i64, i64, u64]),
            "sk_init_ex": (st, [ctypes.POINTER(vp), i64, i64, u64, ctypes.c_uint32]),
            "sk_flags": (ctypes.c_uint32, [vp]),
            "sk_destroy": (None, [vp]),
            "sk_ptilde": (i64, [vp]),
            "sk_compress": (st, [vp, vp, i64, i64, i64, vp, vp, vp]),
            "sk_precondition": (st, [vp, vp, i64, i64, vp, vp]),
            "sk_cov_accumulate": (st, [vp, ctypes.c_int, vp, vp, i64, vp, vp, i64, vp]),
            "sk_cov_workspace_bytes": (i64, [vp, ctypes.c_int, i64]),
            "sk_cov_finalize": (st, [vp, vp, i64, vp, vp]),
            "sk_cov_reset": (st, [vp, vp, vp]),
            "sk_cov_finalize_centred": (st, [vp, vp, vp, i64, vp, vp]),
            "sk_kmeans_reset": (st, [vp, i32, vp, vp, vp, vp]),
            "sk_cov_topk": (st, [vp, vp, i32, i32, vp, vp, vp, vp]),
            "sk_cov_topk_workspace": (i64, [i64, i32]),
            "sk_cov_topk_static": (st, [vp, vp, i32, i32, vp, vp, vp]),
            "sk_kmeans_assign": (st, [vp, vp, vp, i64, vp, i32, vp, vp, vp]),
            "sk_kmeans_update": (st, [vp, vp, vp, vp, i64, i32, vp, vp, vp, vp]),
            "sk_kmeans_step": (st, [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp]),
            "sk_kmeans_step_delta": (st, [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp, vp]),
            "sk_kmeans_step_auto": (st, [vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp, i32,
                                         vp]),
            "sk_kmeans_finalize": (st, [vp, i32, vp, vp, vp, vp]),
            "sk_unmix": (st, [vp, vp, i64, vp, vp]),
            "sk_unmix_f64": (st, [vp, vp, i64, vp, vp]),
            "sk_kmeans2_assign": (st, [vp, vp, i64, i64, vp, i32, vp, vp, vp]),
            "sk_kmeans2_sums": (st, [vp, vp, i64, i64, vp, i32, vp, vp, vp]),
            "sk_kmeans2_finalize": (st, [vp, i32, vp, vp, vp, vp]),
            "sk_mean_accumulate": (st, [vp, vp, vp, i64, vp, vp]),
            "sk_kmeanspp": (st, [vp, vp, vp, i64, i32, ctypes.c_uint32, vp, vp, vp, i64, vp]),
            "sk_kmeanspp_workspace_bytes": (i64, [vp, i64]),
            "sk_kmeans_objective": (st, [vp, i64, vp, vp]),
            "sk_kmeans_hk": (st, [vp, i32, vp, vp, vp, vp]),
            "sk_mean_finalize": (st, [vp, vp, i64, vp, vp]),
            "sk_batch_create": (st, [ctypes.POINTER(vp), vp, i32, i32]),
            "sk_batch_workspace_bytes": (i64, [vp]),
            "sk_batch_upload": (st, [vp, vp, i64, vp]),
            "sk_batch_compress": (st, [vp, vp]),
            "sk_batch_cov_reset": (st, [vp, vp]),
            "sk_batch_cov_accumulate": (st, [vp, vp]),
            "sk_batch_kmeans_reset": (st, [vp, vp]),
            "sk_batch_kmeans_step": (st, [vp, i32, vp]),
            "sk_batch_kmeans_finalize": (st, [vp, vp]),
            "sk_batch_destroy": (None, [vp]),
            "sk_batch_autotune": (st, [vp, vp, i64, vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "sk_autotune_gram": (st, [vp, ctypes.c_int, vp, vp, i64, vp, vp, i64, vp,
                                      ctypes.POINTER(i32), ctypes.POINTER(i32)]),
            "sk_autotune_compress": (st, [vp, vp, i64, i64, vp, vp, vp, ctypes.POINTER(i32)]),
            "sk_device_status": (st, [vp]),
            "sk_debug_set_wait_cycles": (st, [i64]),
            "sk_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def header_symbols() -> list[str]:
    """Names of the entry points declared in include/sk.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sk_[a-z0-9_]+)\s*\(", text)))


def _check(fn: str, status: int):
    if status != SK_OK:
        msg = load().sk_last_error()
        raise SkError(fn, status, msg.decode() if msg else "")


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t, dtype, name, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() and t.dim() != 2:
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Ctx:
    """Owns an sk_ctx* (host memory only)."""

    def __init__(self, handle: int, p: int, m: int, seed: int):
        self._h = ctypes.c_void_p(handle)
        self.p, self.m, self.seed = p, m, seed
        self.pt = int(load().sk_ptilde(self._h))
        self.flags = int(load().sk_flags(self._h))

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.sk_destroy(self._h)
                self._h = ctypes.c_void_p(0)
        except Exception:
            pass


def sk_init(p: int, m: int, seed: int) -> Ctx:
    h = ctypes.c_void_p(0)
    _check("sk_init", load().sk_init(ctypes.byref(h), int(p), int(m), int(seed) & (2**64 - 1)))
    return Ctx(h.value, int(p), int(m), int(seed))


def sk_init_ex(p: int, m: int, seed: int, flags: int) -> Ctx:
    h = ctypes.c_void_p(0)
    _check("sk_init_ex", load().sk_init_ex(ctypes.byref(h), int(p), int(m),
                                           int(seed) & (2**64 - 1), int(flags)))
    return Ctx(h.value, int(p), int(m), int(seed))


def sk_flags(ctx: Ctx) -> int:
    return int(load().sk_flags(ctx.handle))


def sk_ptilde(ctx: Ctx) -> int:
    return int(load().sk_ptilde(ctx.handle))


def _rows_ld(X, p):
    _need(X, torch.float32, "X")
    if X.dim() != 2 or X.shape[1] != p or X.stride(1) != 1:
        raise ValueError("X must be n x p with unit column stride")
    return X.shape[0], X.stride(0) if X.shape[0] > 1 else p


def sk_compress(ctx: Ctx, X, row0: int = 0, idx=None, val=None, stream=None):
    n, ldx = _rows_ld(X, ctx.p)
    dev = X.device
    if idx is None:
        idx = torch.empty((n, ctx.m), dtype=torch.int32, device=dev)
    if val is None:
        val = torch.empty((n, ctx.m), dtype=torch.float32, device=dev)
    _need(idx, torch.int32, "idx", (n, ctx.m))
    _need(val, torch.float32, "val", (n, ctx.m))
    _check("sk_compress", load().sk_compress(ctx.handle, _ptr(X), n, ldx, int(row0), _ptr(idx),
                                             _ptr(val), _stream(stream)))
    return idx, val


def sk_precondition(ctx: Ctx, X, Y=None, stream=None):
    n, ldx = _rows_ld(X, ctx.p)
    if Y is None:
        Y = torch.empty((n, ctx.pt), dtype=torch.float32, device=X.device)
    _need(Y, torch.float32, "Y", (n, ctx.pt))
    _check("sk_precondition", load().sk_precondition(ctx.handle, _ptr(X), n, ldx, _ptr(Y),
                                                     _stream(stream)))
    return Y


def sk_cov_workspace_bytes(ctx: Ctx, mode: int, n: int) -> int:
    return int(load().sk_cov_workspace_bytes(ctx.handle, int(mode), int(n)))


def sk_cov_accumulate(ctx: Ctx, mode: int, idx, val, G, work=None, stream=None):
    """G += sum of w w^T; `work` (uint8 CUDA tensor) is allocated if not given."""
    n = idx.shape[0]
    _need(idx, torch.int32, "idx", (n, ctx.m))
    _need(val, torch.float32, "val", (n, ctx.m))
    _need(G, torch.float64, "G", (ctx.pt, ctx.pt))
    need = sk_cov_workspace_bytes(ctx, mode, n)
    if work is None and need > 0:
        work = torch.empty(need, dtype=torch.uint8, device=idx.device)
    wbytes = 0 if work is None else work.numel() * work.element_size()
    _check("sk_cov_accumulate", load().sk_cov_accumulate(ctx.handle, int(mode), _ptr(idx),
                                                         _ptr(val), n, _ptr(G), _ptr(work),
                                                         wbytes, _stream(stream)))
    return G


def sk_cov_reset(ctx: Ctx, G, stream=None):
    _need(G, torch.float64, "G", (ctx.pt, ctx.pt))
    _check("sk_cov_reset", load().sk_cov_reset(ctx.handle, _ptr(G), _stream(stream)))
    return G


def sk_kmeans_reset(ctx: Ctx, S, cnt, nk, stream=None):
    K = nk.shape[0]
    _need(S, torch.float64, "S", (K, ctx.pt))
    _need(cnt, torch.int32, "cnt", (K, ctx.pt))
    _need(nk, torch.int64, "nk", (K,))
    _check("sk_kmeans_reset", load().sk_kmeans_reset(ctx.handle, K, _ptr(S), _ptr(cnt), _ptr(nk),
                                                     _stream(stream)))
    return S, cnt, nk


def sk_cov_finalize(ctx: Ctx, G, n_total: int, C=None, stream=None):
    _need(G, torch.float64, "G", (ctx.pt, ctx.pt))
    if C is None:
        C = torch.empty_like(G)
    _need(C, torch.float64, "C", (ctx.pt, ctx.pt))
    _check("sk_cov_finalize", load().sk_cov_finalize(ctx.handle, _ptr(G), int(n_total), _ptr(C),
                                                     _stream(stream)))
    return C


def sk_cov_finalize_centred(ctx: Ctx, G, mean, n_total: int, C=None, stream=None):
    """Centred estimate C_n - xbar xbar^T + B(C_n)/n from G and the sample mean."""
    _need(G, torch.float64, "G", (ctx.pt, ctx.pt))
    _need(mean, torch.float64, "mean", (ctx.pt,))
    if C is None:
        C = torch.empty_like(G)
    _need(C, torch.float64, "C", (ctx.pt, ctx.pt))
    _check("sk_cov_finalize_centred",
           load().sk_cov_finalize_centred(ctx.handle, _ptr(G), _ptr(mean), int(n_total), _ptr(C),
                                          _stream(stream)))
    return C


def sk_cov_topk_workspace(pt: int, k: int) -> int:
    return int(load().sk_cov_topk_workspace(int(pt), int(k)))


def sk_cov_topk(ctx: Ctx, C, k: int, iters: int = 40, evals=None, U=None, work=None,
                stream=None):
    """Returns (evals descending [k], U [k, pt] with row c the c-th eigenvector)."""
    _need(C, torch.float64, "C", (ctx.pt, ctx.pt))
    dev = C.device
    if evals is None:
        evals = torch.empty(k, dtype=torch.float64, device=dev)
    if U is None:
        U = torch.empty((k, ctx.pt), dtype=torch.float64, device=dev)
    if work is None:
        ws = sk_cov_topk_workspace(ctx.pt, k)
        if ws < 0:
            raise SkError("sk_cov_topk_workspace", SK_EINVAL, "bad k")
        work = torch.empty(ws, dtype=torch.float64, device=dev)
    _check("sk_cov_topk", load().sk_cov_topk(ctx.handle, _ptr(C), int(k), int(iters), _ptr(evals),
                                             _ptr(U), _ptr(work), _stream(stream)))
    return evals, U


def sk_kmeans_assign(ctx: Ctx, idx, val, mu, labels=None, dist=None, stream=None):
    n = idx.shape[0]
    K = mu.shape[0]
    _need(mu, torch.float32, "mu", (K, ctx.pt))
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=idx.device)
    _check("sk_kmeans_assign", load().sk_kmeans_assign(ctx.handle, _ptr(idx), _ptr(val), n,
                                                       _ptr(mu), K, _ptr(labels), _ptr(dist),
                                                       _stream(stream)))
    return labels, dist


def sk_kmeans_update(ctx: Ctx, idx, val, labels, K: int, S, cnt, nk, stream=None):
    n = idx.shape[0]
    _need(S, torch.float64, "S", (K, ctx.pt))
    _need(cnt, torch.int32, "cnt", (K, ctx.pt))
    _need(nk, torch.int64, "nk", (K,))
    _check("sk_kmeans_update", load().sk_kmeans_update(ctx.handle, _ptr(idx), _ptr(val),
                                                       _ptr(labels), n, int(K), _ptr(S),
                                                       _ptr(cnt), _ptr(nk), _stream(stream)))
    return S, cnt, nk


def sk_kmeans_step(ctx: Ctx, idx, val, mu, labels, S, cnt, nk, dist=None, stream=None):
    n = idx.shape[0]
    K = mu.shape[0]
    _check("sk_kmeans_step", load().sk_kmeans_step(ctx.handle, _ptr(idx), _ptr(val), n, _ptr(mu),
                                                   K, _ptr(labels), _ptr(dist), _ptr(S),
                                                   _ptr(cnt), _ptr(nk), _stream(stream)))
    return labels


def sk_kmeans_step_delta(ctx: Ctx, idx, val, mu, labels, S, cnt, nk, dist=None, changed=None,
                         stream=None):
    n = idx.shape[0]
    K = mu.shape[0]
    _check("sk_kmeans_step_delta", load().sk_kmeans_step_delta(
        ctx.handle, _ptr(idx), _ptr(val), n, _ptr(mu), K, _ptr(labels), _ptr(dist), _ptr(S),
        _ptr(cnt), _ptr(nk), _ptr(changed), _stream(stream)))
    return labels


def sk_kmeans_step_auto(ctx: Ctx, idx, val, mu, labels, S, cnt, nk, state, first: bool,
                        dist=None, stream=None):
    n = idx.shape[0]
    K = mu.shape[0]
    _need(state, torch.int64, "state", (3,))
    _check("sk_kmeans_step_auto", load().sk_kmeans_step_auto(
        ctx.handle, _ptr(idx), _ptr(val), n, _ptr(mu), K, _ptr(labels), _ptr(dist), _ptr(S),
        _ptr(cnt), _ptr(nk), _ptr(state), 1 if first else 0, _stream(stream)))
    return labels


def sk_kmeans_finalize(ctx: Ctx, S, cnt, mu, stream=None):
    K = mu.shape[0]
    _need(mu, torch.float32, "mu", (K, ctx.pt))
    _check("sk_kmeans_finalize", load().sk_kmeans_finalize(ctx.handle, K, _ptr(S), _ptr(cnt),
                                                           _ptr(mu), _stream(stream)))
    return mu


def sk_unmix(ctx: Ctx, M, out=None, stream=None):
    r = M.shape[0]
    if M.dtype == torch.float64:
        if out is None:
            out = torch.empty((r, ctx.p), dtype=torch.float64, device=M.device)
        _check("sk_unmix_f64", load().sk_unmix_f64(ctx.handle, _ptr(M), r, _ptr(out),
                                                   _stream(stream)))
        return out
    _need(M, torch.float32, "in", (r, ctx.pt))
    if out is None:
        out = torch.empty((r, ctx.p), dtype=torch.float32, device=M.device)
    _check("sk_unmix", load().sk_unmix(ctx.handle, _ptr(M), r, _ptr(out), _stream(stream)))
    return out


def sk_kmeans2_assign(ctx: Ctx, X, mu, labels=None, dist=None, stream=None):
    """Algorithm 2: labels of the raw rows against the un-mixed centres mu (K x p)."""
    n, ldx = _rows_ld(X, ctx.p)
    K = mu.shape[0]
    _need(mu, torch.float32, "mu", (K, ctx.p))
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device=X.device)
    _need(labels, torch.int32, "labels", (n,))
    if dist is not None:
        _need(dist, torch.float32, "dist", (n,))
    _check("sk_kmeans2_assign", load().sk_kmeans2_assign(ctx.handle, _ptr(X), n, ldx, _ptr(mu),
                                                         K, _ptr(labels), _ptr(dist),
                                                         _stream(stream)))
    return labels, dist


def sk_kmeans2_sums(ctx: Ctx, X, labels1, K: int, sums, counts, stream=None):
    """Algorithm 2: sums (K x p float64) and counts (K int64) under the 1-pass labels."""
    n, ldx = _rows_ld(X, ctx.p)
    _need(labels1, torch.int32, "labels1", (n,))
    _need(sums, torch.float64, "sums", (K, ctx.p))
    _need(counts, torch.int64, "counts", (K,))
    _check("sk_kmeans2_sums", load().sk_kmeans2_sums(ctx.handle, _ptr(X), n, ldx, _ptr(labels1),
                                                     int(K), _ptr(sums), _ptr(counts),
                                                     _stream(stream)))
    return sums, counts


def sk_kmeans2_finalize(ctx: Ctx, sums, counts, mu, stream=None):
    K = mu.shape[0]
    _need(mu, torch.float32, "mu", (K, ctx.p))
    _need(sums, torch.float64, "sums", (K, ctx.p))
    _need(counts, torch.int64, "counts", (K,))
    _check("sk_kmeans2_finalize", load().sk_kmeans2_finalize(ctx.handle, K, _ptr(sums),
                                                             _ptr(counts), _ptr(mu),
                                                             _stream(stream)))
    return mu


def sk_kmeanspp_workspace_bytes(ctx: Ctx, n: int) -> int:
    return int(load().sk_kmeanspp_workspace_bytes(ctx.handle, int(n)))


def sk_kmeanspp(ctx: Ctx, idx, val, K: int, restart: int = 0, mu=None, rows=None, work=None,
                stream=None):
    """K-means++ seeding: (centres K x pt float32, chosen rows K int64), on the device."""
    n = idx.shape[0]
    _need(idx, torch.int32, "idx", (n, ctx.m))
    _need(val, torch.float32, "val", (n, ctx.m))
    dev = idx.device
    if mu is None:
        mu = torch.empty((K, ctx.pt), dtype=torch.float32, device=dev)
    if rows is None:
        rows = torch.empty(K, dtype=torch.int64, device=dev)
    _need(mu, torch.float32, "mu", (K, ctx.pt))
    _need(rows, torch.int64, "rows", (K,))
    need = sk_kmeanspp_workspace_bytes(ctx, n)
    if work is None:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    _check("sk_kmeanspp", load().sk_kmeanspp(ctx.handle, _ptr(idx), _ptr(val), n, int(K),
                                             int(restart), _ptr(mu), _ptr(rows), _ptr(work),
                                             work.numel() * work.element_size(), _stream(stream)))
    return mu, rows


def sk_kmeans_objective(dist, J=None, stream=None):
    """J' = sum of the winning distances (device float64 scalar)."""
    _need(dist, torch.float32, "dist")
    if J is None:
        J = torch.empty(1, dtype=torch.float64, device=dist.device)
    _check("sk_kmeans_objective", load().sk_kmeans_objective(_ptr(dist), dist.numel(), _ptr(J),
                                                             _stream(stream)))
    return J


def sk_kmeans_hk(ctx: Ctx, cnt, nk, dev=None, stream=None):
    """||H_k - I||_2 per cluster (device float64 K; -1 for an empty cluster)."""
    K = nk.shape[0]
    _need(cnt, torch.int32, "cnt", (K, ctx.pt))
    _need(nk, torch.int64, "nk", (K,))
    if dev is None:
        dev = torch.empty(K, dtype=torch.float64, device=nk.device)
    _check("sk_kmeans_hk", load().sk_kmeans_hk(ctx.handle, K, _ptr(cnt), _ptr(nk), _ptr(dev),
                                               _stream(stream)))
    return dev


def sk_mean_accumulate(ctx: Ctx, idx, val, sums, stream=None):
    n = idx.shape[0]
    _need(idx, torch.int32, "idx", (n, ctx.m))
    _need(val, torch.float32, "val", (n, ctx.m))
    _need(sums, torch.float64, "sums", (ctx.pt,))
    _check("sk_mean_accumulate", load().sk_mean_accumulate(ctx.handle, _ptr(idx), _ptr(val), n,
                                                           _ptr(sums), _stream(stream)))
    return sums


def sk_mean_finalize(ctx: Ctx, sums, n_total: int, mean=None, stream=None):
    _need(sums, torch.float64, "sums", (ctx.pt,))
    if mean is None:
        mean = torch.empty_like(sums)
    _need(mean, torch.float64, "mean", (ctx.pt,))
    _check("sk_mean_finalize", load().sk_mean_finalize(ctx.handle, _ptr(sums), int(n_total),
                                                       _ptr(mean), _stream(stream)))
    return mean


class SkBatchItem(ctypes.Structure):
    """sk_batch_item of include/sk.h (same field order and types)."""
    _fields_ = [("p", ctypes.c_int64), ("m", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("X", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("ldx", ctypes.c_int64), ("row0", ctypes.c_int64), ("idx", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("G", ctypes.c_void_p), ("gram_work", ctypes.c_void_p),
                ("gram_work_bytes", ctypes.c_int64), ("K", ctypes.c_int32), ("mu", ctypes.c_void_p),
                ("mu_t", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("S", ctypes.c_void_p), ("cnt", ctypes.c_void_p),
                ("nk", ctypes.c_void_p), ("changed", ctypes.c_void_p)]


class Batch:
    """Owns an sk_batch* (host plan) and keeps the item tensors alive."""

    def __init__(self, handle: int, keep):
        self._h = ctypes.c_void_p(handle)
        self._keep = keep

    @property
    def handle(self):
        return self._h

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.sk_batch_destroy(self._h)
                self._h = ctypes.c_void_p(0)
        except Exception:
            pass


def sk_batch_create(items, gram_mode: int, keep=None) -> Batch:
    """items: list of SkBatchItem (device pointers filled in by the caller)."""
    arr = (SkBatchItem * len(items))(*items)
    h = ctypes.c_void_p(0)
    _check("sk_batch_create", load().sk_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p),
                                                     len(items), int(gram_mode)))
    return Batch(h.value, keep)


def sk_batch_workspace_bytes(b: Batch) -> int:
    return int(load().sk_batch_workspace_bytes(b.handle))


def sk_batch_upload(b: Batch, work, stream=None):
    _check("sk_batch_upload", load().sk_batch_upload(b.handle, _ptr(work),
                                                     work.numel() * work.element_size(),
                                                     _stream(stream)))


def sk_batch_compress(b: Batch, stream=None):
    _check("sk_batch_compress", load().sk_batch_compress(b.handle, _stream(stream)))


def sk_batch_cov_reset(b: Batch, stream=None):
    _check("sk_batch_cov_reset", load().sk_batch_cov_reset(b.handle, _stream(stream)))


def sk_batch_cov_accumulate(b: Batch, stream=None):
    _check("sk_batch_cov_accumulate", load().sk_batch_cov_accumulate(b.handle, _stream(stream)))


def sk_batch_kmeans_reset(b: Batch, stream=None):
    _check("sk_batch_kmeans_reset", load().sk_batch_kmeans_reset(b.handle, _stream(stream)))


def sk_batch_kmeans_step(b: Batch, incremental: bool, stream=None):
    _check("sk_batch_kmeans_step", load().sk_batch_kmeans_step(b.handle, 1 if incremental else 0,
                                                               _stream(stream)))


def sk_batch_kmeans_finalize(b: Batch, stream=None):
    _check("sk_batch_kmeans_finalize", load().sk_batch_kmeans_finalize(b.handle, _stream(stream)))


def sk_batch_autotune(b: Batch, work, stream=None):
    """Returns (units per row group, Gram tile width) chosen by the library."""
    u, t = ctypes.c_int32(0), ctypes.c_int32(0)
    _check("sk_batch_autotune", load().sk_batch_autotune(b.handle, _ptr(work),
                                                         work.numel() * work.element_size(),
                                                         _stream(stream), ctypes.byref(u),
                                                         ctypes.byref(t)))
    return int(u.value), int(t.value)


def sk_autotune_gram(ctx: Ctx, mode: int, idx, val, G, work=None, stream=None):
    """Returns (tile width, split multiplier); G is overwritten."""
    n = idx.shape[0]
    need = sk_cov_workspace_bytes(ctx, mode, n)
    if work is None:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device=idx.device)
    a, b = ctypes.c_int32(0), ctypes.c_int32(0)
    _check("sk_autotune_gram", load().sk_autotune_gram(
        ctx.handle, int(mode), _ptr(idx), _ptr(val), n, _ptr(G), _ptr(work),
        work.numel() * work.element_size(), _stream(stream), ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def sk_autotune_compress(ctx: Ctx, X, idx, val, stream=None):
    """Returns the chosen CTAs per SM (0: as many as fit); idx/val are overwritten."""
    n, ldx = _rows_ld(X, ctx.p)
    c = ctypes.c_int32(0)
    _check("sk_autotune_compress", load().sk_autotune_compress(
        ctx.handle, _ptr(X), n, ldx, _ptr(idx), _ptr(val), _stream(stream), ctypes.byref(c)))
    return int(c.value)


def sk_batch_destroy(b: Batch):
    if b._h:
        load().sk_batch_destroy(b._h)
        b._h = ctypes.c_void_p(0)


def sk_device_status(stream=None) -> int:
    """Returns the status code (SK_OK, SK_ETIMEOUT, SK_ECUDA) without raising."""
    return int(load().sk_device_status(_stream(stream)))


def sk_debug_set_wait_cycles(cycles: int) -> None:
    """Limit of the kernels' bounded device waits in SM cycles (0: the default)."""
    _check("sk_debug_set_wait_cycles", load().sk_debug_set_wait_cycles(int(cycles)))


def sk_last_error() -> str:
    msg = load().sk_last_error()
    return msg.decode() if msg else ""
