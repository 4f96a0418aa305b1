"""FP64 CPU oracle for preconditioned data sparsification.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_1511_00152_gb300``) never imports it, and this package never
imports the product.

The arithmetic lives in ``sk_oracle.c`` (plain single-threaded C loops in
double precision); this module compiles it with gcc on first use and wraps
each routine with numpy arrays.  The one library routine used is LAPACK's
symmetric eigensolver (``numpy.linalg.eigh``) for the PCA step.

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``):
  philox4x32_10   -- known-answer vectors published with Random123 (SC'11)
  signs, mask     -- distribution tests: P(keep j) = m/p (Lemma B2), ordered
                     m-tuples uniform, exactly m distinct indices, m = p gives
                     a permutation; Lemire rejection driven by explicit words
  fwht            -- explicit Sylvester matrix at p <= 64, orthonormality,
                     involution, norm preservation (Sec. III)
  compress        -- the above plus the gather identity val = y[idx]
  gram/cov        -- exhaustive enumeration of every mask at p = 8: the mask
                     average equals C_emp (unbiasedness, Sec. V / Appendix C);
                     m = p reduces to (1/n) Y^T Y exactly
  sample_mean     -- exhaustive enumeration: unbiased (Sec. IV)
  cov_centred     -- exhaustive enumeration over every pair of masks of two
                     rows at p = 8: the mask average equals the centred second
                     moment (1/n) Y^T Y - ybar ybar^T; m = p reduces to it
                     exactly
  kmeans          -- m = p reduces to Lloyd's on H D X (Sec. VI-A), brute-force
                     argmin on tiny inputs, J' non-increasing (Sec. VI-B)
  unmix           -- D H (H D x) = x; back-map (HD)^T C_emp(Y) (HD) = C_emp(X)
  pca_topk        -- LAPACK eigh (library); compared as subspaces
  compress_raw    -- val = x[idx] with the (pinned) mask; raw padding is zero
  dct, idct       -- scipy.fft's orthonormal DCT-II / DCT-III (library);
                     orthonormality; closed forms (constant vector, cosine
                     basis vectors); entries bounded by sqrt(2/p), the
                     coherence behind eta = 1/2 of Sec. III, and the tail
                     bound 2 exp(-t^2/4) over random signs
  precondition/compress/unmix with dct -- the same pins as the Hadamard
                     forms with p in place of pt (no padding)
  kmeans_2pass    -- brute-force dense distances and per-label means on small
                     inputs; converged Lloyd's is a fixed point (Algorithm 2)
  kmeans_hk       -- m = pt gives H_k = I exactly; ||H_k - I|| within the
                     matrix-Bernstein bound of Sec. VI-B (Thm. on H_k) at
                     failure probability 1e-6; brute-force diagonal on tiny input
  kpp_draw        -- chi-square uniformity over [0, W); draws stay below W with
                     a rejection rate near 1/2 (W = 2^63 + 1)
  kmeanspp        -- first centre uniform over the rows (chi-square over
                     restarts); second centre distributed as D^2 / sum D^2
                     (chi-square per first centre, SODA'07 D^2 sampling);
                     zero-distance duplicates never chosen; K = n distinct
                     rows gives a permutation; centres are the rows' scatters
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sk_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libsk_oracle.so")
_lock = threading.Lock()
_lib = None

TAG_SIGN = 0x5349474E
TAG_MASK = 0x4D41534B
TAG_INIT = 0x494E4954


def build(force: bool = False) -> str:
    """Compile sk_oracle.c into a shared library (gcc, -O2, no vector ISA flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, u64, u32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        sig = {
            "oracle_philox4x32_10": (None, [vp, vp, vp]),
            "oracle_ptilde": (i64, [i64]),
            "oracle_lemire_from_words": (u32, [u32, vp, i64, vp]),
            "oracle_signs": (None, [i64, u64, vp]),
            "oracle_mask": (None, [i64, i64, u64, i64, vp]),
            "oracle_init_rows": (None, [i64, i64, u64, vp]),
            "oracle_fwht": (None, [vp, i64]),
            "oracle_precondition": (None, [vp, i64, i64, i64, u64, vp]),
            "oracle_compress": (None, [vp, i64, i64, i64, i64, i64, u64, vp, vp]),
            "oracle_gram": (None, [vp, vp, i64, i64, i64, vp]),
            "oracle_cov_finalize": (None, [vp, i64, i64, i64, vp]),
            "oracle_sample_mean": (None, [vp, vp, i64, i64, i64, vp]),
            "oracle_cov_centred": (None, [vp, vp, i64, i64, i64, vp]),
            "oracle_kmeans_assign": (None, [vp, vp, i64, i64, vp, i64, i64, vp, vp]),
            "oracle_kmeans_update": (None, [vp, vp, vp, i64, i64, i64, i64, vp, vp, vp, vp]),
            "oracle_unmix": (None, [vp, i64, i64, i64, u64, vp]),
            "oracle_compress_raw": (None, [vp, i64, i64, i64, i64, i64, u64, vp, vp]),
            "oracle_kmeans_2pass": (None, [vp, i64, i64, vp, vp, i64, vp, vp, vp]),
            "oracle_kpp_draw": (u64, [u64, u32, u32, u64]),
            "oracle_kmeanspp": (None, [vp, vp, i64, i64, i64, i64, u64, u32, vp, vp]),
            "oracle_kmeans_hk": (None, [vp, vp, i64, i64, i64, vp]),
            "oracle_dct2": (None, [vp, i64]),
            "oracle_dct3": (None, [vp, i64]),
            "oracle_precondition_dct": (None, [vp, i64, i64, i64, u64, vp]),
            "oracle_compress_dct": (None, [vp, i64, i64, i64, i64, i64, u64, vp, vp]),
            "oracle_unmix_dct": (None, [vp, i64, i64, u64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- RNG spec

def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: ctr is 4 uint32 words, key is 2 uint32 words."""
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def lemire_from_words(s: int, words) -> tuple[int, int]:
    """U(s) drawn from an explicit word list: (value, words consumed or -1)."""
    w = _c(words, np.uint32)
    used = np.zeros(1, np.int64)
    v = _load().oracle_lemire_from_words(int(s), _p(w), w.size, _p(used))
    return int(v), int(used[0])


def ptilde(p: int) -> int:
    return int(_load().oracle_ptilde(int(p)))


def signs(pt: int, seed: int) -> np.ndarray:
    """Diagonal of D as +-1.0 (Sec. III)."""
    D = np.zeros(pt, np.float64)
    _load().oracle_signs(pt, seed, _p(D))
    return D


def mask(pt: int, m: int, seed: int, row: int) -> np.ndarray:
    """Omega_r: m distinct indices of [0, pt) in draw order."""
    out = np.zeros(max(m, 1), np.int32)
    _load().oracle_mask(pt, m, seed, row, _p(out))
    return out[:m]


def init_rows(n: int, K: int, seed: int) -> np.ndarray:
    """K distinct row indices of [0, n) (seeded K-means start for the harness)."""
    out = np.zeros(max(K, 1), np.int64)
    _load().oracle_init_rows(n, K, seed, _p(out))
    return out[:K]


# ------------------------------------------------------------ preconditioner

def fwht(y) -> np.ndarray:
    """Orthonormal Sylvester Walsh-Hadamard transform of a length-2^L vector."""
    a = _c(y, np.float64).copy()
    _load().oracle_fwht(_p(a), a.size)
    return a


def dct(y) -> np.ndarray:
    """Orthonormal DCT-II of a vector (the direct sum, Sec. III's DCT H)."""
    a = _c(y, np.float64).copy()
    _load().oracle_dct2(_p(a), a.size)
    return a


def idct(y) -> np.ndarray:
    """Its transpose, the orthonormal DCT-III (the inverse)."""
    a = _c(y, np.float64).copy()
    _load().oracle_dct3(_p(a), a.size)
    return a


def precondition(X, seed: int, dct: bool = False) -> np.ndarray:
    """Y = H D [X, 0] row by row (n x pt), from float32 samples; with dct the
    DCT of length p (no padding, n x p)."""
    X = _c(X, np.float32)
    n, p = X.shape
    if dct:
        Y = np.zeros((n, p), np.float64)
        _load().oracle_precondition_dct(_p(X), n, p, p, seed, _p(Y))
        return Y
    pt = ptilde(p)
    Y = np.zeros((n, pt), np.float64)
    _load().oracle_precondition(_p(X), n, p, p, seed, _p(Y))
    return Y


def compress(X, m: int, seed: int, row0: int = 0, dct: bool = False):
    """ELL form (idx int32 n x m, val float64 n x m) of rows row0.. of X; with
    dct the DCT preconditioner and masks over [0, p)."""
    X = _c(X, np.float32)
    n, p = X.shape
    idx = np.zeros((n, m), np.int32)
    val = np.zeros((n, m), np.float64)
    fn = _load().oracle_compress_dct if dct else _load().oracle_compress
    fn(_p(X), n, p, p, row0, m, seed, _p(idx), _p(val))
    return idx, val


def compress_raw(X, m: int, seed: int, row0: int = 0):
    """Ablation without preconditioning (H = D = I): ELL of the padded raw rows."""
    X = _c(X, np.float32)
    n, p = X.shape
    idx = np.zeros((n, m), np.int32)
    val = np.zeros((n, m), np.float64)
    _load().oracle_compress_raw(_p(X), n, p, p, row0, m, seed, _p(idx), _p(val))
    return idx, val


# ---------------------------------------------------------------- estimators

def gram(idx, val, pt: int, G=None) -> np.ndarray:
    """G += sum_i w_i w_i^T (pt x pt)."""
    idx = _c(idx, np.int32)
    val = _c(val, np.float64)
    n, m = idx.shape
    if G is None:
        G = np.zeros((pt, pt), np.float64)
    assert G.flags.c_contiguous and G.dtype == np.float64
    _load().oracle_gram(_p(idx), _p(val), n, m, pt, _p(G))
    return G


def cov_finalize(G, n: int, m: int) -> np.ndarray:
    """C_n from the accumulated Gram of n rows (Sec. V)."""
    G = _c(G, np.float64)
    pt = G.shape[0]
    C = np.zeros_like(G)
    _load().oracle_cov_finalize(_p(G), n, m, pt, _p(C))
    return C


def cov(idx, val, pt: int) -> np.ndarray:
    idx = np.asarray(idx)
    return cov_finalize(gram(idx, val, pt), idx.shape[0], idx.shape[1])


def cov_centred(G, mean, n: int, m: int) -> np.ndarray:
    """Centred covariance estimate C_n - xbar xbar^T + B(C_n)/n from the Gram
    of n rows and their sample-mean estimate xbar (unbiased for the centred
    second moment; derivation in sk_oracle.c)."""
    G = _c(G, np.float64)
    mean = _c(mean, np.float64)
    pt = G.shape[0]
    C = np.zeros_like(G)
    _load().oracle_cov_centred(_p(G), _p(mean), n, m, pt, _p(C))
    return C


def sample_mean(idx, val, pt: int) -> np.ndarray:
    idx = _c(idx, np.int32)
    val = _c(val, np.float64)
    n, m = idx.shape
    out = np.zeros(pt, np.float64)
    _load().oracle_sample_mean(_p(idx), _p(val), n, m, pt, _p(out))
    return out


def pca_topk(C, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Top-k eigenpairs of the symmetric estimate C (LAPACK eigh, FP64).

    Returns (eigenvalues descending, eigenvectors as columns).  The sign of
    each vector makes its largest-magnitude entry positive."""
    w, V = np.linalg.eigh(np.asarray(C, np.float64))
    order = np.argsort(w)[::-1][:k]
    w, V = w[order], V[:, order].copy()
    for c in range(V.shape[1]):
        j = np.argmax(np.abs(V[:, c]))
        if V[j, c] < 0:
            V[:, c] = -V[:, c]
    return w, V


def kmeans_assign(idx, val, mu, pt: int):
    idx = _c(idx, np.int32)
    val = _c(val, np.float64)
    mu = _c(mu, np.float64)
    n, m = idx.shape
    K = mu.shape[0]
    labels = np.zeros(n, np.int32)
    dist = np.zeros(n, np.float64)
    _load().oracle_kmeans_assign(_p(idx), _p(val), n, m, _p(mu), K, pt, _p(labels), _p(dist))
    return labels, dist


def kmeans_update(idx, val, labels, mu_prev, pt: int):
    idx = _c(idx, np.int32)
    val = _c(val, np.float64)
    labels = _c(labels, np.int32)
    mu_prev = _c(mu_prev, np.float64)
    n, m = idx.shape
    K = mu_prev.shape[0]
    mu_new = np.zeros_like(mu_prev)
    counts = np.zeros((K, pt), np.int64)
    nk = np.zeros(K, np.int64)
    _load().oracle_kmeans_update(_p(idx), _p(val), _p(labels), n, m, K, pt, _p(mu_prev),
                                 _p(mu_new), _p(counts), _p(nk))
    return mu_new, counts, nk


def kmeans_objective(idx, val, labels, mu) -> float:
    """J'(c, mu') of Sec. VI-A: sum_i || z_i - R_i^T mu'_{c_i} ||^2."""
    idx = np.asarray(idx)
    val = np.asarray(val, np.float64)
    mu = np.asarray(mu, np.float64)
    diff = val - mu[np.asarray(labels)[:, None], idx]
    return float(np.sum(diff * diff))


def kmeans(idx, val, mu0, pt: int, iters: int):
    """Sparsified K-means iterations (Algorithm 1, loop body): assign, then update."""
    mu = np.array(mu0, np.float64, copy=True)
    history = []
    labels = None
    for _ in range(iters):
        labels, _d = kmeans_assign(idx, val, mu, pt)
        history.append(kmeans_objective(idx, val, labels, mu))
        mu, _counts, _nk = kmeans_update(idx, val, labels, mu, pt)
    return labels, mu, history


def kmeans_2pass(X, labels1, mu1):
    """Algorithm 2's second pass: (labels2, mu2, counts) from the raw rows, the
    1-pass labels and the 1-pass (un-mixed) centres."""
    X = _c(X, np.float32)
    n, p = X.shape
    c1 = _c(labels1, np.int32)
    mu1 = _c(mu1, np.float64)
    K = mu1.shape[0]
    c2 = np.zeros(n, np.int32)
    mu2 = np.zeros((K, p), np.float64)
    counts = np.zeros(K, np.int64)
    _load().oracle_kmeans_2pass(_p(X), n, p, _p(c1), _p(mu1), K, _p(c2), _p(mu2), _p(counts))
    return c2, mu2, counts


def kpp_draw(seed: int, k: int, r: int, W: int) -> int:
    """K-means++ draw of step k, restart r, uniform over [0, W)."""
    return int(_load().oracle_kpp_draw(int(seed) & (2**64 - 1), k, r, W))


def kmeanspp(idx, val, pt: int, K: int, seed: int, r: int = 0):
    """K-means++ seeding on the ELL rows (val float32): (rows, centres K x pt float32)."""
    idx = _c(idx, np.int32)
    val = _c(val, np.float32)
    n, m = idx.shape
    rows = np.zeros(K, np.int64)
    cen = np.zeros((K, pt), np.float32)
    _load().oracle_kmeanspp(_p(idx), _p(val), n, m, pt, K, int(seed) & (2**64 - 1), r,
                            _p(rows), _p(cen))
    return rows, cen


def kmeans_hk(counts, nk, pt: int, m: int) -> np.ndarray:
    """||H_k - I||_2 per cluster (Eq. (Hkmk)); -1 for an empty cluster."""
    counts = _c(counts, np.int64)
    nk = _c(nk, np.int64)
    K = nk.shape[0]
    dev = np.zeros(K, np.float64)
    _load().oracle_kmeans_hk(_p(counts), _p(nk), K, pt, m, _p(dev))
    return dev


def unmix(M, p: int, seed: int, dct: bool = False) -> np.ndarray:
    """mu = D H^T mu' truncated to p coordinates, row by row (Eq. (mu-mu'));
    with dct, H is the DCT and mu' has p coordinates."""
    M = _c(M, np.float64)
    r, pt = M.shape
    out = np.zeros((r, p), np.float64)
    if dct:
        _load().oracle_unmix_dct(_p(M), r, p, seed, _p(out))
    else:
        _load().oracle_unmix(_p(M), r, pt, p, seed, _p(out))
    return out
