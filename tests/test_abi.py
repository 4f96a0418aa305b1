"""The C-ABI library loads without a GPU and exports every entry point that
include/sk.h declares (no compute calls)."""
import ctypes
import subprocess

from paper_1511_00152_gb300 import build as skbuild
from paper_1511_00152_gb300 import _lib


def test_library_builds_and_exports_header_symbols():
    path = skbuild.build()
    lib = ctypes.CDLL(path)
    declared = _lib.header_symbols()
    assert len(declared) >= 15
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    # nothing else sk_* is exported that the header does not declare
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    if out.returncode == 0:
        exported = {ln.split()[-1] for ln in out.stdout.splitlines() if " T sk_" in ln}
        assert exported <= set(declared), exported - set(declared)


def test_binding_covers_header():
    lib = _lib.load(skbuild.build())
    for s in _lib.header_symbols():
        assert getattr(lib, s).argtypes is not None or s == "sk_last_error", s


def test_host_validation_without_gpu():
    """Argument checks run on the host and need no device."""
    lib = _lib.load(skbuild.build())
    h = ctypes.c_void_p(0)
    assert lib.sk_init(ctypes.byref(h), 0, 1, 0) == _lib.SK_EINVAL
    assert lib.sk_init(ctypes.byref(h), 9000, 1, 0) == _lib.SK_EUNSUPPORTED
    assert lib.sk_init(ctypes.byref(h), 1000, 1025, 0) == _lib.SK_EINVAL
    assert lib.sk_init(ctypes.byref(h), 1000, 50, 7) == _lib.SK_OK
    assert lib.sk_ptilde(h) == 1024
    nul = ctypes.c_void_p(0)
    assert lib.sk_compress(h, nul, 3, 1000, 0, nul, nul, nul) == _lib.SK_EINVAL
    assert b"NULL" in lib.sk_last_error()
    assert lib.sk_cov_topk_workspace(1024, 10) > 0
    assert lib.sk_cov_topk_workspace(1024, 0) == -1
    lib.sk_destroy(h)
    lib.sk_destroy(nul)
    # flags: the ablation bit is accepted, unknown bits are not
    assert lib.sk_init_ex(ctypes.byref(h), 100, 5, 1, 4) == _lib.SK_EINVAL
    assert lib.sk_init_ex(ctypes.byref(h), 100, 5, 1, _lib.SK_FLAG_NO_PRECONDITION) == _lib.SK_OK
    assert lib.sk_flags(h) == _lib.SK_FLAG_NO_PRECONDITION
    assert lib.sk_kmeans2_assign(h, nul, 4, 100, nul, 3, nul, nul, nul) == _lib.SK_EINVAL
    assert lib.sk_kmeans2_sums(h, nul, 4, 99, nul, 3, nul, nul, nul) == _lib.SK_EINVAL
    assert b"ldx" in lib.sk_last_error()
    assert lib.sk_mean_finalize(h, nul, 0, nul, nul) == _lib.SK_EINVAL
    lib.sk_destroy(h)
    assert lib.sk_flags(nul) == 0
    # the DCT preconditioner: even p with p / 2 13-smooth, pt = p, not with the ablation
    assert lib.sk_init_ex(ctypes.byref(h), 784, 39, 1, _lib.SK_FLAG_DCT) == _lib.SK_OK
    assert lib.sk_ptilde(h) == 784
    lib.sk_destroy(h)
    assert lib.sk_init_ex(ctypes.byref(h), 785, 39, 1, _lib.SK_FLAG_DCT) == _lib.SK_EUNSUPPORTED
    assert lib.sk_init_ex(ctypes.byref(h), 2 * 17, 4, 1, _lib.SK_FLAG_DCT) == _lib.SK_EUNSUPPORTED
    assert lib.sk_init_ex(ctypes.byref(h), 784, 4, 1,
                          _lib.SK_FLAG_DCT | _lib.SK_FLAG_NO_PRECONDITION) == _lib.SK_EINVAL
    it = _lib.SkBatchItem(p=1000, m=50, seed=1, flags=_lib.SK_FLAG_DCT, n=10, ldx=1000, K=3)
    bb = ctypes.c_void_p(0)
    assert lib.sk_batch_create(ctypes.byref(bb), ctypes.cast(ctypes.pointer(it), ctypes.c_void_p),
                               1, _lib.SK_GRAM_BF16) == _lib.SK_EUNSUPPORTED
    # batch plans validate their items on the host before any CUDA call
    it = _lib.SkBatchItem(p=100, m=5, seed=1, n=10, ldx=100, K=3)
    b = ctypes.c_void_p(0)
    assert lib.sk_batch_create(ctypes.byref(b), ctypes.cast(ctypes.pointer(it), ctypes.c_void_p), 1,
                               _lib.SK_GRAM_BF16) == _lib.SK_EUNSUPPORTED  # pt = 128
    it = _lib.SkBatchItem(p=512, m=5, seed=1, n=10, ldx=512, K=100)
    assert lib.sk_batch_create(ctypes.byref(b), ctypes.cast(ctypes.pointer(it), ctypes.c_void_p), 1,
                               _lib.SK_GRAM_BF16) == _lib.SK_EUNSUPPORTED  # K > 64
    it = _lib.SkBatchItem(p=512, m=5, seed=1, n=10, ldx=512, K=4)
    assert lib.sk_batch_create(ctypes.byref(b), ctypes.cast(ctypes.pointer(it), ctypes.c_void_p), 1,
                               _lib.SK_GRAM_BF16) == _lib.SK_EINVAL  # NULL buffers
    assert b"NULL" in lib.sk_last_error()
    assert lib.sk_batch_workspace_bytes(nul) == -1
