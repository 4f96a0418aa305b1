"""sk_cov_topk_static: the top-k entry point for callers that cannot allocate
device memory (for example, an application whose device memory is held by its
own caching allocator).  It runs the same top-k computation with its scratch
in a fixed array inside the library.

Checked through the C ABI against sk_cov_topk with a caller workspace, on two
calls in a row, with the tolerances of the other top-k tests (eigenvalues
rtol 1e-9, max sin of the principal angles <= 1e-6).  This file sorts last so
that a run stopping at the first failure has run every other test first; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sym_with_gap(pt, k, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((pt, pt)))
    lam = np.concatenate([np.linspace(10, 5, k), rng.uniform(-0.5, 1.0, pt - k)])
    C = (Q * lam) @ Q.T
    return 0.5 * (C + C.T)


def _max_sin(U1, U2):
    s = np.linalg.svd(U1 @ U2.T, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - s.min() ** 2)))


def test_static_scratch_matches_workspace_entry_point():
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import build as skbuild
    lib = sk.load(skbuild.build())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (pt, k, seed) in enumerate([(1024, 10, 1), (256, 20, 2)]):
        ctx = sk.sk_init(pt, 2, 8 + call)
        C = torch.as_tensor(_sym_with_gap(pt, k, seed), device="cuda")
        ev_ref, U_ref = sk.sk_cov_topk(ctx, C, k, iters=60)
        ev = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        U = torch.full((k, pt), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.sk_cov_topk_static(ctx.handle, ctypes.c_void_p(C.data_ptr()), k, 60,
                                    ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                    stream)
        assert st == sk.SK_OK, sk.sk_last_error()
        torch.cuda.synchronize()
        assert np.allclose(ev.cpu().numpy(), ev_ref.cpu().numpy(), rtol=1e-9, atol=1e-9)
        assert _max_sin(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-6
    assert sk.sk_device_status() == sk.SK_OK


def test_static_scratch_rejects_shapes_beyond_its_size():
    from paper_1511_00152_gb300 import _lib as sk
    from paper_1511_00152_gb300 import build as skbuild
    lib = sk.load(skbuild.build())
    ctx = sk.sk_init(8192, 2, 1)
    C = torch.zeros(1, dtype=torch.float64, device="cuda")  # never read: rejected first
    out = torch.zeros(64 * 8192, dtype=torch.float64, device="cuda")
    st = lib.sk_cov_topk_static(ctx.handle, ctypes.c_void_p(C.data_ptr()), 64, 10,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(0))
    assert st == sk.SK_EUNSUPPORTED
    assert "fixed array" in sk.sk_last_error()
