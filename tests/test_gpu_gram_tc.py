"""Tensor-core (tcgen05) Gram parity against the FP64 oracle.

Tolerances (relative Frobenius error of the upper-triangular Gram and of C_n):
  SK_GRAM_BF16X3 (split hi/lo, three products)  <= 1e-5
  SK_GRAM_BF16   (one BF16 product)             <= 1e-2  (BF16 keeps 8 bits)
"""
import numpy as np
import pytest

import oracle
from paper_1511_00152_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {1: 1e-2, 2: 1e-5}


@pytest.fixture(scope="module")
def sk():
    from paper_1511_00152_gb300 import _lib
    return _lib


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("mode", [2, 1])
@pytest.mark.parametrize("p,m,n", [
    (128, 13, 3000),     # N = 128 tile, one tile
    (256, 13, 2000),     # one 128-row block pair, N = 256
    (1024, 51, 5000),    # 20 upper tiles, ragged last slab
    (1000, 40, 777),     # padding to 1024, n not a multiple of 64
    (4096, 205, 400),    # PCA shape, 272 tiles
    (2048, 102, 130),
    (8192, 820, 64),     # largest pt
    (512, 512, 300),     # m = pt (dense rows)
])
def test_gram_tc_parity(sk, mode, p, m, n):
    X = synth.lowrank_spiky(n, p, seed=n + 3 * p)
    seed = 11
    ctx = sk.sk_init(p, m, seed)
    pt = ctx.pt
    oi, ov = oracle.compress(X, m, seed)
    # the GPU Gram runs on the oracle's ELL rows rounded to float32, and the
    # oracle's Gram of the same float32 values isolates the Gram
    v32 = ov.astype(np.float32)
    idx, val = _dev(oi), _dev(v32)
    Go = oracle.gram(oi, v32.astype(np.float64), pt)
    G = torch.empty((pt, pt), dtype=torch.float64, device="cuda")
    sk.sk_cov_reset(ctx, G)
    h = n // 2
    sk.sk_cov_accumulate(ctx, mode, idx[:h].contiguous(), val[:h].contiguous(), G)
    sk.sk_cov_accumulate(ctx, mode, idx[h:].contiguous(), val[h:].contiguous(), G)
    C = sk.sk_cov_finalize(ctx, G, n)
    torch.cuda.synchronize()
    assert sk.sk_device_status() == sk.SK_OK
    Gu = np.triu(G.cpu().numpy())
    Gou = np.triu(Go)
    rel = np.linalg.norm(Gu - Gou) / np.linalg.norm(Gou)
    assert rel <= TOL[mode], rel
    Co = oracle.cov_finalize(oracle.gram(oi, ov, pt), n, m)
    relc = np.linalg.norm(C.cpu().numpy() - Co) / np.linalg.norm(Co)
    assert relc <= TOL[mode] + 1e-6, relc


def test_gram_tc_two_segments(sk):
    """More than 65536 rows: several FP32 accumulation segments per tile,
    reduced in FP64."""
    n, p, m, seed = 70000, 256, 26, 5
    X = synth.mixture(n, p, 6, seed=1)[0]
    ctx = sk.sk_init(p, m, seed)
    oi, ov = oracle.compress(X, m, seed)
    v32 = ov.astype(np.float32)
    idx, val = _dev(oi), _dev(v32)
    Go = oracle.gram(oi, v32.astype(np.float64), ctx.pt)
    for mode in (2, 1):
        G = torch.zeros((ctx.pt, ctx.pt), dtype=torch.float64, device="cuda")
        sk.sk_cov_accumulate(ctx, mode, idx, val, G)
        torch.cuda.synchronize()
        rel = np.linalg.norm(np.triu(G.cpu().numpy()) - np.triu(Go)) / np.linalg.norm(np.triu(Go))
        assert rel <= TOL[mode], (mode, rel)


def test_gram_tc_rejects_small_pt(sk):
    ctx = sk.sk_init(64, 8, 1)
    idx = torch.zeros((10, 8), dtype=torch.int32, device="cuda")
    val = torch.zeros((10, 8), dtype=torch.float32, device="cuda")
    G = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SkError) as ei:
        sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G)
    assert ei.value.status == sk.SK_EUNSUPPORTED
