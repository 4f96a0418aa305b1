"""Bounded device waits: a wait that runs out is reported, and the library
keeps working afterwards.

The mbarrier waits of the compress kernel (the bulk copies of each unit of
samples) and of the tensor-core Gram (its operand and accumulator pipeline)
give up after a limit, set the device error word and return once the copies
and tensor-core work already in flight are done.  Here the limit is cut to one
clock cycle through the test hook, so the first wait on a copy that has not
landed yet runs out; no wait is left without an end and no GPU fault is
involved.  Then:
  * sk_device_status reports SK_ETIMEOUT (and clears it),
  * with the default limit restored, the same call matches the FP64 oracle
    (idx bit-exact, val <= 1e-5 ||x_r||; Gram relative Frobenius <= 1e-5).
The compress case at pt = 4096 runs a row over four warps, whose outcome of
each wait is shared so that they leave together.
"""
import numpy as np
import pytest

import oracle
from paper_1511_00152_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    from paper_1511_00152_gb300 import _lib
    return _lib


def _timed_out(sk, fn):
    assert sk.sk_device_status() == sk.SK_OK
    sk.sk_debug_set_wait_cycles(1)
    try:
        fn()
        torch.cuda.synchronize()
    finally:
        sk.sk_debug_set_wait_cycles(0)
    st = sk.sk_device_status()
    assert st == sk.SK_ETIMEOUT, (st, sk.sk_last_error())
    assert sk.sk_device_status() == sk.SK_OK  # reported once, then cleared


@pytest.mark.parametrize("p,m,n", [(1024, 51, 20000), (4096, 205, 600)])
def test_compress_wait_runs_out_then_recovers(sk, p, m, n):
    X = synth.mixture(n, p, 5, seed=p)[0]
    Xd = torch.as_tensor(X, device="cuda")
    ctx = sk.sk_init(p, m, 77)
    _timed_out(sk, lambda: sk.sk_compress(ctx, Xd))
    idx, val = sk.sk_compress(ctx, Xd)
    torch.cuda.synchronize()
    assert sk.sk_device_status() == sk.SK_OK
    oi, ov = oracle.compress(X, m, 77)
    assert np.array_equal(idx.cpu().numpy(), oi)
    norms = np.linalg.norm(X.astype(np.float64), axis=1)
    assert np.all(np.abs(val.cpu().numpy() - ov).max(axis=1) <= 1e-5 * norms)


def test_tensor_core_gram_wait_runs_out_then_recovers(sk):
    p, m, n, seed = 1024, 51, 8000, 5
    X = synth.lowrank_spiky(n, p, seed=seed)
    ctx = sk.sk_init(p, m, seed)
    idx, val = sk.sk_compress(ctx, torch.as_tensor(X, device="cuda"))
    G = torch.zeros((ctx.pt, ctx.pt), dtype=torch.float64, device="cuda")
    _timed_out(sk, lambda: sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G))
    sk.sk_cov_reset(ctx, G)
    sk.sk_cov_accumulate(ctx, sk.SK_GRAM_BF16X3, idx, val, G)
    torch.cuda.synchronize()
    assert sk.sk_device_status() == sk.SK_OK
    oi, ov = oracle.compress(X, m, seed)
    Go = np.triu(oracle.gram(oi, ov, ctx.pt))
    Gg = np.triu(G.cpu().numpy())
    assert np.linalg.norm(Gg - Go) <= 1e-5 * np.linalg.norm(Go)
