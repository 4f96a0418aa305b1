"""The bench's error report against the FP64 oracle (host logic, no GPU).

`bench.accuracy_vs_oracle` runs the library's path on the oracle's row sample
and compares each result with the oracle's.  Here the library calls are
replaced by stand-ins that return the oracle's own results, optionally with
a known error planted, so the report must read zero where nothing was
changed and the planted size where something was.
"""
import importlib.util
import os
import types

import numpy as np
import pytest
import torch

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _stand_ins(cfg, plant=None):
    """Library and pipeline stand-ins computing with the oracle; plant names
    one result to perturb ('val', 'cov', 'angle', 'labels')."""
    p, m, seed = cfg["p"], cfg["m"], cfg["seed"]
    pt = oracle.ptilde(p)
    sk = types.SimpleNamespace()

    def compress(ctx, X):
        i, v = oracle.compress(X.numpy(), m, seed)
        if plant == "val":
            v = v.copy()
            v[0, 0] += 1e-3 * np.linalg.norm(X.numpy()[0].astype(np.float64))
        return torch.as_tensor(i), torch.as_tensor(v)

    def accumulate(ctx, mode, idx, val, G, work=None):
        G.copy_(torch.as_tensor(oracle.gram(idx.numpy(), val.numpy(), pt)))

    def finalize(ctx, G, n, C=None):
        Cn = oracle.cov_finalize(G.numpy(), n, m)
        if plant == "cov":
            Cn = Cn * (1.0 + 1e-4)
        C.copy_(torch.as_tensor(Cn))

    def topk(ctx, C, k, iters, evals=None, U=None, work=None):
        w, V = oracle.pca_topk(C.numpy(), k)
        if plant == "angle":
            # rotate the last vector by 1e-3 rad towards a direction outside the span
            w_all, V_all = np.linalg.eigh(C.numpy())
            out = V_all[:, np.argsort(w_all)[::-1][k]]
            V = V.copy()
            V[:, -1] = np.cos(1e-3) * V[:, -1] + np.sin(1e-3) * out
        evals.copy_(torch.as_tensor(w))
        U.copy_(torch.as_tensor(V.T.copy()))

    sk.sk_compress = compress
    sk.sk_cov_reset = lambda ctx, G: G.zero_()
    sk.sk_cov_accumulate = accumulate
    sk.sk_cov_finalize = finalize
    sk.sk_cov_topk = topk
    sk.sk_precondition = lambda ctx, X: torch.as_tensor(oracle.precondition(X.numpy(), seed))

    class KMeans:
        def __init__(self, ctx, n, K, device=None):
            pass

        def run(self, idx, val, mu0, iters, use_graph=False):
            lab, mu, _ = oracle.kmeans(idx.numpy(), val.numpy(), mu0.numpy(), pt, iters)
            if plant == "labels":
                lab = lab.copy()
                lab[:10] = (lab[:10] + 1) % cfg["K"]
            return torch.as_tensor(lab), torch.as_tensor(mu)

    ctx = types.SimpleNamespace(pt=pt, p=p, m=m)
    return sk, types.SimpleNamespace(KMeansState=KMeans), ctx


@pytest.fixture(scope="module")
def sample():
    b = _bench()
    cfg = dict(b.WORKLOAD)
    _, _, smp = b.time_cpu_baseline(cfg, rows=1000)
    return b, cfg, smp


def _report(b, cfg, smp, plant=None, monkeypatch=None):
    sk, pipeline, ctx = _stand_ins(cfg, plant)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return b.accuracy_vs_oracle(sk, pipeline, ctx, 2, 4, None, None, smp, dict(cfg, gram="bf16x3"),
                                torch.device("cpu"))


def test_report_is_zero_for_the_oracle_itself(sample, monkeypatch):
    b, cfg, smp = sample
    r = _report(b, cfg, smp, monkeypatch=monkeypatch)
    assert r["rows"] == 1000
    assert r["idx_rows_exact"] == 1.0
    assert r["val_max_err_rel_row_norm"] == 0.0
    assert r["cov_rel_frobenius"] == 0.0
    assert r["topk_eigenvalue_max_rel_err"] == 0.0
    assert r["topk_max_sin_principal_angle"] < 1e-12
    assert r["kmeans_label_agreement"] == 1.0
    assert r["kmeans_centre_rel_err"] == 0.0


@pytest.mark.parametrize("plant,key,expect", [
    ("val", "val_max_err_rel_row_norm", 1e-3),
    ("cov", "cov_rel_frobenius", 1e-4),
    ("angle", "topk_max_sin_principal_angle", np.sin(1e-3)),
    ("labels", "kmeans_label_agreement", 1.0 - 10 / 1000),
])
def test_report_reads_a_planted_error(sample, monkeypatch, plant, key, expect):
    b, cfg, smp = sample
    r = _report(b, cfg, smp, plant=plant, monkeypatch=monkeypatch)
    assert r[key] == pytest.approx(expect, rel=1e-6)
