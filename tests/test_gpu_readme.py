"""The documented usage example (compress, covariance, top-k PCA, K-means,
un-mixed centres) runs as written at a smaller n and returns results of the
documented shapes."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_readme_example():
    from paper_1511_00152_gb300 import build, pipeline
    build.build()
    from paper_1511_00152_gb300 import _lib as sk

    X = torch.randn(20_000, 1024, device="cuda")
    ctx = sk.sk_init(1024, 51, seed=7)
    idx, val = sk.sk_compress(ctx, X)
    C = pipeline.covariance(ctx, idx, val, sk.SK_GRAM_BF16X3)
    evals, Up, U = pipeline.pca(ctx, C, k=10)
    mu0 = pipeline.initial_centres(ctx, X, rows=list(range(10)))
    st = pipeline.KMeansState(ctx, X.shape[0], 10)
    st.run(idx, val, mu0, iters=20)
    centres = sk.sk_unmix(ctx, st.mu)
    torch.cuda.synchronize()
    assert idx.shape == (20_000, 51) and val.shape == (20_000, 51)
    assert evals.shape == (10,) and U.shape == (10, 1024)
    assert centres.shape == (10, 1024)
    lab = st.labels
    assert int(lab.min()) >= 0 and int(lab.max()) < 10
    assert sk.sk_device_status() == sk.SK_OK
