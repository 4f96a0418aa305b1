"""GB300 library for preconditioned data sparsification (Pourkamali-Anaraki &
Becker): one-pass H D preconditioning + uniform m-of-p sampling into ELL rows,
the unbiased covariance estimator for PCA, and sparsified K-means.

The compute lives in libsk.so (CUDA, sm_103a) behind the C ABI of
include/sk.h; ``_lib`` is its ctypes binding (same function names) and
``pipeline`` drives the paper's algorithms through it.
"""
from ._lib import (  # noqa: F401
    SK_EINVAL, SK_ECUDA, SK_ENOMEM, SK_ETIMEOUT, SK_EUNSUPPORTED, SK_GRAM_BF16,
    SK_GRAM_BF16X3, SK_GRAM_FP32, SK_OK, Ctx, SkError, sk_compress, sk_cov_accumulate,
    sk_cov_finalize, sk_cov_reset, sk_cov_topk, sk_cov_topk_workspace, sk_device_status,
    sk_init, sk_kmeans_assign, sk_kmeans_finalize, sk_kmeans_reset, sk_kmeans_step,
    sk_kmeans_update, sk_last_error, sk_precondition, sk_ptilde, sk_unmix)
