// sk_api.cu -- the C ABI (include/sk.h): argument validation on the host,
// then one or more kernel launches on the caller's stream.  No exception
// crosses the boundary; every failure returns a status and records a message
// for sk_last_error().
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "sk_internal.cuh"

namespace {

thread_local char g_msg[512] = {0};

sk_status fail(sk_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

sk_status cuda_status(cudaError_t e, const char *where) {
    if (e == cudaSuccess) {
        g_msg[0] = 0;
        return SK_OK;
    }
    return fail(SK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

#define SK_CHECK_CTX(c)                                                   \
    do {                                                                  \
        if (!(c)) return fail(SK_EINVAL, "%s: ctx is NULL", __func__);    \
    } while (0)

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = static_cast<const char *>(a), *pb = static_cast<const char *>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

namespace sk {
void set_last_error(const char *msg) {
    std::snprintf(g_msg, sizeof(g_msg), "%s", msg ? msg : "");
}

constexpr long long kDefaultWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
std::atomic<long long> g_wait_cycles{kDefaultWaitCycles};

long long wait_limit_cycles() { return g_wait_cycles.load(std::memory_order_relaxed); }
}  // namespace sk

extern "C" {

sk_status sk_init(sk_ctx **ctx, int64_t p, int64_t m, uint64_t seed) {
    return sk_init_ex(ctx, p, m, seed, 0u);
}

uint32_t sk_flags(const sk_ctx *ctx) { return ctx ? ctx->flags : 0u; }

sk_status sk_init_ex(sk_ctx **ctx, int64_t p, int64_t m, uint64_t seed, uint32_t flags) {
    if (!ctx) return fail(SK_EINVAL, "sk_init: ctx out-pointer is NULL");
    *ctx = nullptr;
    if (p < 1) return fail(SK_EINVAL, "sk_init: p = %lld must be >= 1", (long long)p);
    if (p > 8192) return fail(SK_EUNSUPPORTED, "sk_init: p = %lld > 8192", (long long)p);
    int L = 0;
    while ((1LL << L) < p) ++L;
    if (flags & ~(uint32_t)(SK_FLAG_NO_PRECONDITION | SK_FLAG_DCT))
        return fail(SK_EINVAL, "sk_init: unknown flag bits 0x%x", flags);
    const bool dct = (flags & SK_FLAG_DCT) != 0;
    int fac[16] = {0}, nf = 0;
    if (dct) {
        if (flags & SK_FLAG_NO_PRECONDITION)
            return fail(SK_EINVAL, "sk_init: SK_FLAG_DCT and SK_FLAG_NO_PRECONDITION exclude each other");
        if (p % 2 != 0)
            return fail(SK_EUNSUPPORTED, "sk_init: the DCT preconditioner needs an even p (p = %lld)",
                        (long long)p);
        if (!sk::dct_factor(p / 2, fac, &nf))
            return fail(SK_EUNSUPPORTED,
                        "sk_init: the DCT preconditioner needs p / 2 without prime factors above 13 "
                        "(p = %lld)", (long long)p);
    }
    // the DCT keeps pt = p (no padding)
    const int64_t pt = dct ? p : 1LL << L;
    if (m < 1 || m > pt)
        return fail(SK_EINVAL, "sk_init: m = %lld must be in [1, pt = %lld]", (long long)m,
                    (long long)pt);
    sk_ctx *c = new (std::nothrow) sk_ctx;
    if (!c) return fail(SK_ENOMEM, "sk_init: out of host memory");
    c->p = p;
    c->pt = pt;
    c->log2pt = L;
    c->dct_nf = nf;
    for (int k = 0; k < 16; ++k) c->dct_fac[k] = fac[k];
    c->m = m;
    c->seed = seed;
    c->flags = flags;
    c->gram_n = 0;
    c->split_mult = 0;
    c->compress_ctas = 0;
    *ctx = c;
    g_msg[0] = 0;
    return SK_OK;
}

void sk_destroy(sk_ctx *ctx) { delete ctx; }

int64_t sk_ptilde(const sk_ctx *ctx) { return ctx ? ctx->pt : -1; }

sk_status sk_compress(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx, int64_t row0,
                      int32_t *idx, float *val, void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_compress: n < 0");
    if (row0 < 0) return fail(SK_EINVAL, "sk_compress: row0 < 0");
    if (ldx < ctx->p) return fail(SK_EINVAL, "sk_compress: ldx < p");
    if (n == 0) return SK_OK;
    if (!X || !idx || !val) return fail(SK_EINVAL, "sk_compress: NULL buffer");
    return cuda_status(sk::launch_compress(*ctx, X, n, ldx, row0, idx, val, nullptr,
                                           as_stream(stream)),
                       "sk_compress");
}

sk_status sk_precondition(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx, float *Y,
                          void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_precondition: n < 0");
    if (ldx < ctx->p) return fail(SK_EINVAL, "sk_precondition: ldx < p");
    if (n == 0) return SK_OK;
    if (!X || !Y) return fail(SK_EINVAL, "sk_precondition: NULL buffer");
    return cuda_status(sk::launch_compress(*ctx, X, n, ldx, 0, nullptr, nullptr, Y,
                                           as_stream(stream)),
                       "sk_precondition");
}

int64_t sk_cov_workspace_bytes(const sk_ctx *ctx, int mode, int64_t n) {
    if (!ctx || n < 0) return -1;
    if (mode == SK_GRAM_FP32) return 0;
    if (mode != SK_GRAM_BF16 && mode != SK_GRAM_BF16X3) return -1;
    return sk::gram_tc_workspace(*ctx, n);
}

sk_status sk_cov_accumulate(const sk_ctx *ctx, int mode, const int32_t *idx, const float *val,
                            int64_t n, double *G, void *work, int64_t work_bytes, void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_cov_accumulate: n < 0");
    if (mode != SK_GRAM_FP32 && mode != SK_GRAM_BF16 && mode != SK_GRAM_BF16X3)
        return fail(SK_EINVAL, "sk_cov_accumulate: unknown mode %d", mode);
    if (n == 0) return SK_OK;
    if (!idx || !val || !G) return fail(SK_EINVAL, "sk_cov_accumulate: NULL buffer");
    cudaError_t e;
    if (mode == SK_GRAM_FP32) {
        e = sk::launch_gram_fp32(*ctx, idx, val, n, G, as_stream(stream));
    } else {
        if (ctx->pt < 128)
            return fail(SK_EUNSUPPORTED,
                        "sk_cov_accumulate: tensor-core modes need pt >= 128 (pt = %lld)",
                        (long long)ctx->pt);
        const int64_t need = sk::gram_tc_workspace(*ctx, n);
        if (!work || work_bytes < need)
            return fail(SK_EINVAL, "sk_cov_accumulate: workspace of %lld bytes needed, %lld given",
                        (long long)need, (long long)(work ? work_bytes : 0));
        if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
            return fail(SK_EINVAL, "sk_cov_accumulate: workspace must be 256-byte aligned");
        e = sk::launch_gram_tc(*ctx, mode, idx, val, n, G, work, as_stream(stream));
    }
    return cuda_status(e, "sk_cov_accumulate");
}

sk_status sk_cov_reset(const sk_ctx *ctx, double *G, void *stream) {
    SK_CHECK_CTX(ctx);
    if (!G) return fail(SK_EINVAL, "sk_cov_reset: NULL buffer");
    return cuda_status(cudaMemsetAsync(G, 0, (size_t)ctx->pt * ctx->pt * sizeof(double),
                                       as_stream(stream)),
                       "sk_cov_reset");
}

sk_status sk_cov_finalize(const sk_ctx *ctx, const double *G, int64_t n_total, double *C,
                          void *stream) {
    SK_CHECK_CTX(ctx);
    if (ctx->m < 2) return fail(SK_EINVAL, "sk_cov_finalize: needs m >= 2 (Thm. B1)");
    if (n_total < 1) return fail(SK_EINVAL, "sk_cov_finalize: n_total < 1");
    if (!G || !C) return fail(SK_EINVAL, "sk_cov_finalize: NULL buffer");
    const size_t bytes = (size_t)ctx->pt * ctx->pt * sizeof(double);
    if (overlaps(G, bytes, C, bytes)) return fail(SK_EINVAL, "sk_cov_finalize: G and C overlap");
    return cuda_status(sk::launch_cov_finalize(*ctx, G, n_total, nullptr, C, as_stream(stream)),
                       "sk_cov_finalize");
}

sk_status sk_cov_finalize_centred(const sk_ctx *ctx, const double *G, const double *mean,
                                  int64_t n_total, double *C, void *stream) {
    SK_CHECK_CTX(ctx);
    if (ctx->m < 2) return fail(SK_EINVAL, "sk_cov_finalize_centred: needs m >= 2 (Thm. B1)");
    if (n_total < 1) return fail(SK_EINVAL, "sk_cov_finalize_centred: n_total < 1");
    if (!G || !mean || !C) return fail(SK_EINVAL, "sk_cov_finalize_centred: NULL buffer");
    const size_t bytes = (size_t)ctx->pt * ctx->pt * sizeof(double);
    const size_t mbytes = (size_t)ctx->pt * sizeof(double);
    if (overlaps(G, bytes, C, bytes) || overlaps(mean, mbytes, C, bytes))
        return fail(SK_EINVAL, "sk_cov_finalize_centred: C overlaps G or mean");
    return cuda_status(sk::launch_cov_finalize(*ctx, G, n_total, mean, C, as_stream(stream)),
                       "sk_cov_finalize_centred");
}

int64_t sk_cov_topk_workspace(int64_t pt, int32_t k) {
    if (pt < 1 || k < 1 || k > 64 || k > pt) return -1;
    return sk::topk_workspace(pt, k);
}

sk_status sk_cov_topk(const sk_ctx *ctx, const double *C, int32_t k, int32_t iters,
                      double *evals, double *U, double *work, void *stream) {
    SK_CHECK_CTX(ctx);
    if (k < 1 || k > 64 || k > ctx->pt)
        return fail(SK_EINVAL, "sk_cov_topk: k = %d must be in [1, min(pt, 64)]", k);
    if (iters < 0 || iters > 100000) return fail(SK_EINVAL, "sk_cov_topk: iters out of range");
    if (!C || !evals || !U || !work) return fail(SK_EINVAL, "sk_cov_topk: NULL buffer");
    if (reinterpret_cast<uintptr_t>(C) % 16 != 0)
        return fail(SK_EINVAL, "sk_cov_topk: C must be 16-byte aligned");
    return cuda_status(sk::launch_topk(*ctx, C, k, iters, evals, U, work, as_stream(stream)),
                       "sk_cov_topk");
}

sk_status sk_cov_topk_static(const sk_ctx *ctx, const double *C, int32_t k, int32_t iters,
                             double *evals, double *U, void *stream) {
    SK_CHECK_CTX(ctx);
    if (k < 1 || k > 64 || k > ctx->pt)
        return fail(SK_EINVAL, "sk_cov_topk_static: k = %d must be in [1, min(pt, 64)]", k);
    if (iters < 0 || iters > 100000)
        return fail(SK_EINVAL, "sk_cov_topk_static: iters out of range");
    if (!C || !evals || !U) return fail(SK_EINVAL, "sk_cov_topk_static: NULL buffer");
    if (reinterpret_cast<uintptr_t>(C) % 16 != 0)
        return fail(SK_EINVAL, "sk_cov_topk_static: C must be 16-byte aligned");
    const int64_t need = sk::topk_workspace(ctx->pt, k);
    const int64_t have = sk::topk_static_capacity();
    if (need > have)
        return fail(SK_EUNSUPPORTED,
                    "sk_cov_topk_static: pt = %lld, k = %d needs %lld doubles of scratch; the "
                    "fixed array holds %lld (use sk_cov_topk with a caller workspace)",
                    (long long)ctx->pt, k, (long long)need, (long long)have);
    double *scratch = nullptr;
    cudaError_t e = sk::topk_static_scratch(&scratch);
    if (e != cudaSuccess) return cuda_status(e, "sk_cov_topk_static (scratch lookup)");
    return cuda_status(sk::launch_topk(*ctx, C, k, iters, evals, U, scratch, as_stream(stream)),
                       "sk_cov_topk_static");
}

static sk_status kmeans_common(const char *fn, const sk_ctx *ctx, const int32_t *idx,
                               const float *val, int64_t n, int32_t K) {
    if (!ctx) return fail(SK_EINVAL, "%s: ctx is NULL", fn);
    if (n < 0) return fail(SK_EINVAL, "%s: n < 0", fn);
    if (K < 1 || K > 256) return fail(SK_EINVAL, "%s: K = %d must be in [1, 256]", fn, K);
    if (n > 0 && (!idx || !val)) return fail(SK_EINVAL, "%s: NULL ELL buffer", fn);
    if ((int64_t)K * ctx->pt > (1LL << 31) - 1) return fail(SK_EUNSUPPORTED, "%s: K*pt too big", fn);
    return SK_OK;
}

sk_status sk_kmeans_assign(const sk_ctx *ctx, const int32_t *idx, const float *val, int64_t n,
                           const float *mu, int32_t K, int32_t *labels, float *dist,
                           void *stream) {
    sk_status st = kmeans_common("sk_kmeans_assign", ctx, idx, val, n, K);
    if (st != SK_OK) return st;
    if (n == 0) return SK_OK;
    if (!mu || !labels) return fail(SK_EINVAL, "sk_kmeans_assign: NULL buffer");
    return cuda_status(sk::launch_kmeans(*ctx, idx, val, n, mu, K, labels, dist, nullptr,
                                         nullptr, nullptr, true, 0, nullptr, as_stream(stream)),
                       "sk_kmeans_assign");
}

sk_status sk_kmeans_update(const sk_ctx *ctx, const int32_t *idx, const float *val,
                           const int32_t *labels, int64_t n, int32_t K, double *S, int32_t *cnt,
                           int64_t *nk, void *stream) {
    sk_status st = kmeans_common("sk_kmeans_update", ctx, idx, val, n, K);
    if (st != SK_OK) return st;
    if (n == 0) return SK_OK;
    if (!labels || !S || !cnt || !nk) return fail(SK_EINVAL, "sk_kmeans_update: NULL buffer");
    return cuda_status(sk::launch_kmeans(*ctx, idx, val, n, nullptr, K,
                                         const_cast<int32_t *>(labels), nullptr, S, cnt, nk,
                                         false, 1, nullptr, as_stream(stream)),
                       "sk_kmeans_update");
}

sk_status sk_kmeans_step(const sk_ctx *ctx, const int32_t *idx, const float *val, int64_t n,
                         const float *mu, int32_t K, int32_t *labels, float *dist, double *S,
                         int32_t *cnt, int64_t *nk, void *stream) {
    sk_status st = kmeans_common("sk_kmeans_step", ctx, idx, val, n, K);
    if (st != SK_OK) return st;
    if (n == 0) return SK_OK;
    if (!mu || !labels || !S || !cnt || !nk) return fail(SK_EINVAL, "sk_kmeans_step: NULL buffer");
    return cuda_status(sk::launch_kmeans(*ctx, idx, val, n, mu, K, labels, dist, S, cnt, nk, true,
                                         1, nullptr, as_stream(stream)),
                       "sk_kmeans_step");
}

sk_status sk_kmeans_step_delta(const sk_ctx *ctx, const int32_t *idx, const float *val,
                               int64_t n, const float *mu, int32_t K, int32_t *labels, float *dist,
                               double *S, int32_t *cnt, int64_t *nk, int64_t *changed,
                               void *stream) {
    sk_status st = kmeans_common("sk_kmeans_step_delta", ctx, idx, val, n, K);
    if (st != SK_OK) return st;
    if (n == 0) return SK_OK;
    if (!mu || !labels || !S || !cnt || !nk)
        return fail(SK_EINVAL, "sk_kmeans_step_delta: NULL buffer");
    return cuda_status(sk::launch_kmeans(*ctx, idx, val, n, mu, K, labels, dist, S, cnt, nk, true,
                                         2, changed, as_stream(stream)),
                       "sk_kmeans_step_delta");
}

sk_status sk_kmeans_step_auto(const sk_ctx *ctx, const int32_t *idx, const float *val,
                              int64_t n, const float *mu, int32_t K, int32_t *labels, float *dist,
                              double *S, int32_t *cnt, int64_t *nk, int64_t *state, int32_t first,
                              void *stream) {
    sk_status st = kmeans_common("sk_kmeans_step_auto", ctx, idx, val, n, K);
    if (st != SK_OK) return st;
    if (n == 0) return SK_OK;
    if (!mu || !labels || !S || !cnt || !nk || !state)
        return fail(SK_EINVAL, "sk_kmeans_step_auto: NULL buffer");
    return cuda_status(sk::launch_kmeans_auto(*ctx, idx, val, n, mu, K, labels, dist, S, cnt, nk,
                                              state, first ? 1 : 0, as_stream(stream)),
                       "sk_kmeans_step_auto");
}

sk_status sk_kmeans_finalize(const sk_ctx *ctx, int32_t K, const double *S, const int32_t *cnt,
                             float *mu, void *stream) {
    SK_CHECK_CTX(ctx);
    if (K < 1 || K > 256) return fail(SK_EINVAL, "sk_kmeans_finalize: K out of range");
    if (!S || !cnt || !mu) return fail(SK_EINVAL, "sk_kmeans_finalize: NULL buffer");
    return cuda_status(sk::launch_kmeans_finalize(*ctx, K, S, cnt, mu, as_stream(stream)),
                       "sk_kmeans_finalize");
}

sk_status sk_kmeans_reset(const sk_ctx *ctx, int32_t K, double *S, int32_t *cnt, int64_t *nk,
                          void *stream) {
    SK_CHECK_CTX(ctx);
    if (K < 1 || K > 256) return fail(SK_EINVAL, "sk_kmeans_reset: K out of range");
    if (!S || !cnt || !nk) return fail(SK_EINVAL, "sk_kmeans_reset: NULL buffer");
    const size_t KP = (size_t)K * ctx->pt;
    cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(S, 0, KP * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, KP * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(nk, 0, (size_t)K * sizeof(int64_t), s);
    return cuda_status(e, "sk_kmeans_reset");
}

sk_status sk_unmix(const sk_ctx *ctx, const float *in, int64_t r, float *out, void *stream) {
    SK_CHECK_CTX(ctx);
    if (r < 0) return fail(SK_EINVAL, "sk_unmix: r < 0");
    if (r == 0) return SK_OK;
    if (!in || !out) return fail(SK_EINVAL, "sk_unmix: NULL buffer");
    if (overlaps(in, (size_t)r * ctx->pt * 4, out, (size_t)r * ctx->p * 4))
        return fail(SK_EINVAL, "sk_unmix: in and out overlap");
    return cuda_status(sk::launch_unmix(*ctx, in, r, out, false, as_stream(stream)), "sk_unmix");
}

sk_status sk_unmix_f64(const sk_ctx *ctx, const double *in, int64_t r, double *out,
                       void *stream) {
    SK_CHECK_CTX(ctx);
    if (r < 0) return fail(SK_EINVAL, "sk_unmix_f64: r < 0");
    if (r == 0) return SK_OK;
    if (!in || !out) return fail(SK_EINVAL, "sk_unmix_f64: NULL buffer");
    if (overlaps(in, (size_t)r * ctx->pt * 8, out, (size_t)r * ctx->p * 8))
        return fail(SK_EINVAL, "sk_unmix_f64: in and out overlap");
    return cuda_status(sk::launch_unmix(*ctx, in, r, out, true, as_stream(stream)),
                       "sk_unmix_f64");
}

int64_t sk_kmeanspp_workspace_bytes(const sk_ctx *ctx, int64_t n) {
    if (!ctx || n < 0) return -1;
    return sk::kmeanspp_workspace(n);
}

sk_status sk_kmeanspp(const sk_ctx *ctx, const int32_t *idx, const float *val, int64_t n,
                      int32_t K, uint32_t restart, float *mu, int64_t *rows, void *work,
                      int64_t work_bytes, void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 1) return fail(SK_EINVAL, "sk_kmeanspp: n < 1");
    if (K < 1 || K > 256 || K > n) return fail(SK_EINVAL, "sk_kmeanspp: K = %d must be in [1, min(n, 256)]", K);
    if (n > ((int64_t)1 << 40)) return fail(SK_EUNSUPPORTED, "sk_kmeanspp: n too large");
    if (!idx || !val || !mu || !rows || !work) return fail(SK_EINVAL, "sk_kmeanspp: NULL buffer");
    if (work_bytes < sk::kmeanspp_workspace(n))
        return fail(SK_EINVAL, "sk_kmeanspp: workspace of %lld bytes needed",
                    (long long)sk::kmeanspp_workspace(n));
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return fail(SK_EINVAL, "sk_kmeanspp: workspace must be 256-byte aligned");
    return cuda_status(sk::launch_kmeanspp(*ctx, idx, val, n, K, restart, mu, rows, work,
                                           as_stream(stream)),
                       "sk_kmeanspp");
}

sk_status sk_kmeans_objective(const float *dist, int64_t n, double *J, void *stream) {
    if (n < 0) return fail(SK_EINVAL, "sk_kmeans_objective: n < 0");
    if (!J || (n > 0 && !dist)) return fail(SK_EINVAL, "sk_kmeans_objective: NULL buffer");
    return cuda_status(sk::launch_objective(dist, n, J, as_stream(stream)), "sk_kmeans_objective");
}

sk_status sk_kmeans_hk(const sk_ctx *ctx, int32_t K, const int32_t *cnt, const int64_t *nk,
                       double *dev, void *stream) {
    SK_CHECK_CTX(ctx);
    if (K < 1 || K > 65535) return fail(SK_EINVAL, "sk_kmeans_hk: K out of range");
    if (!cnt || !nk || !dev) return fail(SK_EINVAL, "sk_kmeans_hk: NULL buffer");
    return cuda_status(sk::launch_kmeans_hk(*ctx, K, cnt, nk, dev, as_stream(stream)),
                       "sk_kmeans_hk");
}

sk_status sk_kmeans2_assign(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                            const float *mu, int32_t K, int32_t *labels, float *dist,
                            void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_kmeans2_assign: n < 0");
    if (ldx < ctx->p) return fail(SK_EINVAL, "sk_kmeans2_assign: ldx < p");
    if (K < 1 || K > 256) return fail(SK_EINVAL, "sk_kmeans2_assign: K = %d must be in [1, 256]", K);
    if (n == 0) return SK_OK;
    if (!X || !mu || !labels) return fail(SK_EINVAL, "sk_kmeans2_assign: NULL buffer");
    return cuda_status(sk::launch_kmeans2_assign(*ctx, X, n, ldx, mu, K, labels, dist,
                                                 as_stream(stream)),
                       "sk_kmeans2_assign");
}

sk_status sk_kmeans2_sums(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                          const int32_t *labels1, int32_t K, double *sums, int64_t *counts,
                          void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_kmeans2_sums: n < 0");
    if (ldx < ctx->p) return fail(SK_EINVAL, "sk_kmeans2_sums: ldx < p");
    if (K < 1 || K > 256) return fail(SK_EINVAL, "sk_kmeans2_sums: K = %d must be in [1, 256]", K);
    if (n == 0) return SK_OK;
    if (!X || !labels1 || !sums || !counts) return fail(SK_EINVAL, "sk_kmeans2_sums: NULL buffer");
    if (n > ((int64_t)1 << 40)) return fail(SK_EUNSUPPORTED, "sk_kmeans2_sums: n too large");
    return cuda_status(sk::launch_kmeans2_sums(*ctx, X, n, ldx, labels1, K, sums, counts,
                                               as_stream(stream)),
                       "sk_kmeans2_sums");
}

sk_status sk_kmeans2_finalize(const sk_ctx *ctx, int32_t K, const double *sums,
                              const int64_t *counts, float *mu, void *stream) {
    SK_CHECK_CTX(ctx);
    if (K < 1 || K > 256) return fail(SK_EINVAL, "sk_kmeans2_finalize: K out of range");
    if (!sums || !counts || !mu) return fail(SK_EINVAL, "sk_kmeans2_finalize: NULL buffer");
    return cuda_status(sk::launch_kmeans2_finalize(*ctx, K, sums, counts, mu, as_stream(stream)),
                       "sk_kmeans2_finalize");
}

sk_status sk_mean_accumulate(const sk_ctx *ctx, const int32_t *idx, const float *val,
                             int64_t n, double *sums, void *stream) {
    SK_CHECK_CTX(ctx);
    if (n < 0) return fail(SK_EINVAL, "sk_mean_accumulate: n < 0");
    if (n == 0) return SK_OK;
    if (!idx || !val || !sums) return fail(SK_EINVAL, "sk_mean_accumulate: NULL buffer");
    return cuda_status(sk::launch_mean_accumulate(*ctx, idx, val, n, sums, as_stream(stream)),
                       "sk_mean_accumulate");
}

sk_status sk_mean_finalize(const sk_ctx *ctx, const double *sums, int64_t n_total, double *mean,
                           void *stream) {
    SK_CHECK_CTX(ctx);
    if (n_total < 1) return fail(SK_EINVAL, "sk_mean_finalize: n_total < 1");
    if (!sums || !mean) return fail(SK_EINVAL, "sk_mean_finalize: NULL buffer");
    return cuda_status(sk::launch_mean_finalize(*ctx, sums, n_total, mean, as_stream(stream)),
                       "sk_mean_finalize");
}

static cudaError_t time_call_ms(cudaStream_t s, float &ms, cudaError_t (*fn)(void *), void *arg) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    e = fn(arg);  // untimed first call (launch attributes, caches)
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = fn(arg);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

namespace {
struct GramCall {
    sk_ctx *c;
    int mode;
    const int32_t *idx;
    const float *val;
    int64_t n;
    double *G;
    void *work;
    cudaStream_t s;
};
cudaError_t gram_call(void *p) {
    GramCall *g = static_cast<GramCall *>(p);
    return sk::launch_gram_tc(*g->c, g->mode, g->idx, g->val, g->n, g->G, g->work, g->s);
}
struct CompressCall {
    sk_ctx *c;
    const float *X;
    int64_t n, ldx;
    int32_t *idx;
    float *val;
    cudaStream_t s;
};
cudaError_t compress_call(void *p) {
    CompressCall *q = static_cast<CompressCall *>(p);
    return sk::launch_compress(*q->c, q->X, q->n, q->ldx, 0, q->idx, q->val, nullptr, q->s);
}
}  // namespace

sk_status sk_autotune_gram(sk_ctx *ctx, int mode, const int32_t *idx, const float *val, int64_t n,
                           double *G, void *work, int64_t work_bytes, void *stream,
                           int32_t *tile_n, int32_t *split_mult) {
    SK_CHECK_CTX(ctx);
    if (mode != SK_GRAM_BF16 && mode != SK_GRAM_BF16X3)
        return fail(SK_EINVAL, "sk_autotune_gram: tensor-core modes only");
    if (ctx->pt < 256) return fail(SK_EUNSUPPORTED, "sk_autotune_gram: needs pt >= 256");
    if (n < 1 || !idx || !val || !G || !work) return fail(SK_EINVAL, "sk_autotune_gram: bad argument");
    if (work_bytes < sk::gram_tc_workspace(*ctx, n))
        return fail(SK_EINVAL, "sk_autotune_gram: workspace too small");
    GramCall g{ctx, mode, idx, val, n, G, work, as_stream(stream)};
    const int cand_n[2] = {256, 128}, cand_s[2] = {1, 2};
    float best = 1e30f;
    int bn = 256, bs = 1;
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            ctx->gram_n = cand_n[a];
            ctx->split_mult = cand_s[c];
            float ms = 0.f;
            cudaError_t e = time_call_ms(g.s, ms, gram_call, &g);
            if (e != cudaSuccess) return cuda_status(e, "sk_autotune_gram");
            if (ms < best) {
                best = ms;
                bn = cand_n[a];
                bs = cand_s[c];
            }
        }
    ctx->gram_n = bn;
    ctx->split_mult = bs;
    if (tile_n) *tile_n = bn;
    if (split_mult) *split_mult = bs;
    g_msg[0] = 0;
    return SK_OK;
}

sk_status sk_autotune_compress(sk_ctx *ctx, const float *X, int64_t n, int64_t ldx, int32_t *idx,
                               float *val, void *stream, int32_t *ctas_per_sm) {
    SK_CHECK_CTX(ctx);
    if (n < 1 || ldx < ctx->p || !X || !idx || !val)
        return fail(SK_EINVAL, "sk_autotune_compress: bad argument");
    CompressCall q{ctx, X, n, ldx, idx, val, as_stream(stream)};
    float best = 1e30f;
    int bc = 0;
    for (int c : {0, 1}) {
        ctx->compress_ctas = c;
        float ms = 0.f;
        cudaError_t e = time_call_ms(q.s, ms, compress_call, &q);
        if (e != cudaSuccess) return cuda_status(e, "sk_autotune_compress");
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    ctx->compress_ctas = bc;
    if (ctas_per_sm) *ctas_per_sm = bc;
    g_msg[0] = 0;
    return SK_OK;
}

sk_status sk_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_status(e, "sk_device_status");
    unsigned int flag = 0;
    e = sk::take_device_error(&flag);
    if (e != cudaSuccess) return cuda_status(e, "sk_device_status");
    if (flag) {
        return fail(SK_ETIMEOUT, "sk_device_status: a bounded device wait ran out (flag 0x%x)",
                    flag);
    }
    g_msg[0] = 0;
    return SK_OK;
}

const char *sk_last_error(void) { return g_msg; }

sk_status sk_debug_set_wait_cycles(int64_t cycles) {
    if (cycles < 0) return fail(SK_EINVAL, "sk_debug_set_wait_cycles: cycles must be >= 0");
    sk::g_wait_cycles.store(cycles == 0 ? sk::kDefaultWaitCycles : (long long)cycles,
                            std::memory_order_relaxed);
    g_msg[0] = 0;
    return SK_OK;
}

}  // extern "C"
