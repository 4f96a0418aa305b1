// batch.cu -- the host plan for many data sets in one launch per stage
// (include/sk.h, sk_batch_*): validation, the per data set handles, and the
// device tables of the persistent compress, the multi-data-set Gram and the
// persistent K-means kernels (built by the kernel files, uploaded once).
#include <cstdarg>
#include <cstdio>
#include <new>
#include <vector>

#include "sk_internal.cuh"

struct sk_batch {
    std::vector<sk_ctx> ctxs;
    std::vector<sk_batch_item> items;
    int nd = 0;
    int mode = 0;
    int units_per_group = 64;  // compress task size (units per row group)
    int gram_n = 256;          // Gram tile width of the multi-data-set launch
    size_t max_table = 0;      // largest table over the autotuner's candidates
    std::vector<unsigned char> table;
    sk::CompressBatchInfo ci{};
    sk::GramBatchInfo gi{};
    sk::KmeansBatchInfo ki{};
    unsigned char *dev = nullptr;
};

// (Re)builds the device tables of a plan for the given launch shapes.
static cudaError_t build_tables(sk_batch *B, int units_per_group, int gram_n) {
    const int nd = B->nd;
    std::vector<sk::BatchRows> rows((size_t)nd);
    std::vector<sk::BatchGram> grams((size_t)nd);
    std::vector<sk::BatchKmeans> kms((size_t)nd);
    for (int d = 0; d < nd; ++d) {
        const sk_batch_item &it = B->items[d];
        rows[d] = sk::BatchRows{it.X, it.n, it.ldx, it.row0, it.idx, it.val};
        grams[d] = sk::BatchGram{it.idx, it.val, it.n, it.G, it.gram_work};
        kms[d] = sk::BatchKmeans{it.idx, it.val, it.n,   it.K,  it.mu,
                                 it.mu_t, it.labels, it.S, it.cnt, it.nk, it.changed};
        B->ctxs[d].gram_n = gram_n;
    }
    B->table.clear();
    cudaError_t e = sk::compress_batch_build(B->ctxs.data(), rows.data(), nd, units_per_group,
                                             B->table, B->ci);
    if (e == cudaSuccess)
        e = sk::gram_batch_build(B->ctxs.data(), grams.data(), nd, B->mode, B->table, B->gi);
    if (e == cudaSuccess) e = sk::kmeans_batch_build(B->ctxs.data(), kms.data(), nd, B->table, B->ki);
    if (e == cudaSuccess) {
        B->units_per_group = units_per_group;
        B->gram_n = gram_n;
    }
    return e;
}

// Milliseconds of one call of fn (after one untimed call), on the stream.
template <typename F>
static cudaError_t time_ms(F fn, cudaStream_t s, float &ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

static const int kUnitsCand[] = {32, 128};
static const int kGramNCand[] = {256, 128};

namespace {

thread_local char g_bmsg[512] = {0};

sk_status bfail(sk_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_bmsg, sizeof(g_bmsg), fmt, ap);
    va_end(ap);
    sk::set_last_error(g_bmsg);
    return st;
}

sk_status bcuda(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return SK_OK;
    return bfail(SK_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

cudaStream_t bstream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

sk_status sk_batch_create(sk_batch **b, const sk_batch_item *items, int32_t nd,
                          int32_t gram_mode) {
    if (!b) return bfail(SK_EINVAL, "sk_batch_create: out-pointer is NULL");
    *b = nullptr;
    if (nd < 1 || !items) return bfail(SK_EINVAL, "sk_batch_create: no items");
    if (gram_mode != SK_GRAM_BF16 && gram_mode != SK_GRAM_BF16X3)
        return bfail(SK_EINVAL, "sk_batch_create: gram_mode must be SK_GRAM_BF16 or SK_GRAM_BF16X3");
    std::vector<sk_ctx> ctxs((size_t)nd);
    for (int d = 0; d < nd; ++d) {
        const sk_batch_item &it = items[d];
        if (it.p < 4 || it.p > 8192)
            return bfail(SK_EUNSUPPORTED, "sk_batch_create: item %d: p = %lld outside [4, 8192]", d,
                         (long long)it.p);
        int L = 0;
        while ((1LL << L) < it.p) ++L;
        const int64_t pt = 1LL << L;
        if (it.m < 2 || it.m > pt)
            return bfail(SK_EINVAL, "sk_batch_create: item %d: m must be in [2, pt]", d);
        if (pt < 256)
            return bfail(SK_EUNSUPPORTED, "sk_batch_create: item %d: pt = %lld < 256", d,
                         (long long)pt);
        if (it.flags & SK_FLAG_DCT)
            return bfail(SK_EUNSUPPORTED,
                         "sk_batch_create: item %d: the DCT preconditioner is not batched", d);
        if (it.flags & ~(uint32_t)SK_FLAG_NO_PRECONDITION)
            return bfail(SK_EINVAL, "sk_batch_create: item %d: unknown flags", d);
        if (it.n < 0 || it.ldx < it.p || it.row0 < 0)
            return bfail(SK_EINVAL, "sk_batch_create: item %d: bad n / ldx / row0", d);
        if (it.K < 1 || it.K > 64)
            return bfail(SK_EUNSUPPORTED, "sk_batch_create: item %d: K = %d outside [1, 64]", d,
                         it.K);
        if (it.n > 0 && (!it.X || !it.idx || !it.val || !it.G || !it.gram_work || !it.mu ||
                         !it.labels || !it.S || !it.cnt || !it.nk))
            return bfail(SK_EINVAL, "sk_batch_create: item %d: NULL buffer", d);
        sk_ctx &c = ctxs[d];
        c.p = it.p;
        c.pt = pt;
        c.log2pt = L;
        c.m = it.m;
        c.seed = it.seed;
        c.flags = it.flags;
        c.gram_n = 0;
        c.split_mult = 0;
        c.compress_ctas = 0;
        if (it.n > 0 && !sk::compress_batchable(c, it.X, it.ldx))
            return bfail(SK_EUNSUPPORTED,
                         "sk_batch_create: item %d: rows must be 16-byte aligned with p, ldx "
                         "multiples of 4", d);
        if (it.n > 0 && it.gram_work_bytes < sk::gram_tc_workspace(c, it.n))
            return bfail(SK_EINVAL, "sk_batch_create: item %d: gram_work of %lld bytes needed", d,
                         (long long)sk::gram_tc_workspace(c, it.n));
        if (it.n > 0 && (reinterpret_cast<uintptr_t>(it.gram_work) & 255) != 0)
            return bfail(SK_EINVAL, "sk_batch_create: item %d: gram_work must be 256-byte aligned",
                         d);
    }
    sk_batch *B = new (std::nothrow) sk_batch;
    if (!B) return bfail(SK_ENOMEM, "sk_batch_create: out of host memory");
    B->ctxs = ctxs;
    B->items.assign(items, items + nd);
    B->nd = nd;
    B->mode = gram_mode;
    // the autotuner's candidates may need a larger table than the default
    cudaError_t e = cudaSuccess;
    for (int u : kUnitsCand)
        for (int gn : kGramNCand) {
            if (e == cudaSuccess) e = build_tables(B, u, gn);
            if (e == cudaSuccess && B->table.size() > B->max_table) B->max_table = B->table.size();
        }
    if (e == cudaSuccess) e = build_tables(B, 64, 256);
    if (e == cudaSuccess && B->table.size() > B->max_table) B->max_table = B->table.size();
    if (e != cudaSuccess) {
        delete B;
        if (e == cudaErrorInvalidValue)
            return bfail(SK_EUNSUPPORTED, "sk_batch_create: items need different launch shapes");
        return bcuda(e, "sk_batch_create");
    }
    *b = B;
    return SK_OK;
}

int64_t sk_batch_workspace_bytes(const sk_batch *b) {
    return b ? (int64_t)b->max_table : -1;
}

sk_status sk_batch_upload(sk_batch *b, void *work, int64_t work_bytes, void *stream) {
    if (!b || !work) return bfail(SK_EINVAL, "sk_batch_upload: NULL argument");
    if (work_bytes < (int64_t)b->table.size())
        return bfail(SK_EINVAL, "sk_batch_upload: %lld bytes needed", (long long)b->table.size());
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return bfail(SK_EINVAL, "sk_batch_upload: work must be 256-byte aligned");
    cudaError_t e = cudaMemcpyAsync(work, b->table.data(), b->table.size(), cudaMemcpyHostToDevice,
                                    bstream(stream));
    if (e != cudaSuccess) return bcuda(e, "sk_batch_upload");
    // the host table is pageable: the copy has read it when the call returns
    b->dev = static_cast<unsigned char *>(work);
    return SK_OK;
}

static sk_status need_upload(const sk_batch *b, const char *fn) {
    if (!b) return bfail(SK_EINVAL, "%s: batch is NULL", fn);
    if (!b->dev) return bfail(SK_EINVAL, "%s: call sk_batch_upload first", fn);
    return SK_OK;
}

sk_status sk_batch_compress(const sk_batch *b, void *stream) {
    sk_status st = need_upload(b, "sk_batch_compress");
    if (st != SK_OK) return st;
    return bcuda(sk::compress_batch_launch(b->ci, b->dev, bstream(stream)), "sk_batch_compress");
}

sk_status sk_batch_cov_reset(const sk_batch *b, void *stream) {
    if (!b) return bfail(SK_EINVAL, "sk_batch_cov_reset: batch is NULL");
    for (int d = 0; d < b->nd; ++d) {
        if (b->items[d].n == 0) continue;
        cudaError_t e = cudaMemsetAsync(b->items[d].G, 0,
                                        (size_t)b->ctxs[d].pt * b->ctxs[d].pt * sizeof(double),
                                        bstream(stream));
        if (e != cudaSuccess) return bcuda(e, "sk_batch_cov_reset");
    }
    return SK_OK;
}

sk_status sk_batch_cov_accumulate(const sk_batch *b, void *stream) {
    sk_status st = need_upload(b, "sk_batch_cov_accumulate");
    if (st != SK_OK) return st;
    return bcuda(sk::gram_batch_launch(b->gi, b->dev, bstream(stream)), "sk_batch_cov_accumulate");
}

sk_status sk_batch_kmeans_reset(const sk_batch *b, void *stream) {
    sk_status st = need_upload(b, "sk_batch_kmeans_reset");
    if (st != SK_OK) return st;
    return bcuda(sk::kmeans_batch_launch(b->ki, b->dev, 0, bstream(stream)), "sk_batch_kmeans_reset");
}

sk_status sk_batch_kmeans_step(const sk_batch *b, int32_t incremental, void *stream) {
    sk_status st = need_upload(b, "sk_batch_kmeans_step");
    if (st != SK_OK) return st;
    if (incremental != 0 && incremental != 1)
        return bfail(SK_EINVAL, "sk_batch_kmeans_step: incremental must be 0 or 1");
    return bcuda(sk::kmeans_batch_launch(b->ki, b->dev, incremental ? 2 : 1, bstream(stream)),
                 "sk_batch_kmeans_step");
}

sk_status sk_batch_kmeans_finalize(const sk_batch *b, void *stream) {
    sk_status st = need_upload(b, "sk_batch_kmeans_finalize");
    if (st != SK_OK) return st;
    return bcuda(sk::kmeans_batch_launch(b->ki, b->dev, 3, bstream(stream)),
                 "sk_batch_kmeans_finalize");
}

sk_status sk_batch_autotune(sk_batch *b, void *work, int64_t work_bytes, void *stream,
                            int32_t *units_per_group, int32_t *gram_tile_n) {
    if (!b || !work) return bfail(SK_EINVAL, "sk_batch_autotune: NULL argument");
    if (work_bytes < (int64_t)b->max_table)
        return bfail(SK_EINVAL, "sk_batch_autotune: %lld bytes needed", (long long)b->max_table);
    cudaStream_t s = bstream(stream);
    float best = 1e30f;
    int best_u = b->units_per_group, best_n = b->gram_n;
    for (int u : kUnitsCand) {
        cudaError_t e = build_tables(b, u, best_n);
        sk_status st = e == cudaSuccess ? sk_batch_upload(b, work, work_bytes, stream) : bcuda(e, "sk_batch_autotune");
        if (st != SK_OK) return st;
        float ms = 0.f;
        e = time_ms([&] { return sk::compress_batch_launch(b->ci, b->dev, s); }, s, ms);
        if (e != cudaSuccess) return bcuda(e, "sk_batch_autotune (compress)");
        if (ms < best) {
            best = ms;
            best_u = u;
        }
    }
    best = 1e30f;
    for (int gn : kGramNCand) {
        cudaError_t e = build_tables(b, best_u, gn);
        sk_status st = e == cudaSuccess ? sk_batch_upload(b, work, work_bytes, stream) : bcuda(e, "sk_batch_autotune");
        if (st != SK_OK) return st;
        float ms = 0.f;
        e = time_ms([&] { return sk::gram_batch_launch(b->gi, b->dev, s); }, s, ms);
        if (e != cudaSuccess) return bcuda(e, "sk_batch_autotune (Gram)");
        if (ms < best) {
            best = ms;
            best_n = gn;
        }
    }
    cudaError_t e = build_tables(b, best_u, best_n);
    if (e != cudaSuccess) return bcuda(e, "sk_batch_autotune");
    sk_status st = sk_batch_upload(b, work, work_bytes, stream);
    if (st != SK_OK) return st;
    if (units_per_group) *units_per_group = best_u;
    if (gram_tile_n) *gram_tile_n = best_n;
    return SK_OK;
}

void sk_batch_destroy(sk_batch *b) { delete b; }

}  // extern "C"
