/*
 * sk.h -- C ABI of the GB300 library for preconditioned data sparsification
 * (Pourkamali-Anaraki & Becker, "Preconditioned Data Sparsification for Big
 * Data with Applications to PCA and K-means").
 *
 * Conventions shared by every entry point:
 *  - Samples are rows: X is n x p, row-major float32 with leading dimension
 *    ldx >= p (the paper's p x n matrix with samples as columns, same bytes).
 *  - pt ("p tilde") is the smallest power of two >= p.  Samples are
 *    zero-padded to pt before the Walsh-Hadamard transform; all sampling
 *    and rescaling uses pt in place of the paper's p.  Supported: 1 <= p <= 8192.
 *    With SK_FLAG_DCT (sk_init_ex) pt = p: the DCT needs no padding.
 *  - Every pointer argument named as device memory must be device memory the
 *    caller owns (for example torch storage); the library never frees it and
 *    keeps no reference to it after the call returns.  Host pointers are
 *    named as such.
 *  - Every call that takes `stream` enqueues asynchronous work on that CUDA
 *    stream (a cudaStream_t passed as void*; NULL is the legacy default
 *    stream) and returns without synchronising.
 *  - Argument errors are found on the host before any launch and return
 *    SK_EINVAL (or SK_EUNSUPPORTED for a valid but unsupported shape); nothing
 *    is enqueued.  A CUDA launch error returns SK_ECUDA.  sk_last_error()
 *    gives a message for the calling thread's most recent failure.
 *  - Device-side waits in the library's own kernels are bounded; a wait that
 *    runs out sets a device error word and the kernel returns early.
 *    sk_device_status() reports (and clears) it as SK_ETIMEOUT.
 *  - No call throws; no call allocates device memory except where stated.
 *
 * Random-number spec (bit-exact; the same text is implemented independently
 * by the CPU oracle):  Philox4x32-10 (Salmon et al., SC'11) with key =
 * (seed_lo, seed_hi).  Sign D_j = -1 iff bit (j mod 32) of word (j/32) mod 4
 * of Philox(ctr = (j/128, 0, 0, 0x5349474E)) is set.  The mask of global row
 * r draws words w = 0,1,... = word (w mod 4) of Philox(ctr = (w/4, r_lo,
 * r_hi, 0x4D41534B)); U(s) is Lemire's multiply-shift with rejection; the
 * mask is partial Fisher-Yates: for t = 0..m-1, k = t + U(pt - t), swap
 * a[t], a[k] of the virtual identity array, emit a[t].
 */
#ifndef SK_H
#define SK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sk_status {
    SK_OK = 0,
    SK_EINVAL = 1,        /* invalid argument (nothing enqueued) */
    SK_ENOMEM = 2,        /* allocation refused */
    SK_ECUDA = 3,         /* CUDA runtime or launch error */
    SK_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
    SK_EUNSUPPORTED = 5   /* valid request outside the supported shapes */
} sk_status;

/* Gram precision modes for sk_cov_accumulate. */
enum {
    SK_GRAM_FP32 = 0,   /* FP32 products, shared-memory scatter, FP64 flush */
    SK_GRAM_BF16 = 1,   /* BF16 x BF16 -> FP32 on tcgen05 tensor cores */
    SK_GRAM_BF16X3 = 2  /* split-BF16 hi/lo, three tcgen05 products */
};

/* Flags for sk_init_ex. */
enum {
    /* Ablation without preconditioning (H = D = I; the "no preconditioning"
     * comparison of Sec. VII): sk_compress samples the zero-padded raw row,
     * val = [x_i; 0][Omega], sk_precondition pads only, and sk_unmix /
     * sk_unmix_f64 truncate to p.  Estimators and K-means are unchanged. */
    SK_FLAG_NO_PRECONDITION = 1,
    /* The DCT preconditioner (Sec. III: H a DCT matrix; the paper's choice
     * for p that is not a power of two, used in its Sec. VII big-data runs):
     * H is the orthonormal DCT-II of length p, with no zero padding, so
     * pt = p and the masks, the estimators' rescaling and every pt-sized
     * buffer use p.  sk_unmix / sk_unmix_f64 apply D H^T (the DCT-III).
     * Requires an even p whose half has no prime factor above 13 (for
     * example 784 = 2 * 392 = 2 * 8 * 7 * 7, or 1000); otherwise
     * SK_EUNSUPPORTED.  Excludes SK_FLAG_NO_PRECONDITION; not accepted by
     * sk_batch_create (SK_EUNSUPPORTED). */
    SK_FLAG_DCT = 2
};

/* Opaque host-side handle: p, pt, m, the seed and the flags.  Holds no
 * device memory. */
typedef struct sk_ctx sk_ctx;

/* Creates a handle for samples of dimension p keeping m of pt entries per
 * sample, with all randomness keyed by seed.  The paper's problem statement
 * (Sec. VI-B, Algorithm 1 input: X, K, gamma = m/p).  Requires 1 <= p <= 8192
 * and 1 <= m <= pt.  *ctx receives the handle (host memory, freed by
 * sk_destroy).  Returns SK_EINVAL / SK_EUNSUPPORTED / SK_ENOMEM. */
sk_status sk_init(sk_ctx **ctx, int64_t p, int64_t m, uint64_t seed);

/* sk_init with flags (a bitwise OR of SK_FLAG_*; 0 is sk_init).  Unknown
 * bits return SK_EINVAL. */
sk_status sk_init_ex(sk_ctx **ctx, int64_t p, int64_t m, uint64_t seed, uint32_t flags);

/* The flags of a handle (0 for NULL). */
uint32_t sk_flags(const sk_ctx *ctx);

/* Frees a handle from sk_init (NULL is ignored). */
void sk_destroy(sk_ctx *ctx);

/* pt of a handle, or -1 for NULL. */
int64_t sk_ptilde(const sk_ctx *ctx);

/* One-pass compression (Algorithm 1, lines "Y <- HDX" and "w_i = R_i R_i^T
 * y_i"; Sec. III Eq. (ROS)): for local rows i = 0..n-1 with global row
 * r = row0 + i, y_i = H D [x_i; 0] (orthonormal Sylvester H) and the ELL
 * output keeps the m entries of the mask of row r in draw order:
 *   idx[i*m + t] = Omega_r[t]  (int32, device, n*m),
 *   val[i*m + t] = y_i[Omega_r[t]]  (float32, device, n*m).
 * X: device, n x p with leading dimension ldx >= p.  row0 >= 0 lets a chunked
 * stream reproduce a single call exactly.  n = 0 is a no-op. */
sk_status sk_compress(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                      int64_t row0, int32_t *idx, float *val, void *stream);

/* Dense preconditioning only (Sec. III, Eq. (ROS)): Y[i*pt + j] = (H D
 * [x_i; 0])_j, Y device n x pt float32.  Used for K-means starting centres and
 * the second pass of Algorithm 2. */
sk_status sk_precondition(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                          float *Y, void *stream);

/* Covariance accumulation (Sec. V): G += sum_i w_i w_i^T over the n ELL rows
 * (idx, val as produced by sk_compress), w_i the pt-vector with val at idx.
 * G: device float64 pt x pt, caller-zeroed before the first call; only its
 * upper triangle (j <= k) is defined after the call, the strict lower
 * triangle holds unspecified partial sums.  mode is SK_GRAM_*.  The tensor-core
 * modes (pt >= 128) need a device workspace `work` of at least
 * sk_cov_workspace_bytes(ctx, mode, n) bytes, 256-byte aligned, that they
 * overwrite (the rows' entries regrouped by 128-column block); SK_GRAM_FP32
 * needs none (work may be NULL).  Repeated calls on chunks accumulate; the
 * result does not depend on the chunking beyond floating-point summation
 * order. */
sk_status sk_cov_accumulate(const sk_ctx *ctx, int mode, const int32_t *idx,
                            const float *val, int64_t n, double *G, void *work,
                            int64_t work_bytes, void *stream);

/* Workspace bytes sk_cov_accumulate needs for n rows in the given mode (0 for
 * SK_GRAM_FP32; -1 for invalid arguments). */
int64_t sk_cov_workspace_bytes(const sk_ctx *ctx, int mode, int64_t n);

/* Zeroes a pt x pt float64 Gram accumulator G (device) on the stream. */
sk_status sk_cov_reset(const sk_ctx *ctx, double *G, void *stream);

/* Unbiased covariance estimate C_n (Sec. V): with P = pt,
 *   C_emp-hat = P(P-1)/(m(m-1)) * G / n_total,
 *   C_n = C_emp-hat - (P-m)/(P-1) diag(C_emp-hat),
 * written as a full symmetric pt x pt float64 matrix C (device), reading the
 * upper triangle of G (device).  Requires m >= 2 (Thm. B1) and n_total >= 1.
 * G and C must not overlap. */
sk_status sk_cov_finalize(const sk_ctx *ctx, const double *G, int64_t n_total,
                          double *C, void *stream);

/* Centred covariance estimate: the uncentred C_n of Sec. V combined with the
 * sample-mean estimate xbar of Sec. IV (sk_mean_finalize of the same rows),
 *   C_c = C_n - xbar xbar^T + B(C_n) / n_total,
 *   B(A)_jj = ((P-m)/m) A_jj,  B(A)_jk = -((P-m)/(m (P-1))) A_jk (j != k),
 * with P = pt.  B(C_emp)/n is the covariance of xbar over the masks (from the
 * keep probabilities m/P and m(m-1)/(P(P-1)) of Thm. B1), so the correction
 * makes C_c unbiased for the centred second moment C_emp - ybar ybar^T (the
 * plain plug-in C_n - xbar xbar^T is not).  G: the Gram accumulator of the
 * n_total rows (upper triangle read, as sk_cov_finalize); mean: device float64
 * pt; C: device float64 pt x pt (full symmetric), overlapping neither.
 * Requires m >= 2 and n_total >= 1. */
sk_status sk_cov_finalize_centred(const sk_ctx *ctx, const double *G, const double *mean,
                                  int64_t n_total, double *C, void *stream);

/* Top-k principal subspace of the symmetric pt x pt estimate C (device
 * float64), Sec. V PCA: eigenvalues (device float64, k, descending) and
 * eigenvectors (device float64, pt x k column-major, i.e. vector c at
 * U[c*pt .. c*pt+pt)) by block subspace iteration with Rayleigh-Ritz to
 * float64 accuracy on the device (the last two products with C and the
 * Rayleigh-Ritz product in double-float arithmetic, pairs of float32 with
 * error-free products, about 2^-44 relative; the final basis and
 * eigenproblem in float64; the earlier products in float32 and the
 * intermediate re-orthonormalisations, which do not change the iterated
 * subspace, from float32 factors).  iters is the
 * number of iterations (0 is taken as 1); the subspace error shrinks by about
 * (lambda_{b+1} / lambda_k)^iters with b = min(pt, 64, max(k + 8, 2k)).
 * work is a device float64 scratch buffer of sk_cov_topk_workspace(pt, k)
 * doubles.  C must be 16-byte aligned (SK_EINVAL otherwise).  Requires
 * 1 <= k <= min(pt, 64). */
sk_status sk_cov_topk(const sk_ctx *ctx, const double *C, int32_t k, int32_t iters,
                      double *evals, double *U, double *work, void *stream);
int64_t sk_cov_topk_workspace(int64_t pt, int32_t k);

/* sk_cov_topk for callers that cannot allocate device memory: the same
 * computation, with its scratch in a fixed array of 4 MiB (524,288 doubles)
 * inside the library instead of a caller workspace.  (No counterpart in the
 * paper; this is a deployment convenience.)  Meant for code that may not call
 * cudaMalloc or any allocating library routine: an application whose device
 * memory is owned entirely by its own caching allocator, or a latency-critical
 * loop that cannot afford an allocation's implicit device synchronisation.
 * The call allocates nothing; the caller still provides C, evals and U as for
 * sk_cov_topk.  Shapes whose scratch, sk_cov_topk_workspace(pt, k), exceeds
 * 524,288 doubles (for example pt = 8192 with k > 15) are rejected with
 * SK_EUNSUPPORTED before anything is enqueued.  Every GPU that loads the
 * library holds the array until the process exits.  Every call looks up the
 * array's device address for the current device (a query that allocates
 * nothing), so the address stays right after a device reset or a new context;
 * the first call on a device may load the library's device code, so make that
 * first call before any stream capture.  All calls share the one array
 * and leave their intermediate results in it: calls whose work overlaps on the
 * GPU (different streams without ordering) race and must not be issued. */
sk_status sk_cov_topk_static(const sk_ctx *ctx, const double *C, int32_t k, int32_t iters,
                             double *evals, double *U, void *stream);

/* Sparsified K-means assignment (Sec. VI-B, Eq. (assignments)): for each
 * ELL row i, labels[i] = argmin_k sum_t (val[i,t] - mu[k, idx[i,t]])^2 with
 * ties going to the smallest k, the restricted squared distance computed
 * directly in float32.  mu: device K x pt float32 (the preconditioned-domain
 * centres mu').  labels: device int32 n.  dist: device float32 n or NULL
 * (receives the winning distance).  1 <= K <= 256. */
sk_status sk_kmeans_assign(const sk_ctx *ctx, const int32_t *idx, const float *val,
                           int64_t n, const float *mu, int32_t K, int32_t *labels,
                           float *dist, void *stream);

/* Sparsified K-means centre sums (Sec. VI-B, Eq. (mu_update_one)):
 * accumulates S[k*pt + j] += sum of val over rows of cluster k that sampled
 * j, cnt[k*pt + j] += n_k^(j) (how often j was sampled in cluster k) and
 * nk[k] += rows in cluster k.  S: device float64 K x pt; cnt: device int32
 * K x pt; nk: device int64 K; all caller-zeroed before the first call. */
sk_status sk_kmeans_update(const sk_ctx *ctx, const int32_t *idx, const float *val,
                           const int32_t *labels, int64_t n, int32_t K, double *S,
                           int32_t *cnt, int64_t *nk, void *stream);

/* Fused one-pass iteration body: assignment against mu (as
 * sk_kmeans_assign) and, in the same pass over the ELL rows, the sums of
 * sk_kmeans_update under the new labels.  Same argument meanings. */
sk_status sk_kmeans_step(const sk_ctx *ctx, const int32_t *idx, const float *val,
                         int64_t n, const float *mu, int32_t K, int32_t *labels,
                         float *dist, double *S, int32_t *cnt, int64_t *nk,
                         void *stream);

/* Fused pass with incremental sums: assignment against mu (as
 * sk_kmeans_assign) and an exact update of the running sums.  On entry,
 * labels (device int32 n) hold each row's previous cluster (or -1) and S, cnt,
 * nk hold the sums of Eq. (mu_update_one) for those labels (as left by
 * sk_kmeans_step or a previous call); a row whose label changes from c to c'
 * is subtracted from cluster c and added to c'.  On return labels, S, cnt, nk
 * describe the new assignment.  changed (device int64 scalar, or NULL) is
 * incremented by the number of rows whose label changed.  After the first
 * pass few labels change, so later passes do little more than the
 * assignment. */
sk_status sk_kmeans_step_delta(const sk_ctx *ctx, const int32_t *idx, const float *val,
                               int64_t n, const float *mu, int32_t K, int32_t *labels,
                               float *dist, double *S, int32_t *cnt, int64_t *nk,
                               int64_t *changed, void *stream);

/* Adaptive iteration body (Algorithm 1 loop; the sums of Eq.
 * (mu_update_one)): assignment against mu and an update of S, cnt, nk that
 * is either a full rebuild (as sk_kmeans_reset + sk_kmeans_step) or
 * incremental (as sk_kmeans_step_delta), chosen on the device so that the
 * call can sit in a captured CUDA graph.  state: device int64[3], caller-
 * owned; state[0] carries from one pass to the next the number of rows
 * whose label changed, state[1] receives the kind of pass that ran (1 full
 * rebuild, 2 incremental), state[2] is scratch that every pass leaves at 0
 * (a first pass sets it).  The pass is a full rebuild if first != 0 or
 * state[0] > n / 12 (many moved rows: moving each one's entries with global
 * atomics would cost more than rebuilding the sums in shared memory), else
 * incremental.  On return labels, S, cnt, nk describe the new assignment
 * and state[0] holds this pass's count of changed rows (on a first pass,
 * counted against whatever labels held).  The sums are the same either way,
 * up to the order of float64 additions.  Other arguments as
 * sk_kmeans_step_delta; dist may be NULL.  Two kernel launches where K <= 32
 * and the centre table fits shared memory (the assignment kernel makes the
 * choice), else four. */
sk_status sk_kmeans_step_auto(const sk_ctx *ctx, const int32_t *idx, const float *val,
                              int64_t n, const float *mu, int32_t K, int32_t *labels,
                              float *dist, double *S, int32_t *cnt, int64_t *nk,
                              int64_t *state, int32_t first, void *stream);

/* Centre update (Eq. (mu_update_two)): mu[k*pt + j] = S/cnt where cnt > 0;
 * a coordinate no row of cluster k sampled cannot be estimated and keeps its
 * previous value (an empty cluster keeps its whole centre).  mu: device
 * float32 K x pt, updated in place. */
sk_status sk_kmeans_finalize(const sk_ctx *ctx, int32_t K, const double *S,
                             const int32_t *cnt, float *mu, void *stream);

/* Zeroes the K-means sums S (float64 K x pt), cnt (int32 K x pt) and nk
 * (int64 K), all device, on the stream: the start of one accumulation pass. */
sk_status sk_kmeans_reset(const sk_ctx *ctx, int32_t K, double *S, int32_t *cnt, int64_t *nk,
                          void *stream);

/* Un-mixing (Eq. (mu-mu'), Algorithm 1 last step): out_i = first p entries
 * of (HD)^T in_i = D H in_i for r rows.  in: device float32 r x pt; out:
 * device float32 r x p.  in and out must not overlap. */
sk_status sk_unmix(const sk_ctx *ctx, const float *in, int64_t r, float *out,
                   void *stream);

/* float64 variant of sk_unmix (for eigenvectors): in r x pt, out r x p. */
sk_status sk_unmix_f64(const sk_ctx *ctx, const double *in, int64_t r, double *out,
                       void *stream);

/* K-means++ seeding on the sparsified rows (Algorithm 1, "find initial
 * cluster centers via K-means++"; Arthur & Vassilvitskii, SODA 2007), restart
 * `restart` of the handle's seed.  Centre k is a row of the data: the
 * pt-vector of the chosen row's ELL entries (zero elsewhere).  The first row
 * is uniform; each next row is drawn with probability proportional to D2_i,
 * the row's restricted squared distance to its nearest chosen centre.
 * Bit-exact spec: D2_i = min over chosen c of sum_t (val_i[t] - w_c[idx_i[t]])^2
 * in float32 (t ascending, d = fma(v - c, v - c, d)); integer weights
 * q_i = floor(D2_i 2^(B - e)) with e the binary exponent of max D2
 * (max = f 2^e, 0.5 <= f < 1) and B = 62 - ceil(log2(n + 1)); the centre is
 * the first row whose inclusive prefix sum of q exceeds the draw over
 * W = sum q (W = 0: a draw over n).  The draw of step k over [0, W) takes
 * attempt a's word w[2(a%2)+1] 2^32 + w[2(a%2)] of Philox(ctr = (k, restart,
 * a/2, 0x4B4D5050 "KMPP")) and Lemire's 64-bit multiply-shift, rejecting
 * while the low 64 bits of x W are below (2^64 - W) mod W.
 * idx, val: device n x m ELL rows; mu: device K x pt float32 (the centres,
 * output); rows: device int64 K (the chosen rows, output); work: device
 * scratch of sk_kmeanspp_workspace_bytes(ctx, n) bytes, 256-byte aligned.
 * 1 <= K <= min(n, 256). */
sk_status sk_kmeanspp(const sk_ctx *ctx, const int32_t *idx, const float *val, int64_t n,
                      int32_t K, uint32_t restart, float *mu, int64_t *rows, void *work,
                      int64_t work_bytes, void *stream);
int64_t sk_kmeanspp_workspace_bytes(const sk_ctx *ctx, int64_t n);

/* The objective J' of a run (Sec. VI-A): *J = sum of the n winning
 * restricted distances `dist` (device float32, as written by the assignment
 * calls), summed in float64 into the device scalar J (overwritten).  Used to
 * keep the best of several restarts (Sec. VII: the run with the smallest
 * objective). */
sk_status sk_kmeans_objective(const float *dist, int64_t n, double *J, void *stream);

/* Diagnostic of the centre update (Sec. VI-B, Eq. (Hkmk) and the theorem on
 * H_k): dev[k] = || H_k - I ||_2 with H_k = (pt/m)(1/n_k) sum_{i in I_k}
 * R_i R_i^T, diagonal with entries (pt/m) cnt[k*pt + j] / nk[k]; -1 for an
 * empty cluster.  cnt, nk: the sums of sk_kmeans_update / step (device);
 * dev: device float64 K. */
sk_status sk_kmeans_hk(const sk_ctx *ctx, int32_t K, const int32_t *cnt, const int64_t *nk,
                       double *dev, void *stream);

/* Second pass of the 2-pass sparsified K-means (Algorithm 2), first half:
 * for each raw row x_i (X: device n x p float32, leading dimension ldx >= p),
 * labels[i] = argmin_k ||x_i - mu[k]||^2 over all p coordinates, ties to the
 * smallest k, the squared distance formed directly in float32 (no norm
 * expansion).  mu: device K x p float32, the un-mixed 1-pass centres.
 * labels: device int32 n; dist: device float32 n or NULL.  1 <= K <= 256.
 * Pass 2 reads X once; it may be called on row chunks. */
sk_status sk_kmeans2_assign(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                            const float *mu, int32_t K, int32_t *labels, float *dist,
                            void *stream);

/* Second pass of Algorithm 2, second half: the cluster means of the raw rows
 * under the *1-pass* labels (labels1: device int32 n, each in [0, K)):
 * sums[k*p + j] += sum of X[i, j] over rows with labels1[i] = k (device
 * float64 K x p) and counts[k] += rows in cluster k (device int64 K), both
 * caller-zeroed before the first chunk.  Rows with a label outside [0, K)
 * are skipped. */
sk_status sk_kmeans2_sums(const sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                          const int32_t *labels1, int32_t K, double *sums, int64_t *counts,
                          void *stream);

/* Algorithm 2's centres: mu[k*p + j] = sums/counts[k] (device float32 K x p,
 * in place) where counts[k] > 0; a cluster with no 1-pass row keeps its
 * 1-pass centre. */
sk_status sk_kmeans2_finalize(const sk_ctx *ctx, int32_t K, const double *sums,
                              const int64_t *counts, float *mu, void *stream);

/* Sample-mean estimator (Sec. IV), accumulation: sums[j] += sum over the n
 * ELL rows of the values sampled at coordinate j, i.e. sum_i R_i R_i^T y_i.
 * sums: device float64 pt, caller-zeroed before the first chunk. */
sk_status sk_mean_accumulate(const sk_ctx *ctx, const int32_t *idx, const float *val,
                             int64_t n, double *sums, void *stream);

/* Sample-mean estimator (Sec. IV): mean = (pt/m) (1/n_total) sums (device
 * float64 pt, preconditioned domain; sk_unmix_f64 maps it back to the data
 * domain).  n_total >= 1.  sums and mean may be the same buffer. */
sk_status sk_mean_finalize(const sk_ctx *ctx, const double *sums, int64_t n_total,
                           double *mean, void *stream);

/* ---- Many data sets, one launch per stage (two for a K-means pass; no
 * paper counterpart: the paper's method applied to a batch of independent
 * data sets).
 *
 * Each item describes one data set with its own p, m, seed and K and the
 * device buffers of every stage: raw rows X (n x p, leading dimension ldx,
 * global row offset row0), ELL output idx / val (n x m), Gram accumulator G
 * (pt x pt float64) with its workspace gram_work (sk_cov_workspace_bytes of a
 * handle of the same p, m for `gram_mode` and n rows), and the K-means state
 * mu (K x pt float32), labels (n int32), S (K x pt float64), cnt (K x pt
 * int32), nk (K int64) and changed (one int64 or NULL).  mu_t is optional
 * scratch (device float32 pt x 2 ceil(K/2), or NULL): a data set whose
 * centre table does not fit shared memory then reads a transposed copy of
 * its centres kept there (one contiguous segment per sampled entry) instead
 * of gathering each centre from mu.  All device buffers are caller-owned and
 * must stay valid while the batch is used.
 *
 * Supported items: 4 <= p (pt >= 256), p % 4 == 0, ldx % 4 == 0 and X
 * 16-byte aligned (rows staged with bulk copies), 1 <= K <= 64.  Within one
 * launch every data set keeps its own tensor-core Gram plan (operand stages
 * and ring slot size from its density).  Other items are rejected by sk_batch_create
 * with SK_EUNSUPPORTED or SK_EINVAL. */
typedef struct sk_batch_item {
    int64_t p, m;
    uint64_t seed;
    uint32_t flags;
    const float *X;
    int64_t n, ldx, row0;
    int32_t *idx;
    float *val;
    double *G;
    void *gram_work;
    int64_t gram_work_bytes;
    int32_t K;
    float *mu;
    float *mu_t;
    int32_t *labels;
    double *S;
    int32_t *cnt;
    int64_t *nk;
    int64_t *changed;
} sk_batch_item;

/* Opaque host-side plan of a batch: per data set launch parameters and the
 * task lists of the persistent kernels.  Holds no device memory. */
typedef struct sk_batch sk_batch;

/* Validates nd items (host array, copied) and builds the plan for the Gram
 * precision mode gram_mode (SK_GRAM_BF16 or SK_GRAM_BF16X3).  Needs the
 * current CUDA device (launch attributes are set here).  *b receives the
 * plan (host memory, freed by sk_batch_destroy). */
sk_status sk_batch_create(sk_batch **b, const sk_batch_item *items, int32_t nd,
                          int32_t gram_mode);

/* Device bytes of the plan's tables (for sk_batch_upload); -1 for NULL. */
int64_t sk_batch_workspace_bytes(const sk_batch *b);

/* Copies the plan's tables into `work` (device, at least
 * sk_batch_workspace_bytes bytes, 256-byte aligned) on the stream; the calls
 * below read them there, so `work` must stay valid and untouched while the
 * batch is used.  Call it outside stream capture; the calls below may be
 * captured. */
sk_status sk_batch_upload(sk_batch *b, void *work, int64_t work_bytes, void *stream);

/* sk_compress of every data set in one persistent launch. */
sk_status sk_batch_compress(const sk_batch *b, void *stream);

/* sk_cov_reset of every data set's G (one memset each). */
sk_status sk_batch_cov_reset(const sk_batch *b, void *stream);

/* sk_cov_accumulate of every data set in one launch of the bucketing pass
 * and one launch of the tensor-core Gram. */
sk_status sk_batch_cov_accumulate(const sk_batch *b, void *stream);

/* Zeroes every data set's S, cnt, nk in one launch. */
sk_status sk_batch_kmeans_reset(const sk_batch *b, void *stream);

/* One K-means pass over every data set: incremental = 0 as sk_kmeans_step
 * (after sk_batch_kmeans_reset), incremental = 1 as sk_kmeans_step_delta.
 * Two persistent launches: the data sets whose centre table fits shared
 * memory (or that keep none), then those reading it from global memory,
 * which run with the staging region alone so that L1 can hold their
 * tables' lines. */
sk_status sk_batch_kmeans_step(const sk_batch *b, int32_t incremental, void *stream);

/* sk_kmeans_finalize of every data set in one launch. */
sk_status sk_batch_kmeans_finalize(const sk_batch *b, void *stream);

/* Autotuner of a batch (no paper counterpart): times the candidate compress
 * task sizes (32 or 128 units per row group) and Gram tile widths (256 or
 * 128 columns) on the batch's own data, keeps the fastest, rebuilds the plan
 * and uploads it to `work` (sk_batch_workspace_bytes bytes covers every
 * candidate).  Runs the compress and Gram stages (overwriting idx, val and
 * G) and synchronises the stream: call it before capture, then reset G.
 * The chosen sizes are written to the out-pointers when not NULL. */
sk_status sk_batch_autotune(sk_batch *b, void *work, int64_t work_bytes, void *stream,
                            int32_t *units_per_group, int32_t *gram_tile_n);

/* Frees a plan (NULL is ignored). */
void sk_batch_destroy(sk_batch *b);

/* Autotuners of one handle (no paper counterpart): each times its candidate
 * launch shapes on the caller's data with CUDA events, stores the fastest in
 * the handle (used by later calls with it) and reports it.  They synchronise
 * the stream and overwrite their outputs; call them before stream capture.
 * sk_autotune_gram: tile width 256 or 128 columns times a row-split
 * multiplier 1 or 2 for sk_cov_accumulate in `mode` (tensor-core modes,
 * pt >= 256; G is overwritten -- reset it afterwards).
 * sk_autotune_compress: 1 CTA per SM or as many as fit for sk_compress. */
sk_status sk_autotune_gram(sk_ctx *ctx, int mode, const int32_t *idx, const float *val,
                           int64_t n, double *G, void *work, int64_t work_bytes, void *stream,
                           int32_t *tile_n, int32_t *split_mult);
sk_status sk_autotune_compress(sk_ctx *ctx, const float *X, int64_t n, int64_t ldx,
                               int32_t *idx, float *val, void *stream, int32_t *ctas_per_sm);

/* Reports SK_ETIMEOUT if a bounded device wait of this library ran out since
 * the last call (and clears the flag), SK_ECUDA on a pending CUDA error, else
 * SK_OK.  Synchronises the given stream first. */
sk_status sk_device_status(void *stream);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *sk_last_error(void);

/* Test hook (no counterpart in the paper): sets the limit of the bounded
 * mbarrier waits of sk_compress / sk_precondition and of the tensor-core
 * sk_cov_accumulate modes, in SM clock cycles, for kernels launched after the
 * call (process-wide; 0 restores the default of 4e9 cycles, about 2 s).  A
 * short limit makes a wait run out while its copy is still in flight: the
 * kernel then records the error word that sk_device_status reports as
 * SK_ETIMEOUT, waits with the default limit for its copies and tensor-core
 * work in flight, frees its tensor memory and returns, and its outputs are
 * unspecified.  The next calls with the default limit are unaffected.
 * Returns SK_EINVAL for cycles < 0. */
sk_status sk_debug_set_wait_cycles(int64_t cycles);

#ifdef __cplusplus
}
#endif

#endif /* SK_H */
