/*
 * sk_oracle.c -- plain, slow, FP64 CPU oracle for preconditioned data
 * sparsification (Pourkamali-Anaraki & Becker, "Preconditioned Data
 * Sparsification for Big Data with Applications to PCA and K-means").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA library: the random
 * number spec below is implemented here a second time, from its
 * published definitions, so that agreement between the two sides is
 * evidence rather than tautology.
 *
 * Every routine is a direct, single-threaded loop over the definition it
 * cites.  Floating point is double throughout.  Input samples arrive as
 * float (the data type the GPU path reads) and are widened on load.
 *
 * Written random-number spec (shared in prose with the CUDA side):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random
 *   numbers: as easy as 1, 2, 3"), key = (seed_lo, seed_hi).
 *   Signs D (Sec. III, Eq. (ROS)): coordinate j uses bit (j mod 32) of
 *     output word (j/32) mod 4 of Philox(ctr = (j/128, 0, 0, TAG_SIGN));
 *     bit 0 -> D_j = +1, bit 1 -> D_j = -1.  One D for the whole data set.
 *   Mask of global row r (Sec. I-A, Thm. B1): words w = 0,1,2,... are
 *     output word (w mod 4) of Philox(ctr = (w/4, r_lo, r_hi, TAG_MASK)).
 *     Bounded integers in [0,s) by Lemire's multiply-shift with rejection
 *     (D. Lemire, "Fast random integer generation in an interval", ACM
 *     TOMACS 2019).  Partial Fisher-Yates over the virtual identity array
 *     a[0..pt): for t = 0..m-1, k = t + U(pt - t), swap a[t], a[k],
 *     emit a[t].  Indices are kept in draw order.
 *   Initial K-means rows (test harness): partial Fisher-Yates over [0,n)
 *     with words of Philox(ctr = (w/4, 0, 0, TAG_INIT)).
 *   K-means++ seeding on the sparsified rows, restart r (Algorithm 1, "find
 *     initial cluster centers via K-means++"; D. Arthur, S. Vassilvitskii,
 *     "k-means++: the advantages of careful seeding", SODA 2007):
 *     the draw of step k over [0, W) takes attempt a's 64-bit word
 *     x = w[2(a%2)+1] 2^32 + w[2(a%2)] of Philox(ctr = (k, r, a/2,
 *     TAG_KMPP)) and Lemire's multiply-shift on 64 bits (reject while the
 *     low 64 bits of x W are below (2^64 - W) mod W; value = high 64 bits).
 *     Step 0: the first centre is the draw over W = n.  Step k >= 1: D2_i is
 *     the smallest restricted squared distance of row i to a chosen centre,
 *     sum over t of (val_i[t] - w_c[idx_i[t]])^2 with w_c the pt-vector of
 *     row c's ELL entries (zero elsewhere), formed in float32 (t ascending,
 *     d = fmaf(v - c, v - c, d)); the weights are the integers
 *     q_i = floor(D2_i 2^(B - e)), e the binary exponent of max_i D2_i
 *     (max = f 2^e, 0.5 <= f < 1) and B = 62 - ceil(log2(n + 1)); the centre
 *     is the first i whose inclusive prefix sum of q exceeds the draw over
 *     W = sum q (if W = 0, the draw over n).  The integer weights make the
 *     choice independent of summation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TAG_SIGN 0x5349474Eu /* "SIGN" */
#define TAG_MASK 0x4D41534Bu /* "MASK" */
#define TAG_INIT 0x494E4954u /* "INIT" */
#define TAG_KMPP 0x4B4D5050u /* "KMPP" */

/* ---------------- Philox4x32-10 (Salmon et al., SC'11) ---------------- */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key bumps */
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k[2] = {key_in[0], key_in[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k[0] += W0;
            k[1] += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k[0];
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k[1];
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Word w of the stream (c1, c2, tag) under key seed. */
static uint32_t stream_word(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t tag,
                            uint64_t w) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(w / 4), c1, c2, tag};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[w % 4];
}

/* Smallest power of two >= p (the padded dimension p~). */
int64_t oracle_ptilde(int64_t p) {
    int64_t q = 1;
    while (q < p) q *= 2;
    return q;
}

/* ---------------- Lemire bounded integer ---------------- */

/* U(s) from an explicit word list (exposed so tests can drive rejection).
 * Returns the value; *consumed receives how many words were used, or -1
 * if the list ran out. */
uint32_t oracle_lemire_from_words(uint32_t s, const uint32_t *words, int64_t nwords,
                                  int64_t *consumed) {
    int64_t used = 0;
    uint32_t threshold = (uint32_t)(((uint64_t)1 << 32) % s); /* 2^32 mod s */
    for (;;) {
        if (used >= nwords) { *consumed = -1; return 0; }
        uint64_t L = (uint64_t)words[used++] * (uint64_t)s;
        uint32_t low = (uint32_t)L;
        if (low < threshold) continue; /* reject: keeps U(s) exactly uniform */
        *consumed = used;
        return (uint32_t)(L >> 32);
    }
}

/* ---------------- Signs D (Sec. III, Eq. (ROS)) ---------------- */

void oracle_signs(int64_t pt, uint64_t seed, double *D) {
    for (int64_t j = 0; j < pt; ++j) {
        uint32_t word = stream_word(seed, 0u, 0u, TAG_SIGN, (uint64_t)(j / 32));
        /* stream_word(w) takes word w of block w/4: coordinate j lives in
         * block j/128, word (j/32) mod 4 -> stream word index j/32. */
        uint32_t bit = (word >> (j % 32)) & 1u;
        D[j] = bit ? -1.0 : 1.0;
    }
}

/* ---------------- Mask Omega_r (Sec. I-A; Thm. B1) ---------------- */

/* Partial Fisher-Yates over a[0..pt) on the virtual identity array, stored
 * here as an explicit array (this is the slow, obvious form). */
static void fisher_yates_stream(int64_t N, int64_t m, uint64_t seed, uint32_t c1,
                                uint32_t c2, uint32_t tag, int64_t *out) {
    int64_t *a = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    for (int64_t j = 0; j < N; ++j) a[j] = j;
    uint64_t w = 0;
    for (int64_t t = 0; t < m; ++t) {
        uint32_t s = (uint32_t)(N - t);
        uint32_t threshold = (uint32_t)(((uint64_t)1 << 32) % s);
        uint64_t L;
        for (;;) {
            uint32_t v = stream_word(seed, c1, c2, tag, w++);
            L = (uint64_t)v * (uint64_t)s;
            if ((uint32_t)L >= threshold) break;
        }
        int64_t k = t + (int64_t)(L >> 32);
        int64_t tmp = a[t];
        a[t] = a[k];
        a[k] = tmp;
        out[t] = a[t];
    }
    free(a);
}

void oracle_mask(int64_t pt, int64_t m, uint64_t seed, int64_t row, int32_t *omega) {
    int64_t *tmp = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    fisher_yates_stream(pt, m, seed, (uint32_t)row, (uint32_t)((uint64_t)row >> 32),
                        TAG_MASK, tmp);
    for (int64_t t = 0; t < m; ++t) omega[t] = (int32_t)tmp[t];
    free(tmp);
}

void oracle_init_rows(int64_t n, int64_t K, uint64_t seed, int64_t *rows) {
    fisher_yates_stream(n, K, seed, 0u, 0u, TAG_INIT, rows);
}

/* ---------------- Walsh-Hadamard transform (Sec. III) ---------------- */

/* In-place y <- H y with H the Sylvester-ordered Hadamard matrix scaled to
 * be orthonormal, H[u][l] = (-1)^popcount(u & l) / sqrt(pt).  Textbook
 * radix-2 butterflies followed by one scaling. */
void oracle_fwht(double *y, int64_t pt) {
    for (int64_t h = 1; h < pt; h *= 2) {
        for (int64_t i = 0; i < pt; i += 2 * h) {
            for (int64_t j = i; j < i + h; ++j) {
                double a = y[j], b = y[j + h];
                y[j] = a + b;
                y[j + h] = a - b;
            }
        }
    }
    double scale = 1.0 / sqrt((double)pt);
    for (int64_t j = 0; j < pt; ++j) y[j] *= scale;
}

/* y_i = H D [x_i; 0] for each row (Sec. III, Eq. (ROS); Algorithm 1, line
 * "Y <- HDX"), zero-padding p -> pt.  Y is n x pt, row-major. */
void oracle_precondition(const float *X, int64_t n, int64_t p, int64_t ldx,
                         uint64_t seed, double *Y) {
    int64_t pt = oracle_ptilde(p);
    double *D = (double *)malloc((size_t)pt * sizeof(double));
    oracle_signs(pt, seed, D);
    for (int64_t i = 0; i < n; ++i) {
        double *y = Y + i * pt;
        for (int64_t j = 0; j < pt; ++j) {
            double xj = (j < p) ? (double)X[i * ldx + j] : 0.0;
            y[j] = D[j] * xj;
        }
        oracle_fwht(y, pt);
    }
    free(D);
}

/* Ablation without preconditioning (H = D = I, the "no preconditioning"
 * variant of Sec. VII): the mask of row r over [0, pt) of the zero-padded x,
 * val = x[idx].  Same mask stream as oracle_compress. */
void oracle_compress_raw(const float *X, int64_t n, int64_t p, int64_t ldx, int64_t row0,
                         int64_t m, uint64_t seed, int32_t *idx, double *val) {
    int64_t pt = oracle_ptilde(p);
    for (int64_t i = 0; i < n; ++i) {
        oracle_mask(pt, m, seed, row0 + i, idx + i * m);
        for (int64_t t = 0; t < m; ++t) {
            int64_t j = idx[i * m + t];
            val[i * m + t] = (j < p) ? (double)X[i * ldx + j] : 0.0;
        }
    }
}

/* Compression of rows row0..row0+n-1: w_i = R_i R_i^T y_i stored as ELL
 * (idx[i][t] = Omega_r[t], val[i][t] = y_i[Omega_r[t]]), Algorithm 1. */
void oracle_compress(const float *X, int64_t n, int64_t p, int64_t ldx, int64_t row0,
                     int64_t m, uint64_t seed, int32_t *idx, double *val) {
    int64_t pt = oracle_ptilde(p);
    double *y = (double *)malloc((size_t)pt * sizeof(double));
    double *D = (double *)malloc((size_t)pt * sizeof(double));
    oracle_signs(pt, seed, D);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < pt; ++j)
            y[j] = (j < p) ? D[j] * (double)X[i * ldx + j] : 0.0;
        oracle_fwht(y, pt);
        oracle_mask(pt, m, seed, row0 + i, idx + i * m);
        for (int64_t t = 0; t < m; ++t) val[i * m + t] = y[idx[i * m + t]];
    }
    free(D);
    free(y);
}

/* ---------------- Covariance estimator (Sec. V) ---------------- */

/* G += sum_i w_i w_i^T, the unscaled sparse Gram of the ELL rows. */
void oracle_gram(const int32_t *idx, const double *val, int64_t n, int64_t m, int64_t pt,
                 double *G) {
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *ix = idx + i * m;
        const double *vx = val + i * m;
        for (int64_t s = 0; s < m; ++s)
            for (int64_t t = 0; t < m; ++t)
                G[(int64_t)ix[s] * pt + ix[t]] += vx[s] * vx[t];
    }
}

/* C_emp-hat = pt(pt-1)/(m(m-1)) * G / n; C_n = C_emp-hat - (pt-m)/(pt-1) diag(C_emp-hat)
 * (Sec. V, definitions of C_emp-hat and C_n).  Requires m >= 2. */
void oracle_cov_finalize(const double *G, int64_t n, int64_t m, int64_t pt, double *C) {
    double P = (double)pt, M = (double)m;
    double scale = P * (P - 1.0) / (M * (M - 1.0)) / (double)n;
    for (int64_t a = 0; a < pt * pt; ++a) C[a] = scale * G[a];
    double corr = (P - M) / (P - 1.0);
    for (int64_t j = 0; j < pt; ++j) C[j * pt + j] -= corr * C[j * pt + j];
}

/* Centred covariance estimate, built from the paper's two estimators: with
 * C_n the covariance estimate above (Sec. V) and xbar the sample-mean estimate
 * (Sec. IV) of the same n rows,
 *   C_c = C_n - xbar xbar^T + (1/n) B(C_n),
 *   B(A)_jj = ((P - m)/m) A_jj,  B(A)_jk = -((P - m)/(m (P - 1))) A_jk (j != k).
 * B(C_emp)/n is the covariance of xbar over the masks: by Thm. B1 a mask keeps
 * j with probability m/P and the pair (j, k) with m(m-1)/(P(P-1)), so
 * Cov((P/m) R R^T y) has diagonal (P/m - 1) y_j^2 and off-diagonal
 * (P(m-1)/(m(P-1)) - 1) y_j y_k; summed over independent rows and divided by
 * n^2 that is B(C_emp)/n.  Hence E[xbar xbar^T] = ybar ybar^T + B(C_emp)/n,
 * and since E[C_n] = C_emp and B is linear, E[C_c] = C_emp - ybar ybar^T, the
 * centred second moment.  mean: xbar (length pt); C: pt x pt output. */
void oracle_cov_centred(const double *G, const double *mean, int64_t n, int64_t m, int64_t pt,
                        double *C) {
    oracle_cov_finalize(G, n, m, pt, C);
    double P = (double)pt, M = (double)m, N = (double)n;
    double dcoef = (P - M) / M / N;
    double ocoef = -(P - M) / (M * (P - 1.0)) / N;
    for (int64_t j = 0; j < pt; ++j)
        for (int64_t k = 0; k < pt; ++k) {
            double cn = C[j * pt + k];
            double b = (j == k ? dcoef : ocoef) * cn;
            C[j * pt + k] = cn + b - mean[j] * mean[k];
        }
}

/* Sample-mean estimator (Sec. IV, Thm. "sampleMean"): (pt/m)(1/n) sum_i w_i. */
void oracle_sample_mean(const int32_t *idx, const double *val, int64_t n, int64_t m,
                        int64_t pt, double *mean) {
    for (int64_t j = 0; j < pt; ++j) mean[j] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t t = 0; t < m; ++t) mean[idx[i * m + t]] += val[i * m + t];
    double scale = (double)pt / (double)m / (double)n;
    for (int64_t j = 0; j < pt; ++j) mean[j] *= scale;
}

/* ---------------- Sparsified K-means (Sec. VI-B) ---------------- */

/* Eq. (assignments): c_i = argmin_k || z_i - R_i^T mu'_k ||^2, computed
 * directly over the m sampled coordinates.  Ties go to the smallest k. */
void oracle_kmeans_assign(const int32_t *idx, const double *val, int64_t n, int64_t m,
                          const double *mu, int64_t K, int64_t pt, int32_t *labels,
                          double *dist) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = 0;
        double bestd = INFINITY;
        for (int64_t k = 0; k < K; ++k) {
            double d = 0.0;
            for (int64_t t = 0; t < m; ++t) {
                double diff = val[i * m + t] - mu[k * pt + idx[i * m + t]];
                d += diff * diff;
            }
            if (d < bestd) { bestd = d; best = k; }
        }
        labels[i] = (int32_t)best;
        if (dist) dist[i] = bestd;
    }
}

/* Eq. (mu_update_one)/(mu_update_two): mu'_kj = S_kj / n_k^(j) with
 * S_kj = sum over rows of cluster k that sampled j.  A coordinate that no
 * row of the cluster sampled (n_k^(j) = 0) cannot be estimated; it keeps
 * its previous value.  counts is K x pt, nk is K. */
void oracle_kmeans_update(const int32_t *idx, const double *val, const int32_t *labels,
                          int64_t n, int64_t m, int64_t K, int64_t pt,
                          const double *mu_prev, double *mu_new, int64_t *counts,
                          int64_t *nk) {
    double *S = (double *)calloc((size_t)(K * pt), sizeof(double));
    for (int64_t a = 0; a < K * pt; ++a) counts[a] = 0;
    for (int64_t k = 0; k < K; ++k) nk[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = labels[i];
        nk[k] += 1;
        for (int64_t t = 0; t < m; ++t) {
            int64_t j = idx[i * m + t];
            S[k * pt + j] += val[i * m + t];
            counts[k * pt + j] += 1;
        }
    }
    for (int64_t a = 0; a < K * pt; ++a)
        mu_new[a] = counts[a] > 0 ? S[a] / (double)counts[a] : mu_prev[a];
    free(S);
}

/* Eq. (mu-mu'): mu = (HD)^T mu' = D H mu' (Sylvester H is symmetric),
 * truncated to the first p coordinates.  in is r x pt, out is r x p. */
/* ---------------- DCT preconditioner (Sec. III: H a DCT matrix) ----------------
 *
 * H is the orthonormal DCT-II of length p (no padding: the sampling and the
 * estimators then use p itself):
 *   (H x)_k = s_k sum_{l=0}^{p-1} x_l cos(pi (2l + 1) k / (2p)),
 *   s_0 = sqrt(1/p), s_k = sqrt(2/p) for k >= 1,
 * written out as the direct O(p^2) sum.  Its transpose (the orthonormal
 * DCT-III) is the un-mixing map.  The cosine's argument is reduced exactly in
 * integers, (2l + 1) k mod 4p, before the one floating-point division. */
static double dct_cos(int64_t a, int64_t p) {
    const double pi = 3.14159265358979323846;
    return cos(pi * (double)(a % (4 * p)) / (2.0 * (double)p));
}

void oracle_dct2(double *y, int64_t p) {
    double *t = (double *)malloc((size_t)p * sizeof(double));
    for (int64_t k = 0; k < p; ++k) {
        double acc = 0.0;
        for (int64_t l = 0; l < p; ++l) acc += y[l] * dct_cos((2 * l + 1) * k, p);
        t[k] = (k == 0 ? sqrt(1.0 / (double)p) : sqrt(2.0 / (double)p)) * acc;
    }
    memcpy(y, t, (size_t)p * sizeof(double));
    free(t);
}

void oracle_dct3(double *y, int64_t p) {
    double *t = (double *)malloc((size_t)p * sizeof(double));
    for (int64_t l = 0; l < p; ++l) {
        double acc = 0.0;
        for (int64_t k = 0; k < p; ++k)
            acc += (k == 0 ? sqrt(1.0 / (double)p) : sqrt(2.0 / (double)p)) * y[k] *
                   dct_cos((2 * l + 1) * k, p);
        t[l] = acc;
    }
    memcpy(y, t, (size_t)p * sizeof(double));
    free(t);
}

/* y = H D x with the DCT H (Eq. (ROS)), row by row: Y is n x p. */
void oracle_precondition_dct(const float *X, int64_t n, int64_t p, int64_t ldx, uint64_t seed,
                             double *Y) {
    double *D = (double *)malloc((size_t)p * sizeof(double));
    oracle_signs(p, seed, D);
    for (int64_t i = 0; i < n; ++i) {
        double *y = Y + i * p;
        for (int64_t j = 0; j < p; ++j) y[j] = D[j] * (double)X[i * ldx + j];
        oracle_dct2(y, p);
    }
    free(D);
}

/* ELL form with the DCT preconditioner: the mask of global row r is the
 * written spec's partial Fisher-Yates over [0, p). */
void oracle_compress_dct(const float *X, int64_t n, int64_t p, int64_t ldx, int64_t row0,
                         int64_t m, uint64_t seed, int32_t *idx, double *val) {
    double *y = (double *)malloc((size_t)p * sizeof(double));
    double *D = (double *)malloc((size_t)p * sizeof(double));
    oracle_signs(p, seed, D);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < p; ++j) y[j] = D[j] * (double)X[i * ldx + j];
        oracle_dct2(y, p);
        oracle_mask(p, m, seed, row0 + i, idx + i * m);
        for (int64_t t = 0; t < m; ++t) val[i * m + t] = y[idx[i * m + t]];
    }
    free(D);
    free(y);
}

/* Un-mixing with the DCT: out_i = D H^T in_i (in, out: r x p). */
void oracle_unmix_dct(const double *in, int64_t r, int64_t p, uint64_t seed, double *out) {
    double *D = (double *)malloc((size_t)p * sizeof(double));
    oracle_signs(p, seed, D);
    for (int64_t i = 0; i < r; ++i) {
        double *o = out + i * p;
        memcpy(o, in + i * p, (size_t)p * sizeof(double));
        oracle_dct3(o, p);
        for (int64_t j = 0; j < p; ++j) o[j] *= D[j];
    }
    free(D);
}

void oracle_unmix(const double *in, int64_t r, int64_t pt, int64_t p, uint64_t seed,
                  double *out) {
    double *D = (double *)malloc((size_t)pt * sizeof(double));
    double *y = (double *)malloc((size_t)pt * sizeof(double));
    oracle_signs(pt, seed, D);
    for (int64_t i = 0; i < r; ++i) {
        memcpy(y, in + i * pt, (size_t)pt * sizeof(double));
        oracle_fwht(y, pt);
        for (int64_t j = 0; j < p; ++j) out[i * p + j] = D[j] * y[j];
    }
    free(D);
    free(y);
}

/* Second pass of the 2-pass sparsified K-means (Algorithm 2): with the 1-pass
 * labels c1 and the 1-pass centres mu1 (data domain, K x p), every raw row is
 * assigned to its nearest mu1 (dense squared distance, ties to the smallest
 * k) and added to the mean of its 1-pass cluster.  mu2 = sum / |I_k|; a
 * cluster with no 1-pass row keeps mu1 (the algorithm does not define it). */
void oracle_kmeans_2pass(const float *X, int64_t n, int64_t p, const int32_t *c1,
                         const double *mu1, int64_t K, int32_t *c2, double *mu2,
                         int64_t *counts) {
    double *sum = (double *)calloc((size_t)(K * p), sizeof(double));
    for (int64_t k = 0; k < K; ++k) counts[k] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const float *x = X + i * p;
        int64_t k1 = c1[i];
        counts[k1] += 1;
        for (int64_t j = 0; j < p; ++j) sum[k1 * p + j] += (double)x[j];
        int64_t best = 0;
        double bestd = INFINITY;
        for (int64_t k = 0; k < K; ++k) {
            double d = 0.0;
            for (int64_t j = 0; j < p; ++j) {
                double diff = (double)x[j] - mu1[k * p + j];
                d += diff * diff;
            }
            if (d < bestd) { bestd = d; best = k; }
        }
        c2[i] = (int32_t)best;
    }
    for (int64_t k = 0; k < K; ++k)
        for (int64_t j = 0; j < p; ++j)
            mu2[k * p + j] = counts[k] > 0 ? sum[k * p + j] / (double)counts[k] : mu1[k * p + j];
    free(sum);
}

/* ---------------- K-means++ seeding on sparse rows ---------------- */

/* Draw of step k, restart r, uniform over [0, W) (W >= 1): 64-bit Lemire
 * multiply-shift with rejection on the KMPP stream (header spec). */
uint64_t oracle_kpp_draw(uint64_t seed, uint32_t k, uint32_t r, uint64_t W) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint64_t threshold = (0 - W) % W; /* (2^64 - W) mod W */
    for (uint32_t a = 0;; ++a) {
        const uint32_t ctr[4] = {k, r, a / 2, TAG_KMPP};
        uint32_t out[4];
        oracle_philox4x32_10(ctr, key, out);
        const uint64_t x = ((uint64_t)out[2 * (a % 2) + 1] << 32) | out[2 * (a % 2)];
        const __uint128_t prod = (__uint128_t)x * W;
        if ((uint64_t)prod < threshold) continue;
        return (uint64_t)(prod >> 64);
    }
}

/* Restricted squared distance of ELL row i to the dense pt-vector cen, in
 * float32 with t ascending (the precision the seeding decides in). */
static float kpp_dist(const int32_t *idx, const float *val, int64_t i, int64_t m,
                      const float *cen) {
    float d = 0.0f;
    for (int64_t t = 0; t < m; ++t) {
        const float diff = val[i * m + t] - cen[idx[i * m + t]];
        d = fmaf(diff, diff, d);
    }
    return d;
}

/* K-means++ seeding of restart r (header spec).  idx, val: the n x m ELL
 * rows (val in float32).  rows_out: K chosen row indices; centres_out:
 * K x pt, row k the dense pt-vector of the chosen row's entries. */
void oracle_kmeanspp(const int32_t *idx, const float *val, int64_t n, int64_t m, int64_t pt,
                     int64_t K, uint64_t seed, uint32_t r, int64_t *rows_out,
                     float *centres_out) {
    float *D2 = (float *)malloc((size_t)n * sizeof(float));
    int B = 62;
    while (((uint64_t)1 << (62 - B)) < (uint64_t)(n + 1)) --B; /* B = 62 - ceil(log2(n+1)) */
    for (int64_t k = 0; k < K; ++k) {
        int64_t c;
        if (k == 0) {
            c = (int64_t)oracle_kpp_draw(seed, 0u, r, (uint64_t)n);
        } else {
            float mx = 0.0f;
            for (int64_t i = 0; i < n; ++i)
                if (D2[i] > mx) mx = D2[i];
            uint64_t W = 0;
            int e = 0;
            if (mx > 0.0f) {
                frexp((double)mx, &e);
                for (int64_t i = 0; i < n; ++i) W += (uint64_t)ldexp((double)D2[i], B - e);
            }
            if (W == 0) {
                c = (int64_t)oracle_kpp_draw(seed, (uint32_t)k, r, (uint64_t)n);
            } else {
                const uint64_t u = oracle_kpp_draw(seed, (uint32_t)k, r, W);
                uint64_t acc = 0;
                c = n - 1;
                for (int64_t i = 0; i < n; ++i) {
                    acc += (uint64_t)ldexp((double)D2[i], B - e);
                    if (acc > u) { c = i; break; }
                }
            }
        }
        rows_out[k] = c;
        float *cen = centres_out + k * pt;
        for (int64_t j = 0; j < pt; ++j) cen[j] = 0.0f;
        for (int64_t t = 0; t < m; ++t) cen[idx[c * m + t]] = val[c * m + t];
        for (int64_t i = 0; i < n; ++i) {
            const float d = kpp_dist(idx, val, i, m, cen);
            if (k == 0 || d < D2[i]) D2[i] = d;
        }
    }
    free(D2);
}

/* ---------------- H_k of the centre update (Eq. (Hkmk)) ---------------- */

/* dev[k] = || H_k - I ||_2 with H_k = (pt/m)(1/n_k) sum_{i in I_k} R_i R_i^T,
 * a diagonal matrix whose entry j is (pt/m) counts[k][j] / nk[k]; -1 for an
 * empty cluster (H_k undefined). */
void oracle_kmeans_hk(const int64_t *counts, const int64_t *nk, int64_t K, int64_t pt,
                      int64_t m, double *dev) {
    for (int64_t k = 0; k < K; ++k) {
        if (nk[k] == 0) { dev[k] = -1.0; continue; }
        double worst = 0.0;
        for (int64_t j = 0; j < pt; ++j) {
            const double h = (double)pt / (double)m * (double)counts[k * pt + j] / (double)nk[k];
            const double d = fabs(h - 1.0);
            if (d > worst) worst = d;
        }
        dev[k] = worst;
    }
}
