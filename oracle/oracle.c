/*
 * oracle.c -- plain, slow, single-threaded FP64 reference for the sparse
 * MTTKRP / CP-ALS path (plus one all-core form of the MTTKRP definition,
 * for the timed CPU baseline).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Every routine is the textbook definition of what it computes, evaluated
 * directly in double precision, in storage order, with no blocking, fusion
 * or reordering.  Inputs narrower than double (fp32 values, fp32/bf16/f16
 * factors) are widened exactly by the caller before they arrive here.
 *
 * Layout conventions (shared with the tests, not with the CUDA code):
 *   idx   : d*P int32, mode-major; idx[m*P + i] is the 0-based mode-m
 *           coordinate of nonzero i (the paper's l_{i,m+1}, Sec. 3).
 *   vals  : P doubles (x_i).
 *   A[m]  : I_m x lda[m] row-major factor matrix A^(m) (Sec. 3, eq. CP).
 *   V     : I_n x ldv row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <fenv.h>
#include <pthread.h>

/* ---------------------------------------------------------------------- */
/* MTTKRP, Sec. 3 eq. (mttkrp):                                            */
/*   v(k,j) = lambda_j * sum_{i : l_in = k} x_i * prod_{m != n} a^(m)(l_im, j) */
/* lambda == NULL means lambda_j = 1.  Columns j >= R of V are set to 0.    */
/* ---------------------------------------------------------------------- */
void oracle_mttkrp(int d, const int64_t *dims, int64_t P, const int32_t *idx,
                   const double *vals, int n, int R, const double *const *A,
                   const int64_t *lda, const double *lambda, double *V, int64_t ldv)
{
    int64_t In = dims[n];
    memset(V, 0, sizeof(double) * (size_t)In * (size_t)ldv);
    for (int64_t i = 0; i < P; ++i) {
        int64_t k = idx[(int64_t)n * P + i];
        for (int j = 0; j < R; ++j) {
            double t = vals[i];
            for (int m = 0; m < d; ++m) {
                if (m == n) continue;
                int64_t row = idx[(int64_t)m * P + i];
                t *= A[m][row * lda[m] + j];
            }
            V[k * ldv + j] += t;
        }
    }
    if (lambda)
        for (int64_t k = 0; k < In; ++k)
            for (int j = 0; j < R; ++j) V[k * ldv + j] *= lambda[j];
}

/* The same definition on T host threads (the CPU baseline's all-core form).
 * Thread t owns the output rows [lo_t, hi_t), the ranges cut so that each
 * holds about P / T nonzeros; it walks all nonzeros in storage order and
 * applies those whose row it owns, exactly as oracle_mttkrp does.  Every
 * row therefore receives the same additions in the same order as in
 * oracle_mttkrp, and V is bit-identical to it for every T.
 * Returns 0, or 1 if a thread or an array could not be created. */
struct mt_job {
    int d, n, R;
    int64_t P, lo, hi, ldv;
    const int32_t *idx;
    const double *vals;
    const double *const *A;
    const int64_t *lda;
    const double *lambda;
    double *V;
};

static void *mt_worker(void *arg)
{
    const struct mt_job *w = (const struct mt_job *)arg;
    for (int64_t i = 0; i < w->P; ++i) {
        int64_t k = w->idx[(int64_t)w->n * w->P + i];
        if (k < w->lo || k >= w->hi) continue;
        for (int j = 0; j < w->R; ++j) {
            double t = w->vals[i];
            for (int m = 0; m < w->d; ++m) {
                if (m == w->n) continue;
                int64_t row = w->idx[(int64_t)m * w->P + i];
                t *= w->A[m][row * w->lda[m] + j];
            }
            w->V[k * w->ldv + j] += t;
        }
    }
    if (w->lambda)
        for (int64_t k = w->lo; k < w->hi; ++k)
            for (int j = 0; j < w->R; ++j) w->V[k * w->ldv + j] *= w->lambda[j];
    return NULL;
}

int oracle_mttkrp_threads(int d, const int64_t *dims, int64_t P, const int32_t *idx,
                          const double *vals, int n, int R, const double *const *A,
                          const int64_t *lda, const double *lambda, double *V, int64_t ldv,
                          int T)
{
    int64_t In = dims[n];
    if (T < 1) T = 1;
    memset(V, 0, sizeof(double) * (size_t)In * (size_t)ldv);
    int64_t *cnt = (int64_t *)calloc((size_t)In + 1, sizeof(int64_t));
    struct mt_job *jobs = (struct mt_job *)calloc((size_t)T, sizeof(struct mt_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)T, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)T, sizeof(int));
    int status = (cnt && jobs && tid && started) ? 0 : 1;
    if (!status) {
        for (int64_t i = 0; i < P; ++i) cnt[idx[(int64_t)n * P + i]] += 1;
        /* row ranges: thread t starts at the first row whose nonzeros before
         * it number at least t P / T */
        int64_t k = 0, before = 0;
        for (int t = 0; t < T; ++t) {
            int64_t target = P * t / T;
            while (k < In && before < target) before += cnt[k++];
            jobs[t].lo = (t == 0) ? 0 : k;
        }
        for (int t = 0; t < T; ++t) {
            struct mt_job *w = &jobs[t];
            w->hi = (t + 1 < T) ? jobs[t + 1].lo : In;
            w->d = d; w->n = n; w->R = R; w->P = P; w->ldv = ldv;
            w->idx = idx; w->vals = vals; w->A = A; w->lda = lda; w->lambda = lambda; w->V = V;
        }
        for (int t = 0; t < T; ++t) {
            if (jobs[t].lo >= jobs[t].hi) continue;
            if (pthread_create(&tid[t], NULL, mt_worker, &jobs[t]) != 0) { status = 1; break; }
            started[t] = 1;
        }
        for (int t = 0; t < T; ++t)
            if (started[t]) pthread_join(tid[t], NULL);
    }
    free(cnt);
    free(jobs);
    free(tid);
    free(started);
    return status;
}

/* The same definition restricted to a list of output rows: Vrows[r*ldv + j]
 * = v(rows[r], j).  Used to check single rows of very large problems. */
void oracle_mttkrp_rows(int d, const int64_t *dims, int64_t P, const int32_t *idx,
                        const double *vals, int n, int R, const double *const *A,
                        const int64_t *lda, const double *lambda, int64_t nrows,
                        const int32_t *rows, double *Vrows, int64_t ldv)
{
    int64_t In = dims[n];
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)In);
    for (int64_t k = 0; k < In; ++k) slot[k] = -1;
    for (int64_t r = 0; r < nrows; ++r) slot[rows[r]] = r;
    memset(Vrows, 0, sizeof(double) * (size_t)nrows * (size_t)ldv);
    for (int64_t i = 0; i < P; ++i) {
        int64_t k = idx[(int64_t)n * P + i];
        int64_t r = slot[k];
        if (r < 0) continue;
        for (int j = 0; j < R; ++j) {
            double t = vals[i];
            for (int m = 0; m < d; ++m) {
                if (m == n) continue;
                t *= A[m][(int64_t)idx[(int64_t)m * P + i] * lda[m] + j];
            }
            Vrows[r * ldv + j] += t;
        }
    }
    /* a row listed twice gets the sum only once: copy from its last slot */
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t s = slot[rows[r]];
        if (s != r) memcpy(Vrows + r * ldv, Vrows + s * ldv, sizeof(double) * (size_t)R);
    }
    if (lambda)
        for (int64_t r = 0; r < nrows; ++r)
            for (int j = 0; j < R; ++j) Vrows[r * ldv + j] *= lambda[j];
    free(slot);
}

/* ---------------------------------------------------------------------- */
/* Mode permutation, Sec. 6: perm lists the nonzeros in increasing mode-n   */
/* index; the sort is stable, so equal indices keep their storage order.    */
/* Definition used here: sort positions by the pair (key, position).        */
/* ---------------------------------------------------------------------- */
static const int32_t *g_keys;
static int cmp_key_pos(const void *a, const void *b)
{
    int32_t ia = *(const int32_t *)a, ib = *(const int32_t *)b;
    if (g_keys[ia] != g_keys[ib]) return g_keys[ia] < g_keys[ib] ? -1 : 1;
    return (ia > ib) - (ia < ib);
}

void oracle_stable_argsort(int64_t P, const int32_t *keys, int32_t *perm)
{
    for (int64_t i = 0; i < P; ++i) perm[i] = (int32_t)i;
    g_keys = keys;
    qsort(perm, (size_t)P, sizeof(int32_t), cmp_key_pos);
}

/* ---------------------------------------------------------------------- */
/* Coalescing duplicate coordinates (COO, Sec. 3): the tensor entry at a    */
/* coordinate is the sum of all nonzeros stored with that coordinate.       */
/* Output: distinct coordinates in lexicographic order (mode 0 slowest),    */
/* each value the FP64 sum of its duplicates in storage order.              */
/* ---------------------------------------------------------------------- */
static const int32_t *g_idx;
static int64_t g_P;
static int g_d;
static int cmp_coord_pos(const void *a, const void *b)
{
    int32_t ia = *(const int32_t *)a, ib = *(const int32_t *)b;
    for (int m = 0; m < g_d; ++m) {
        int32_t x = g_idx[(int64_t)m * g_P + ia], y = g_idx[(int64_t)m * g_P + ib];
        if (x != y) return x < y ? -1 : 1;
    }
    return (ia > ib) - (ia < ib);
}

int64_t oracle_coalesce(int d, int64_t P, const int32_t *idx, const double *vals,
                        int32_t *out_idx /* d*P capacity, mode-major with stride P */,
                        double *out_vals)
{
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    for (int64_t i = 0; i < P; ++i) ord[i] = (int32_t)i;
    g_idx = idx; g_P = P; g_d = d;
    qsort(ord, (size_t)P, sizeof(int32_t), cmp_coord_pos);
    int64_t u = -1;
    for (int64_t q = 0; q < P; ++q) {
        int64_t i = ord[q];
        int same = (u >= 0);
        if (same)
            for (int m = 0; m < d; ++m)
                if (idx[(int64_t)m * P + i] != out_idx[(int64_t)m * P + u]) { same = 0; break; }
        if (!same) {
            ++u;
            for (int m = 0; m < d; ++m) out_idx[(int64_t)m * P + u] = idx[(int64_t)m * P + i];
            out_vals[u] = 0.0;
        }
        out_vals[u] += vals[i];
    }
    free(ord);
    return u + 1;
}

/* ||X||^2 = sum over distinct coordinates of (sum of duplicates)^2. */
double oracle_norm2(int d, int64_t P, const int32_t *idx, const double *vals)
{
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(d * (P > 0 ? P : 1)));
    double *cv = (double *)malloc(sizeof(double) * (size_t)(P > 0 ? P : 1));
    int64_t u = oracle_coalesce(d, P, idx, vals, ci, cv);
    double s = 0.0;
    for (int64_t q = 0; q < u; ++q) s += cv[q] * cv[q];
    free(ci); free(cv);
    return s;
}

/* ---------------------------------------------------------------------- */
/* Dense pieces of one CP-ALS update (Sec. 3 refers to ALS; the steps are   */
/* the standard normal-equation update).                                    */
/* ---------------------------------------------------------------------- */

/* Gram matrix G = A^T A (R x R), A is I x lda row-major. */
void oracle_gram(int64_t I, int R, const double *A, int64_t lda, double *G)
{
    for (int r = 0; r < R; ++r)
        for (int s = 0; s < R; ++s) {
            double acc = 0.0;
            for (int64_t i = 0; i < I; ++i) acc += A[i * lda + r] * A[i * lda + s];
            G[r * R + s] = acc;
        }
}

/* Cholesky H = L L^T (lower triangular L, row-major R x R, upper part 0).
 * Returns 0 on success, 1 if a pivot is not positive. */
int oracle_cholesky(int R, const double *H, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)R * (size_t)R);
    for (int i = 0; i < R; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = H[i * R + j];
            for (int k = 0; k < j; ++k) s -= L[i * R + k] * L[j * R + k];
            if (i == j) {
                if (!(s > 0.0)) return 1;
                L[i * R + i] = sqrt(s);
            } else {
                L[i * R + j] = s / L[j * R + j];
            }
        }
    }
    return 0;
}

/* Round a double to the nearest bfloat16 value, ties to even.  bfloat16 is
 * the upper half of an IEEE binary32: 8 exponent bits (bias 127) and 8
 * significant bits (7 stored), so
 *   normal numbers, |x| >= 2^-126 : 8 significant bits;
 *   subnormals,     |x| <  2^-126 : multiples of 2^-133 (the spacing of
 *                                   the smallest normal binade);
 *   the largest finite value is (2 - 2^-7) * 2^127; anything that rounds
 *   past it becomes +-infinity.
 * The value is scaled by a power of two (exact) so that the kept bits are
 * its integer part, rounded with nearbyint (the default rounding mode,
 * nearest-even), and scaled back. */
static double round_bf16(double x)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    double m = frexp(x, &e);               /* x = m * 2^e, 0.5 <= |m| < 1 */
    int bits = e - 1 >= -126 ? 8 : e + 133; /* significant bits kept: x's leading
                                              bit is 2^(e-1), the last kept 2^-133 */
    double q = nearbyint(ldexp(m, bits));  /* bits <= 0: |m 2^bits| <= 1/2 -> 0 */
    double r = ldexp(q, e - bits);
    if (fabs(r) > ldexp(255.0, 120)) return copysign(INFINITY, x);
    return r;
}

/* Elementwise round_bf16 (exported so the rounding can be checked alone). */
void oracle_round_bf16(int64_t n, const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) y[i] = round_bf16(x[i]);
}

/* One CP-ALS iteration (all modes in order 0..d-1), in place.
 *   A[m]   : I_m x R (lda = R) current factors; overwritten.
 *   lambda : R weights (output).
 *   bf16   : nonzero -> round each updated factor to bf16 after normalizing.
 *   xnorm2 : ||X||^2 (coalesced, see oracle_norm2).
 *   fit    : output, 1 - ||X - M|| / ||X||.
 * Per mode n:
 *   V = MTTKRP_n(X, A) without weights;  H = *_{m != n} A^(m)^T A^(m)
 *   (elementwise product);  solve A^(n) H = V by Cholesky (one retry with a
 *   ridge of 1e-12 * trace(H)/R on the diagonal);  lambda_j = ||A^(n)(:,j)||_2
 *   and A^(n)(:,j) /= lambda_j for lambda_j > 0.
 * Fit, by definition: ||M||^2 = sum_{r,s} lambda_r lambda_s prod_m G_m(r,s);
 *   <X,M> = sum_i x_i M(l_i) with M(l) = sum_j lambda_j prod_m a^(m)(l_m, j);
 *   ||X - M||^2 = ||X||^2 + ||M||^2 - 2<X,M> (clamped at 0).
 * Returns 0, or 2 if a Gram-Hadamard matrix is not positive definite. */
int oracle_cp_als_iter(int d, const int64_t *dims, int64_t P, const int32_t *idx,
                       const double *vals, int R, double *const *A, double *lambda,
                       int bf16, double xnorm2, double *fit)
{
    int64_t *lda = (int64_t *)malloc(sizeof(int64_t) * (size_t)d);
    for (int m = 0; m < d; ++m) lda[m] = R;
    double *G = (double *)malloc(sizeof(double) * (size_t)d * R * R);
    double *H = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *L = (double *)malloc(sizeof(double) * (size_t)R * R);
    double *y = (double *)malloc(sizeof(double) * (size_t)R);
    int status = 0;
    for (int n = 0; n < d && status == 0; ++n) {
        int64_t In = dims[n];
        double *V = (double *)malloc(sizeof(double) * (size_t)In * R);
        oracle_mttkrp(d, dims, P, idx, vals, n, R, (const double *const *)A, lda, NULL, V, R);
        for (int m = 0; m < d; ++m) oracle_gram(dims[m], R, A[m], R, G + (size_t)m * R * R);
        for (int q = 0; q < R * R; ++q) {
            double h = 1.0;
            for (int m = 0; m < d; ++m) if (m != n) h *= G[(size_t)m * R * R + q];
            H[q] = h;
        }
        if (oracle_cholesky(R, H, L)) {
            double tr = 0.0;
            for (int r = 0; r < R; ++r) tr += H[r * R + r];
            for (int r = 0; r < R; ++r) H[r * R + r] += 1e-12 * tr / R;
            if (oracle_cholesky(R, H, L)) { status = 2; free(V); break; }
        }
        /* row by row: L y = v (forward), L^T a = y (backward) */
        for (int64_t k = 0; k < In; ++k) {
            const double *v = V + k * R;
            for (int r = 0; r < R; ++r) {
                double s = v[r];
                for (int c = 0; c < r; ++c) s -= L[r * R + c] * y[c];
                y[r] = s / L[r * R + r];
            }
            double *a = A[n] + k * R;
            for (int r = R - 1; r >= 0; --r) {
                double s = y[r];
                for (int c = r + 1; c < R; ++c) s -= L[c * R + r] * a[c];
                a[r] = s / L[r * R + r];
            }
        }
        for (int j = 0; j < R; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < In; ++k) s += A[n][k * R + j] * A[n][k * R + j];
            lambda[j] = sqrt(s);
            if (lambda[j] > 0.0)
                for (int64_t k = 0; k < In; ++k) A[n][k * R + j] /= lambda[j];
        }
        if (bf16)
            for (int64_t q = 0; q < In * R; ++q) A[n][q] = round_bf16(A[n][q]);
        free(V);
    }
    if (status == 0 && fit) {
        for (int m = 0; m < d; ++m) oracle_gram(dims[m], R, A[m], R, G + (size_t)m * R * R);
        double mnorm2 = 0.0;
        for (int r = 0; r < R; ++r)
            for (int s = 0; s < R; ++s) {
                double h = lambda[r] * lambda[s];
                for (int m = 0; m < d; ++m) h *= G[(size_t)m * R * R + r * R + s];
                mnorm2 += h;
            }
        double inner = 0.0;
        for (int64_t i = 0; i < P; ++i) {
            double mi = 0.0;
            for (int j = 0; j < R; ++j) {
                double t = lambda[j];
                for (int m = 0; m < d; ++m) t *= A[m][(int64_t)idx[(int64_t)m * P + i] * R + j];
                mi += t;
            }
            inner += vals[i] * mi;
        }
        double r2 = xnorm2 + mnorm2 - 2.0 * inner;
        if (r2 < 0.0) r2 = 0.0;
        *fit = 1.0 - sqrt(r2) / sqrt(xnorm2);
    }
    free(lda); free(G); free(H); free(L); free(y);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Generalised CP gradient (the count- and binary-data losses that Sec. 8   */
/* names as the next use of the MTTKRP machinery).  Model value of entry i: */
/*   m_i = sum_j prod_l a^(l)(i_l, j)                                        */
/* Loss F = sum over the loss's entry set of f(x, m); the gradient of F     */
/* with respect to A^(n) is                                                  */
/*   g(k, j) = sum_{entries e of the set, e_n = k} df/dm(x_e, m_e)           */
/*                                      * prod_{l != n} a^(l)(e_l, j).       */
/* loss 0, Poisson with identity link: f = m - x log m over EVERY entry of   */
/*   the tensor (x = 0 off the stored coordinates, a stored coordinate's x   */
/*   is the sum of its duplicates).  Off the stored coordinates df/dm = 1,   */
/*   and summing prod_{l != n} a^(l)(e_l, j) over all entries with e_n = k  */
/*   factorises into prod_{l != n} (sum_r a^(l)(r, j)); so                   */
/*     g(k, j) = prod_{l != n} colsum_l(j) - sum_{stored i, i_n = k}         */
/*               (x_i / m_i) prod_{l != n} a^(l)(i_l, j)                     */
/*     F = sum_j prod_l colsum_l(j) - sum_{stored i} x_i log m_i.            */
/* loss 1, Bernoulli with logit link: f = log(1 + e^m) - x m over the        */
/*   STORED entries (sampled zeros are stored explicitly by the caller; a    */
/*   duplicated coordinate counts once per copy).  df/dm = 1/(1+e^-m) - x.   */
/* loss 2, Gaussian: f = (m - x)^2 over the stored entries; df/dm = 2(m-x).  */
/* G: I_n x ldg (columns >= R set to 0).  Returns F.                          */
/* ---------------------------------------------------------------------- */
static double model_value(int d, int64_t P, const int32_t *idx, int64_t i, int R,
                          const double *const *A, const int64_t *lda)
{
    double m = 0.0;
    for (int j = 0; j < R; ++j) {
        double t = 1.0;
        for (int l = 0; l < d; ++l) t *= A[l][(int64_t)idx[(int64_t)l * P + i] * lda[l] + j];
        m += t;
    }
    return m;
}

double oracle_gcp_grad(int d, const int64_t *dims, int64_t P, const int32_t *idx,
                       const double *vals, int n, int R, const double *const *A,
                       const int64_t *lda, int loss, double *G, int64_t ldg)
{
    int64_t In = dims[n];
    memset(G, 0, sizeof(double) * (size_t)In * (size_t)ldg);
    double F = 0.0;
    for (int64_t i = 0; i < P; ++i) {
        double x = vals[i];
        double m = model_value(d, P, idx, i, R, A, lda);
        double y;
        if (loss == 0) {
            y = -x / m;                 /* the stored entry's part of 1 - x/m */
            F -= x * log(m);
        } else if (loss == 1) {
            y = 1.0 / (1.0 + exp(-m)) - x;
            F += (m > 0.0 ? m + log1p(exp(-m)) : log1p(exp(m))) - x * m;
        } else {
            y = 2.0 * (m - x);
            F += (m - x) * (m - x);
        }
        int64_t k = idx[(int64_t)n * P + i];
        for (int j = 0; j < R; ++j) {
            double t = y;
            for (int l = 0; l < d; ++l) {
                if (l == n) continue;
                t *= A[l][(int64_t)idx[(int64_t)l * P + i] * lda[l] + j];
            }
            G[k * ldg + j] += t;
        }
    }
    if (loss == 0) {
        /* the df/dm = 1 share of every entry of the tensor */
        for (int j = 0; j < R; ++j) {
            double c = 1.0, call = 1.0;
            for (int l = 0; l < d; ++l) {
                double cs = 0.0;
                for (int64_t r = 0; r < dims[l]; ++r) cs += A[l][r * lda[l] + j];
                call *= cs;
                if (l != n) c *= cs;
            }
            F += call;
            for (int64_t k = 0; k < In; ++k) G[k * ldg + j] += c;
        }
    }
    return F;
}

/* ---------------------------------------------------------------------- */
/* Schedule-selector network (not in the paper): a 3-layer perceptron       */
/*   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3             */
/* with W_l row-major (out x in), rows of X / Y are samples.                 */
/* Loss: masked mean squared error  (1/sum M) sum_{b,k} M_bk (y_bk - T_bk)^2 */
/* ---------------------------------------------------------------------- */
static void dense_fwd(int B, int In, int Out, const double *X, const double *W,
                      const double *b, double *Y, int relu)
{
    for (int s = 0; s < B; ++s)
        for (int o = 0; o < Out; ++o) {
            double acc = b[o];
            for (int i = 0; i < In; ++i) acc += W[o * In + i] * X[s * In + i];
            Y[s * Out + o] = (relu && acc < 0.0) ? 0.0 : acc;
        }
}

void oracle_mlp_forward(int B, int F, int H1, int H2, int K, const double *X,
                        const double *W1, const double *b1, const double *W2,
                        const double *b2, const double *W3, const double *b3,
                        double *h1, double *h2, double *Y)
{
    dense_fwd(B, F, H1, X, W1, b1, h1, 1);
    dense_fwd(B, H1, H2, h1, W2, b2, h2, 1);
    dense_fwd(B, H2, K, h2, W3, b3, Y, 0);
}

/* Returns the loss; writes dW*, db* (same shapes as the parameters). */
double oracle_mlp_loss_grad(int B, int F, int H1, int H2, int K, const double *X,
                            const double *W1, const double *b1, const double *W2,
                            const double *b2, const double *W3, const double *b3,
                            const double *T, const double *M, double *dW1, double *db1,
                            double *dW2, double *db2, double *dW3, double *db3)
{
    double *h1 = (double *)malloc(sizeof(double) * (size_t)B * H1);
    double *h2 = (double *)malloc(sizeof(double) * (size_t)B * H2);
    double *Y = (double *)malloc(sizeof(double) * (size_t)B * K);
    double *gY = (double *)malloc(sizeof(double) * (size_t)B * K);
    double *g2 = (double *)malloc(sizeof(double) * (size_t)B * H2);
    double *g1 = (double *)malloc(sizeof(double) * (size_t)B * H1);
    oracle_mlp_forward(B, F, H1, H2, K, X, W1, b1, W2, b2, W3, b3, h1, h2, Y);
    double msum = 0.0, loss = 0.0;
    for (int q = 0; q < B * K; ++q) msum += M[q];
    if (msum <= 0.0) msum = 1.0;
    for (int q = 0; q < B * K; ++q) {
        double e = Y[q] - T[q];
        loss += M[q] * e * e;
        gY[q] = 2.0 * M[q] * e / msum;
    }
    loss /= msum;
    /* layer 3 */
    memset(dW3, 0, sizeof(double) * (size_t)K * H2);
    memset(db3, 0, sizeof(double) * (size_t)K);
    for (int s = 0; s < B; ++s)
        for (int o = 0; o < K; ++o) {
            db3[o] += gY[s * K + o];
            for (int i = 0; i < H2; ++i) dW3[o * H2 + i] += gY[s * K + o] * h2[s * H2 + i];
        }
    for (int s = 0; s < B; ++s)
        for (int i = 0; i < H2; ++i) {
            double acc = 0.0;
            for (int o = 0; o < K; ++o) acc += W3[o * H2 + i] * gY[s * K + o];
            g2[s * H2 + i] = h2[s * H2 + i] > 0.0 ? acc : 0.0;
        }
    /* layer 2 */
    memset(dW2, 0, sizeof(double) * (size_t)H2 * H1);
    memset(db2, 0, sizeof(double) * (size_t)H2);
    for (int s = 0; s < B; ++s)
        for (int o = 0; o < H2; ++o) {
            db2[o] += g2[s * H2 + o];
            for (int i = 0; i < H1; ++i) dW2[o * H1 + i] += g2[s * H2 + o] * h1[s * H1 + i];
        }
    for (int s = 0; s < B; ++s)
        for (int i = 0; i < H1; ++i) {
            double acc = 0.0;
            for (int o = 0; o < H2; ++o) acc += W2[o * H1 + i] * g2[s * H2 + o];
            g1[s * H1 + i] = h1[s * H1 + i] > 0.0 ? acc : 0.0;
        }
    /* layer 1 */
    memset(dW1, 0, sizeof(double) * (size_t)H1 * F);
    memset(db1, 0, sizeof(double) * (size_t)H1);
    for (int s = 0; s < B; ++s)
        for (int o = 0; o < H1; ++o) {
            db1[o] += g1[s * H1 + o];
            for (int i = 0; i < F; ++i) dW1[o * F + i] += g1[s * H1 + o] * X[s * F + i];
        }
    free(h1); free(h2); free(Y); free(gY); free(g2); free(g1);
    return loss;
}
