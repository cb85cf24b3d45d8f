/*
 * oracle.c -- plain, slow CPU reference for FST Viterbi and forward-backward.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes (Argueta & Chiang, "Decoding with Finite-State
 * Transducers on GPUs", EACL 2017):
 *
 *   weight(w) = s^T (prod_t delta[w_t]) f                       (Eq. 1)
 *
 * evaluated in two semirings over natural-log weights theta = log p:
 *
 *   - Viterbi (Sec. 3, the (p, k) pair semiring; Alg. 1): max-plus in
 *     float32.  Each candidate is one float32 addition; arcs of the slice
 *     are visited in ascending caller arc id and a candidate replaces the
 *     current value only if strictly larger, so ties go to the lowest arc
 *     id; a -inf candidate never sets a backpointer.  The final choice over
 *     states takes the lowest state id on ties.
 *   - Forward-backward (Alg. 2): log-sum-exp in float64.  Expected counts
 *     are kept per arc (not per state pair), so parallel arcs stay distinct.
 *
 * Readings of the paper (where it is silent or ambiguous):
 *   - log domain throughout; the start vector s is a per-state log-weight
 *     (-inf = not a start), f likewise (-inf = not final);
 *   - alpha entries that the recursion does not reach are -inf (Alg. 1 and 2
 *     leave them implicitly zero in the probability domain);
 *   - log-sum-exp of an empty set, or of only -inf terms, is -inf (Eq. 3
 *     would produce NaN from -inf - -inf);
 *   - the delta[w] in the count update of Alg. 2 is delta[w_{t+1}].
 *
 * Training (Sec. 4: the expected counts serve EM): oracle_em_update sets
 * each state's outgoing arc weights to its normalised expected counts.
 *
 * Parity status: every function below is pinned by the non-GPU tests
 * (worked example of Figs. 1-2, brute-force path enumeration, a dense HMM,
 * single-state and unweighted closed forms, the alpha-beta invariants; for
 * the EM update the worked example's counts, per-state normalisation, the
 * pseudo-count closed form and the monotone likelihood of EM).
 *
 * Build: gcc -O2 -ffp-contract=off -std=c11 -shared -fPIC (no FMA
 * contraction, so each float32 candidate is one rounded addition).
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID 1
#define OR_NO_PATH 2
#define OR_OOM 3

/* Arcs grouped by input symbol, ascending arc id within each symbol: the
 * R offsets and slice of Sec. 4 / Fig. 2, built by a counting sort. */
typedef struct {
    int32_t m;
    int64_t *off;   /* [m+1] */
    int64_t *arcs;  /* [A]   */
} sym_index;

/* The slices delta[a] of Sec. 4 / Fig. 2: the R offsets and the arcs of each
 * input symbol, by a counting sort over the arcs. */
static int build_index(int64_t A, const int32_t *ilabel, int32_t m, sym_index *ix)
{
    ix->m = m;
    ix->off = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    ix->arcs = (int64_t *)malloc((size_t)(A > 0 ? A : 1) * sizeof(int64_t));
    if (!ix->off || !ix->arcs) return OR_OOM;
    for (int64_t k = 0; k < A; ++k) ix->off[ilabel[k] + 1] += 1;
    for (int32_t a = 0; a < m; ++a) ix->off[a + 1] += ix->off[a];
    int64_t *fill = (int64_t *)malloc((size_t)m * sizeof(int64_t) + 1);
    if (!fill) return OR_OOM;
    for (int32_t a = 0; a < m; ++a) fill[a] = ix->off[a];
    for (int64_t k = 0; k < A; ++k) ix->arcs[fill[ilabel[k]]++] = k;
    free(fill);
    return OR_OK;
}

/* Release a slice index (no counterpart in the paper). */
static void free_index(sym_index *ix)
{
    free(ix->off);
    free(ix->arcs);
}

typedef struct {
    int32_t Q;
    int64_t A;
    const int32_t *src, *dst, *ilabel;
    const float *theta, *theta_s, *theta_f;
    int32_t m;
} fst_view;

/* ---------------------------------------------------------------------- */
/* Viterbi, float32 max-plus (Sec. 3 pair semiring; Alg. 1; backtrace of   */
/* Sec. 5.1).                                                               */
/* ---------------------------------------------------------------------- */
static int viterbi_one(const fst_view *f, const sym_index *ix, const int32_t *x, int32_t n,
                       float *best_out, int32_t *final_state, int32_t *path,
                       float *V_out, int32_t *bp_out)
{
    const int32_t Q = f->Q;
    for (int32_t t = 0; t < n; ++t)
        if (x[t] < 0 || x[t] >= f->m) return OR_INVALID;
    float *prev = (float *)malloc((size_t)Q * sizeof(float));
    float *cur = (float *)malloc((size_t)Q * sizeof(float));
    int32_t *bp = bp_out ? bp_out : (int32_t *)malloc((size_t)(n > 0 ? n : 1) * (size_t)Q * sizeof(int32_t));
    if (!prev || !cur || !bp) { free(prev); free(cur); if (!bp_out) free(bp); return OR_OOM; }

    /* V_0 = s */
    for (int32_t q = 0; q < Q; ++q) prev[q] = f->theta_s[q];
    if (V_out) memcpy(V_out, prev, (size_t)Q * sizeof(float));

    for (int32_t t = 1; t <= n; ++t) {
        int32_t *bpt = bp + (size_t)(t - 1) * Q;
        for (int32_t q = 0; q < Q; ++q) { cur[q] = -INFINITY; bpt[q] = -1; }
        const int32_t a = x[t - 1];
        for (int64_t j = ix->off[a]; j < ix->off[a + 1]; ++j) {
            const int64_t k = ix->arcs[j];             /* ascending arc id */
            const float c = prev[f->src[k]] + f->theta[k];  /* one float32 add */
            const int32_t q2 = f->dst[k];
            if (c > cur[q2]) { cur[q2] = c; bpt[q2] = (int32_t)k; }
        }
        float *tmp = prev; prev = cur; cur = tmp;
        if (V_out) memcpy(V_out + (size_t)t * Q, prev, (size_t)Q * sizeof(float));
    }

    /* best = max_q V_n[q] + f[q], lowest q on ties */
    float best = -INFINITY;
    int32_t qb = -1;
    for (int32_t q = 0; q < Q; ++q) {
        const float c = prev[q] + f->theta_f[q];
        if (c > best) { best = c; qb = q; }
    }
    *best_out = best;
    if (final_state) *final_state = qb;
    int rc = OR_OK;
    if (qb < 0) {
        for (int32_t t = 0; t < n; ++t) path[t] = -1;
        rc = OR_NO_PATH;
    } else {
        int32_t q = qb;
        for (int32_t t = n; t >= 1; --t) {
            const int32_t k = bp[(size_t)(t - 1) * Q + q];
            path[t - 1] = k;
            q = f->src[k];
        }
    }
    free(prev); free(cur);
    if (!bp_out) free(bp);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Forward-backward, float64 log-sum-exp (Alg. 2; Eq. 3 read as a plain    */
/* two-pass log-sum-exp).                                                   */
/* ---------------------------------------------------------------------- */

/* One forward step of Alg. 2: out[q'] = LSE_{k in slice, dst_k = q'}
 * (in[src_k] + theta_k).  With `reverse`, the roles of src and dst swap
 * (backward step). */
static void lse_step(const fst_view *f, const sym_index *ix, int32_t a, const double *in,
                     double *out, double *mx, int reverse)
{
    const int32_t Q = f->Q;
    const int32_t *from = reverse ? f->dst : f->src;
    const int32_t *to = reverse ? f->src : f->dst;
    for (int32_t q = 0; q < Q; ++q) { mx[q] = -INFINITY; out[q] = 0.0; }
    for (int64_t j = ix->off[a]; j < ix->off[a + 1]; ++j) {
        const int64_t k = ix->arcs[j];
        const double v = in[from[k]] + (double)f->theta[k];
        if (v > mx[to[k]]) mx[to[k]] = v;
    }
    for (int64_t j = ix->off[a]; j < ix->off[a + 1]; ++j) {
        const int64_t k = ix->arcs[j];
        const double v = in[from[k]] + (double)f->theta[k];
        if (mx[to[k]] > -INFINITY) out[to[k]] += exp(v - mx[to[k]]);
    }
    for (int32_t q = 0; q < Q; ++q)
        out[q] = (mx[q] > -INFINITY) ? mx[q] + log(out[q]) : -INFINITY;
}

/* Alg. 2 for one string: the forward and backward loops, log Z, and the
 * expected count of each arc (per arc, reading R6). */
static int fb_one(const fst_view *f, const sym_index *ix, const int32_t *x, int32_t n,
                  double scale, double *logz_out, double *counts /* += scale*gamma */,
                  double *alpha_out, double *beta_out)
{
    const int32_t Q = f->Q;
    for (int32_t t = 0; t < n; ++t)
        if (x[t] < 0 || x[t] >= f->m) return OR_INVALID;
    const size_t rows = (size_t)n + 1;
    double *al = alpha_out ? alpha_out : (double *)malloc(rows * (size_t)Q * sizeof(double));
    double *be = beta_out ? beta_out : (double *)malloc(rows * (size_t)Q * sizeof(double));
    double *mx = (double *)malloc((size_t)Q * sizeof(double));
    if (!al || !be || !mx) {
        if (!alpha_out) free(al);
        if (!beta_out) free(be);
        free(mx);
        return OR_OOM;
    }
    /* forward: alpha_0 = s; alpha_t = LSE over slice w_t */
    for (int32_t q = 0; q < Q; ++q) al[q] = (double)f->theta_s[q];
    for (int32_t t = 1; t <= n; ++t)
        lse_step(f, ix, x[t - 1], al + (size_t)(t - 1) * Q, al + (size_t)t * Q, mx, 0);
    /* backward: beta_n = f; beta_{t-1} = LSE over slice w_t, reduced by source */
    for (int32_t q = 0; q < Q; ++q) be[(size_t)n * Q + q] = (double)f->theta_f[q];
    for (int32_t t = n; t >= 1; --t)
        lse_step(f, ix, x[t - 1], be + (size_t)t * Q, be + (size_t)(t - 1) * Q, mx, 1);
    /* Z = sum_q alpha_n[q] f[q]  (log domain, two-pass) */
    double m = -INFINITY;
    for (int32_t q = 0; q < Q; ++q) {
        const double v = al[(size_t)n * Q + q] + (double)f->theta_f[q];
        if (v > m) m = v;
    }
    double logz = -INFINITY;
    if (m > -INFINITY) {
        double s = 0.0;
        for (int32_t q = 0; q < Q; ++q)
            s += exp(al[(size_t)n * Q + q] + (double)f->theta_f[q] - m);
        logz = m + log(s);
    }
    *logz_out = logz;
    /* expected counts: count[k] += alpha_{t-1}[src] * delta_k * beta_t[dst] / Z */
    if (counts && logz > -INFINITY) {
        for (int32_t t = 1; t <= n; ++t) {
            const int32_t a = x[t - 1];
            for (int64_t j = ix->off[a]; j < ix->off[a + 1]; ++j) {
                const int64_t k = ix->arcs[j];
                const double e = al[(size_t)(t - 1) * Q + f->src[k]] + (double)f->theta[k]
                                 + be[(size_t)t * Q + f->dst[k]] - logz;
                counts[k] += scale * exp(e);
            }
        }
    }
    if (!alpha_out) free(al);
    if (!beta_out) free(be);
    free(mx);
    return logz > -INFINITY ? OR_OK : OR_NO_PATH;
}

/* The FST of Sec. 3 is well formed: states and labels in range, no NaN and
 * no +inf log-weight (reading R1). */
static int check_fst(const fst_view *f)
{
    if (f->Q <= 0 || f->A < 0 || f->m <= 0) return OR_INVALID;
    for (int64_t k = 0; k < f->A; ++k) {
        if (f->src[k] < 0 || f->src[k] >= f->Q || f->dst[k] < 0 || f->dst[k] >= f->Q) return OR_INVALID;
        if (f->ilabel[k] < 0 || f->ilabel[k] >= f->m) return OR_INVALID;
        if (isnan(f->theta[k]) || f->theta[k] == INFINITY) return OR_INVALID;
    }
    for (int32_t q = 0; q < f->Q; ++q) {
        if (isnan(f->theta_s[q]) || f->theta_s[q] == INFINITY) return OR_INVALID;
        if (isnan(f->theta_f[q]) || f->theta_f[q] == INFINITY) return OR_INVALID;
    }
    return OR_OK;
}

#define FST_ARGS int32_t Q, int64_t A, const int32_t *src, const int32_t *dst, \
    const int32_t *ilabel, const float *theta, const float *theta_s, const float *theta_f, int32_t m
#define FST_VIEW fst_view f = {Q, A, src, dst, ilabel, theta, theta_s, theta_f, m}

/* Single string, Viterbi (Alg. 1, Sec. 5.1).  V_out [(n+1)*Q] and bp_out
 * [n*Q] are optional. */
int oracle_viterbi(FST_ARGS, const int32_t *x, int32_t n, float *best, int32_t *final_state,
                   int32_t *path, float *V_out, int32_t *bp_out)
{
    FST_VIEW;
    if (check_fst(&f) != OR_OK || n < 0) return OR_INVALID;
    sym_index ix;
    if (build_index(A, ilabel, m, &ix) != OR_OK) { free_index(&ix); return OR_OOM; }
    const int rc = viterbi_one(&f, &ix, x, n, best, final_state, path, V_out, bp_out);
    free_index(&ix);
    return rc;
}

/* Single string, forward-backward (Alg. 2, Sec. 5.2).  counts [A] receives
 * sum_t gamma_t(k) (it is overwritten); alpha_out / beta_out [(n+1)*Q] are
 * optional. */
int oracle_forward_backward(FST_ARGS, const int32_t *x, int32_t n, double *logz,
                            double *counts, double *alpha_out, double *beta_out)
{
    FST_VIEW;
    if (check_fst(&f) != OR_OK || n < 0) return OR_INVALID;
    sym_index ix;
    if (build_index(A, ilabel, m, &ix) != OR_OK) { free_index(&ix); return OR_OOM; }
    if (counts) memset(counts, 0, (size_t)(A > 0 ? A : 1) * sizeof(double));
    const int rc = fb_one(&f, &ix, x, n, 1.0, logz, counts, alpha_out, beta_out);
    free_index(&ix);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Batches over threads (sentence-parallel; used for timing and for the    */
/* large parity cases).                                                     */
/* ---------------------------------------------------------------------- */
typedef struct {
    const fst_view *f;
    const sym_index *ix;
    const int32_t *ids;
    const int64_t *off;
    int32_t B;
    int kind;                /* 0 = viterbi, 1 = forward-backward */
    atomic_int next;
    /* viterbi outputs */
    float *best;
    int32_t *paths;
    /* fb outputs */
    const double *weights;
    double *logz;
    double *counts;          /* [nthreads][A] partials */
    int32_t *status;
    atomic_int fail;
} batch_job;

typedef struct { batch_job *job; int tid; } batch_arg;

/* One thread of a batch: Alg. 1 or Alg. 2 string by string, unchanged (the
 * strings are independent; threads only split the batch). */
static void *batch_worker(void *p)
{
    batch_arg *arg = (batch_arg *)p;
    batch_job *j = arg->job;
    for (;;) {
        const int b = atomic_fetch_add(&j->next, 1);
        if (b >= j->B) break;
        const int32_t *x = j->ids + j->off[b];
        const int32_t n = (int32_t)(j->off[b + 1] - j->off[b]);
        int rc;
        if (j->kind == 0) {
            rc = viterbi_one(j->f, j->ix, x, n, &j->best[b], NULL, j->paths + j->off[b], NULL, NULL);
        } else {
            const double sc = j->weights ? j->weights[b] : 1.0;
            double *cnt = j->counts ? j->counts + (size_t)arg->tid * (size_t)j->f->A : NULL;
            rc = fb_one(j->f, j->ix, x, n, sc, &j->logz[b], cnt, NULL, NULL);
        }
        j->status[b] = rc;
        if (rc == OR_OOM || rc == OR_INVALID) atomic_store(&j->fail, rc);
    }
    return NULL;
}

/* Start the batch's threads and wait for them (no counterpart in the paper). */
static int run_batch(batch_job *job, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    batch_arg args[256];
    atomic_store(&job->next, 0);
    atomic_store(&job->fail, 0);
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        args[i].job = job;
        args[i].tid = i;
        if (nthreads == 1) { batch_worker(&args[i]); started = 0; break; }
        if (pthread_create(&th[i], NULL, batch_worker, &args[i]) != 0) break;
        ++started;
    }
    if (nthreads > 1 && started == 0) batch_worker(&args[0]);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return atomic_load(&job->fail);
}

/* Alg. 1 for every string of a batch (ids, off as the batched calls). */
int oracle_viterbi_batch(FST_ARGS, const int32_t *ids, const int64_t *off, int32_t B,
                         int32_t nthreads, float *best, int32_t *paths, int32_t *status)
{
    FST_VIEW;
    if (check_fst(&f) != OR_OK || B < 0) return OR_INVALID;
    sym_index ix;
    if (build_index(A, ilabel, m, &ix) != OR_OK) { free_index(&ix); return OR_OOM; }
    batch_job job;
    memset(&job, 0, sizeof(job));
    job.f = &f; job.ix = &ix; job.ids = ids; job.off = off; job.B = B; job.kind = 0;
    job.best = best; job.paths = paths; job.status = status;
    const int rc = run_batch(&job, nthreads);
    free_index(&ix);
    return rc;
}

/* Alg. 2 for every string of a batch.  counts_sum [A] (optional) receives
 * sum_b weights[b] * count_b (weights NULL = all 1). */
int oracle_fb_batch(FST_ARGS, const int32_t *ids, const int64_t *off, int32_t B,
                    int32_t nthreads, const double *weights, double *logz,
                    double *counts_sum, int32_t *status)
{
    FST_VIEW;
    if (check_fst(&f) != OR_OK || B < 0) return OR_INVALID;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    sym_index ix;
    if (build_index(A, ilabel, m, &ix) != OR_OK) { free_index(&ix); return OR_OOM; }
    double *part = NULL;
    if (counts_sum) {
        part = (double *)calloc((size_t)nthreads * (size_t)(A > 0 ? A : 1), sizeof(double));
        if (!part) { free_index(&ix); return OR_OOM; }
    }
    batch_job job;
    memset(&job, 0, sizeof(job));
    job.f = &f; job.ix = &ix; job.ids = ids; job.off = off; job.B = B; job.kind = 1;
    job.weights = weights; job.logz = logz; job.counts = part; job.status = status;
    const int rc = run_batch(&job, nthreads);
    if (counts_sum) {
        for (int64_t k = 0; k < A; ++k) {
            double s = 0.0;
            for (int i = 0; i < nthreads; ++i) s += part[(size_t)i * (size_t)A + k];
            counts_sum[k] = s;
        }
        free(part);
    }
    free_index(&ix);
    return rc;
}

/*
 * EM re-estimation of the arc weights from expected counts (the use the
 * paper gives the counts of Alg. 2: training by expectation-maximisation,
 * Sec. 4).  Each state's outgoing arcs form one categorical distribution, so
 * the M-step sets
 *
 *     p'_k = (count_k + alpha) / sum_{j: src_j = src_k} (count_j + alpha)
 *
 * (alpha >= 0 a pseudo-count added to every arc) and returns theta'_k =
 * log p'_k in float64.  A state whose arcs have a zero total (never used and
 * alpha = 0) keeps its arcs' old log-weights.
 */
int oracle_em_update(int32_t Q, int64_t A, const int32_t *src, const double *counts, const float *theta,
                     double alpha, double *theta_out)
{
    if (Q < 1 || A < 0 || !(alpha >= 0.0)) return OR_INVALID;
    for (int64_t k = 0; k < A; ++k)
        if (src[k] < 0 || src[k] >= Q || !(counts[k] >= 0.0)) return OR_INVALID;
    double *total = (double *)calloc((size_t)Q, sizeof(double));
    if (!total) return OR_OOM;
    for (int64_t k = 0; k < A; ++k) total[src[k]] += counts[k] + alpha;
    for (int64_t k = 0; k < A; ++k) {
        const double t = total[src[k]];
        theta_out[k] = t > 0.0 ? log((counts[k] + alpha) / t) : (double)theta[k];
    }
    free(total);
    return OR_OK;
}
