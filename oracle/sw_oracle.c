/*
 * CPU oracle for batched Smith-Waterman local alignment with affine (Gotoh)
 * gaps.  TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg call it; the CUDA library never does.  It
 * shares no code with the CUDA path.
 *
 * What it computes (paper Section II-B.1 and Fig. 2):
 *   A = a_1..a_n (query, matrix rows), B = b_1..b_m (reference, columns).
 *   H is an (n+1) x (m+1) scoring matrix whose cell H[i][j] is the best score
 *   of an alignment ending with a_i and b_j, floored at zero; it is filled
 *   top-left to bottom-right from its diagonal, upper and left neighbours.
 *   Gaps are affine as in the E update of Fig. 8 ("E = prev E + extendGap"
 *   against "H + startGap"): a gap of length k costs go + (k-1)*ge.
 *     E[i][j] = max(H[i][j-1] + go, E[i][j-1] + ge)   (gap in the query)
 *     F[i][j] = max(H[i-1][j] + go, F[i-1][j] + ge)   (gap in the reference)
 *     H[i][j] = max(0, H[i-1][j-1] + s(a_i, b_j), E[i][j], F[i][j])
 *   with H[i][0] = H[0][j] = 0 and E[i][0] = F[0][j] = -infinity.
 *
 * Outputs (0-based residue indices, inclusive):
 *   score = S = max H.
 *   (qend, rend): among cells with H = S the smallest rend, then the
 *     smallest qend.
 *   (qstart, rstart): the forward pass of Fig. 2(a) is followed by a reverse
 *     pass (Fig. 2(c); ADEPT's second kernel, Section III-B).  Here the
 *     reverse pass is the same recurrence run on the reversed prefixes
 *     a_qend..a_0 and b_rend..b_0; its maximum is S again, and the same
 *     end rule applied in reversed coordinates (smallest reversed column,
 *     then smallest reversed row) gives rstart = rend - l, qstart = qend - k.
 *     Every score-S alignment inside [0..qend]x[0..rend] ends at
 *     (qend, rend), so this selects, among the score-S alignments ending
 *     there, the largest rstart and then the largest qstart.
 *   S = 0 (including n = 0 or m = 0): score 0 and all coordinates -1.
 *
 * Precondition: go <= ge <= 0 (a gap is never cheaper to open than to
 * extend); other values are rejected.
 *
 * Arithmetic is int64 with -infinity = INT64_MIN / 4, so no input the
 * library accepts can overflow here.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NEG_INF (INT64_MIN / 4)

/* Status codes returned by the oracle entry points. */
#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-3)
#define OR_EINTERNAL (-9)

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/*
 * One forward pass of the recurrence above over a (length n) vs b (length m),
 * whose residues are fetched through a stride so that the same loop reads a
 * sequence forwards (step +1) or backwards (step -1).  Returns the maximum
 * score and the (row, column) of the chosen maximal cell, 0-based, or -1/-1
 * when the maximum is 0.
 */
static int forward_pass(const uint8_t *a, int64_t a_step, int64_t n,
                        const uint8_t *b, int64_t b_step, int64_t m,
                        const int8_t *mat, int32_t alpha, int64_t go, int64_t ge,
                        int64_t *best, int64_t *bi, int64_t *bj) {
    *best = 0;
    *bi = -1;
    *bj = -1;
    if (n <= 0 || m <= 0) return OR_OK;
    int64_t *h_prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *h_cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *f = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!h_prev || !h_cur || !f) {
        free(h_prev); free(h_cur); free(f);
        return OR_ENOMEM;
    }
    for (int64_t j = 0; j <= m; ++j) {
        h_prev[j] = 0;          /* H[0][j] = 0 */
        f[j] = NEG_INF;         /* F[0][j] = -inf */
    }
    for (int64_t i = 1; i <= n; ++i) {
        const int ai = a[(i - 1) * a_step];
        h_cur[0] = 0;           /* H[i][0] = 0 */
        int64_t e = NEG_INF;    /* E[i][0] = -inf */
        for (int64_t j = 1; j <= m; ++j) {
            const int bj_res = b[(j - 1) * b_step];
            e = max2(h_cur[j - 1] + go, e + ge);
            f[j] = max2(h_prev[j] + go, f[j] + ge);
            int64_t h = h_prev[j - 1] + (int64_t)mat[ai * alpha + bj_res];
            h = max2(h, e);
            h = max2(h, f[j]);
            h = max2(h, 0);
            h_cur[j] = h;
            /* end rule: larger score; then smaller column; then smaller row */
            if (h > *best || (h == *best && h > 0 &&
                              (j - 1 < *bj || (j - 1 == *bj && i - 1 < *bi)))) {
                *best = h;
                *bi = i - 1;
                *bj = j - 1;
            }
        }
        int64_t *t = h_prev; h_prev = h_cur; h_cur = t;
    }
    free(h_prev); free(h_cur); free(f);
    if (*best == 0) { *bi = -1; *bj = -1; }
    return OR_OK;
}

static int check_residues(const uint8_t *s, int64_t n, int32_t alpha) {
    for (int64_t k = 0; k < n; ++k)
        if (s[k] >= alpha) return OR_EINVAL;
    return OR_OK;
}

/*
 * Align one pair.  out[0..4] = score, qend, rend, qstart, rstart.
 * Returns OR_OK, OR_EINVAL (bad residue / arguments), OR_ENOMEM, or
 * OR_EINTERNAL if the reverse pass does not reproduce the forward score.
 */
int oracle_align(const uint8_t *q, int64_t n, const uint8_t *r, int64_t m,
                 const int8_t *mat, int32_t alpha, int32_t gap_open,
                 int32_t gap_extend, int32_t *out) {
    if (n < 0 || m < 0 || alpha < 1 || !mat || !out) return OR_EINVAL;
    /* The recurrence equals the run-cost definition only when opening a gap
     * costs at least as much as extending one (go <= ge <= 0): otherwise two
     * adjacent runs charged go each beat one run charged go + ge. */
    if (gap_extend > 0 || gap_open > gap_extend) return OR_EINVAL;
    if (check_residues(q, n, alpha) || check_residues(r, m, alpha)) return OR_EINVAL;
    int64_t s, qe, re;
    int rc = forward_pass(q, 1, n, r, 1, m, mat, alpha, gap_open, gap_extend, &s, &qe, &re);
    if (rc) return rc;
    out[0] = (int32_t)s;
    out[1] = (int32_t)qe;
    out[2] = (int32_t)re;
    out[3] = -1;
    out[4] = -1;
    if (s == 0) return OR_OK;
    /* reverse pass over the reversed prefixes a_qend..a_0 and b_rend..b_0 */
    int64_t s2, k, l;
    rc = forward_pass(q + qe, -1, qe + 1, r + re, -1, re + 1, mat, alpha, gap_open,
                      gap_extend, &s2, &k, &l);
    if (rc) return rc;
    if (s2 != s) return OR_EINTERNAL;
    out[3] = (int32_t)(qe - k);
    out[4] = (int32_t)(re - l);
    return OR_OK;
}

/* ----------------------------------------------------------- batch runner */

typedef struct {
    const uint8_t *q_seqs, *r_seqs;
    const int64_t *q_off, *r_off;
    int32_t n_pairs;
    const int8_t *mat;
    int32_t alpha, go, ge;
    int32_t *out;           /* n_pairs x 5, row-major */
    int32_t *status;        /* n_pairs */
    int64_t next;           /* shared work counter */
    pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *job = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t lo = job->next;
        job->next += 16;
        pthread_mutex_unlock(&job->lock);
        if (lo >= job->n_pairs) break;
        int64_t hi = lo + 16 < job->n_pairs ? lo + 16 : job->n_pairs;
        for (int64_t p = lo; p < hi; ++p) {
            job->status[p] = oracle_align(
                job->q_seqs + job->q_off[p], job->q_off[p + 1] - job->q_off[p],
                job->r_seqs + job->r_off[p], job->r_off[p + 1] - job->r_off[p],
                job->mat, job->alpha, job->go, job->ge, job->out + 5 * p);
        }
    }
    return NULL;
}

/*
 * Align every pair of a CSR batch on nthreads host threads (one pair per
 * task).  out is n_pairs x 5 (score, qend, rend, qstart, rstart); status
 * receives each pair's return code.  Returns the first non-OK status, or OK.
 */
int oracle_align_batch(const uint8_t *q_seqs, const int64_t *q_off,
                       const uint8_t *r_seqs, const int64_t *r_off, int32_t n_pairs,
                       const int8_t *mat, int32_t alpha, int32_t gap_open,
                       int32_t gap_extend, int32_t *out, int32_t *status,
                       int32_t nthreads) {
    if (n_pairs < 0 || nthreads < 1) return OR_EINVAL;
    batch_job job;
    job.q_seqs = q_seqs; job.r_seqs = r_seqs; job.q_off = q_off; job.r_off = r_off;
    job.n_pairs = n_pairs; job.mat = mat; job.alpha = alpha;
    job.go = gap_open; job.ge = gap_extend; job.out = out; job.status = status;
    job.next = 0;
    pthread_mutex_init(&job.lock, NULL);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return OR_ENOMEM;
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &job) == 0) ++started;
    if (started == 0) batch_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
    for (int32_t p = 0; p < n_pairs; ++p)
        if (status[p] != OR_OK) return status[p];
    return OR_OK;
}
