/*
 * CPU oracle for the alignment itself (traceback, as a CIGAR) of a local
 * alignment already located by sw_oracle.c.  TEST INFRASTRUCTURE ONLY: the
 * tests call it; the CUDA library never does, and it shares no code with
 * the CUDA path.
 *
 * The paper's Fig. 2(c) ends the method with a traceback from the maximal
 * cell.  Given the outputs (S, qend, rend, qstart, rstart), every score-S
 * local alignment that ends at (qend, rend) and starts at (qstart, rstart)
 * is a global alignment of the substrings A' = a[qstart..qend] (N rows)
 * and B' = b[rstart..rend] (M columns) under the same affine scoring, and
 * no global alignment of them scores more (it would be a better local
 * alignment).  So the traceback is that of the global Gotoh recurrence:
 *
 *   H[0][0] = 0, H[0][j] = E[0][j] = go + (j-1) ge, H[i][0] = F[i][0] =
 *   go + (i-1) ge, E[i][0] = F[0][j] = -infinity, and for i, j >= 1
 *     E[i][j] = max(E[i][j-1] + ge, H[i][j-1] + go)     ends with D
 *     F[i][j] = max(F[i-1][j] + ge, H[i-1][j] + go)     ends with I
 *     H[i][j] = max(H[i-1][j-1] + s(a'_i, b'_j), E[i][j], F[i][j])
 *
 * whose H[N][M] equals S.  Ops (the SAM meanings, B' as the reference):
 * M aligns a query and a reference residue, I takes a query residue only,
 * D a reference residue only.  Among co-optimal alignments the path is
 * fixed by this rule, walking back from (N, M) in state H:
 *   state H: M if i, j >= 1 and H[i][j] = H[i-1][j-1] + s; else state E
 *            if H[i][j] = E[i][j]; else state F.
 *   state E: emit D; step to (i, j-1) in state H if E[i][j] = H[i][j-1] +
 *            go (the run opens here), else in state E.
 *   state F: emit I; step to (i-1, j) in state H if F[i][j] = H[i-1][j] +
 *            go, else in state F.
 * The ops, read forwards, are run-length encoded as (length << 4) | code
 * with M = 0, I = 1, D = 2 (the BAM numbering).  S = 0 gives no ops.
 *
 * Arithmetic is int64, -infinity = INT64_MIN / 4.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NEG_INF (INT64_MIN / 4)
#define OC_OK 0
#define OC_EINVAL (-1)
#define OC_ERANGE (-2)
#define OC_ENOMEM (-3)
#define OC_EINTERNAL (-9)

enum { OP_M = 0, OP_I = 1, OP_D = 2 };

static int64_t max2(int64_t a, int64_t b) { return a > b ? a : b; }

/* Appends one op (walking backwards) to the run-length list in `rev`. */
static int push_op(uint32_t *rev, int *n, int cap, int op) {
    if (*n > 0 && (int)(rev[*n - 1] & 15u) == op) {
        rev[*n - 1] += 16u;
        return OC_OK;
    }
    if (*n >= cap) return OC_ERANGE;
    rev[(*n)++] = (1u << 4) | (uint32_t)op;
    return OC_OK;
}

/*
 * Traceback of pair (a, n) x (b, m) whose local alignment is
 * (score, qend, rend, qstart, rstart).  Writes at most `cap` run-length ops
 * to `ops` (forward order) and their count to *n_ops; *global_score gets
 * H[N][M] (= score).  Returns OC_OK or an error code.
 */
int oracle_cigar(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, const int8_t *mat,
                 int32_t A, int32_t go, int32_t ge, const int32_t *res, uint32_t *ops,
                 int32_t cap, int32_t *n_ops, int64_t *global_score) {
    *n_ops = 0;
    *global_score = 0;
    if (A < 1 || A > 32 || ge > 0 || go > ge) return OC_EINVAL;
    const int32_t S = res[0], qend = res[1], rend = res[2], qstart = res[3], rstart = res[4];
    if (S <= 0) return OC_OK;
    if (qstart < 0 || qstart > qend || qend >= n || rstart < 0 || rstart > rend || rend >= m)
        return OC_EINVAL;
    const int64_t N = (int64_t)qend - qstart + 1, M = (int64_t)rend - rstart + 1;
    if ((N + 1) * (M + 1) > ((int64_t)1 << 26)) return OC_ERANGE;
    const uint8_t *qa = a + qstart, *rb = b + rstart;
    const int64_t W = M + 1;
    int64_t *H = malloc(sizeof(int64_t) * (size_t)((N + 1) * W));
    int64_t *E = malloc(sizeof(int64_t) * (size_t)((N + 1) * W));
    int64_t *F = malloc(sizeof(int64_t) * (size_t)((N + 1) * W));
    uint32_t *rev = malloc(sizeof(uint32_t) * (size_t)(N + M + 1));
    int rc = OC_OK;
    if (!H || !E || !F || !rev) {
        rc = OC_ENOMEM;
        goto done;
    }
    H[0] = 0;
    E[0] = F[0] = NEG_INF;
    for (int64_t j = 1; j <= M; ++j) {
        H[j] = E[j] = go + (j - 1) * (int64_t)ge;
        F[j] = NEG_INF;
    }
    for (int64_t i = 1; i <= N; ++i) {
        H[i * W] = F[i * W] = go + (i - 1) * (int64_t)ge;
        E[i * W] = NEG_INF;
        const int x = qa[i - 1] < A ? qa[i - 1] : A - 1;
        for (int64_t j = 1; j <= M; ++j) {
            const int y = rb[j - 1] < A ? rb[j - 1] : A - 1;
            const int64_t c = i * W + j;
            E[c] = max2(E[c - 1] + ge, H[c - 1] + go);
            F[c] = max2(F[c - W] + ge, H[c - W] + go);
            H[c] = max2(H[c - W - 1] + mat[x * A + y], max2(E[c], F[c]));
        }
    }
    *global_score = H[N * W + M];
    /* walk back from (N, M) in state H */
    int nr = 0, state = 0; /* 0 = H, 1 = E, 2 = F */
    int64_t i = N, j = M;
    while (i > 0 || j > 0) {
        const int64_t c = i * W + j;
        if (state == 0) {
            if (i > 0 && j > 0) {
                const int x = qa[i - 1] < A ? qa[i - 1] : A - 1;
                const int y = rb[j - 1] < A ? rb[j - 1] : A - 1;
                if (H[c] == H[c - W - 1] + mat[x * A + y]) {
                    if ((rc = push_op(rev, &nr, (int)(N + M), OP_M)) != OC_OK) goto done;
                    --i;
                    --j;
                    continue;
                }
            }
            if (j > 0 && H[c] == E[c])
                state = 1;
            else if (i > 0 && H[c] == F[c])
                state = 2;
            else {
                rc = OC_EINTERNAL;
                goto done;
            }
        } else if (state == 1) {
            if ((rc = push_op(rev, &nr, (int)(N + M), OP_D)) != OC_OK) goto done;
            const int open = E[c] == H[c - 1] + go;
            --j;
            if (open) state = 0;
        } else {
            if ((rc = push_op(rev, &nr, (int)(N + M), OP_I)) != OC_OK) goto done;
            const int open = F[c] == H[c - W] + go;
            --i;
            if (open) state = 0;
        }
    }
    if (nr > cap) {
        rc = OC_ERANGE;
        goto done;
    }
    for (int k = 0; k < nr; ++k) ops[k] = rev[nr - 1 - k];
    *n_ops = nr;
done:
    free(H);
    free(E);
    free(F);
    free(rev);
    return rc;
}

/* ---- batch over host threads */

struct cig_job {
    const uint8_t *q, *r;
    const int64_t *qo, *ro, *co;
    const int32_t *res;
    const int8_t *mat;
    int32_t A, go, ge, n_pairs;
    uint32_t *ops;
    int32_t *n_ops;
    int32_t *status;
    int next;
    pthread_mutex_t mu;
};

static void *cig_worker(void *arg) {
    struct cig_job *jb = arg;
    for (;;) {
        pthread_mutex_lock(&jb->mu);
        const int p = jb->next++;
        pthread_mutex_unlock(&jb->mu);
        if (p >= jb->n_pairs) break;
        int64_t g = 0;
        jb->status[p] = oracle_cigar(jb->q + jb->qo[p], jb->qo[p + 1] - jb->qo[p],
                                     jb->r + jb->ro[p], jb->ro[p + 1] - jb->ro[p], jb->mat, jb->A,
                                     jb->go, jb->ge, jb->res + 5 * (int64_t)p,
                                     jb->ops + jb->co[p], (int32_t)(jb->co[p + 1] - jb->co[p]),
                                     jb->n_ops + p, &g);
    }
    return NULL;
}

/*
 * Batch form: results are n_pairs x 5 (row-major, as oracle_align_batch
 * writes them); cig_off[p] .. cig_off[p+1] is pair p's room in ops.
 */
int oracle_cigar_batch(const uint8_t *q, const int64_t *qo, const uint8_t *r, const int64_t *ro,
                       int32_t n_pairs, const int8_t *mat, int32_t A, int32_t go, int32_t ge,
                       const int32_t *res, const int64_t *cig_off, uint32_t *ops, int32_t *n_ops,
                       int32_t *status, int32_t threads) {
    struct cig_job jb = {q, r, qo, ro, cig_off, res, mat, A, go, ge, n_pairs, ops, n_ops,
                         status, 0, PTHREAD_MUTEX_INITIALIZER};
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&th[t], NULL, cig_worker, &jb) == 0) ++started;
    if (started == 0) cig_worker(&jb);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    for (int p = 0; p < n_pairs; ++p)
        if (status[p] != OC_OK) return status[p];
    return OC_OK;
}
