/*
 * Brute-force local alignment by enumeration.  TEST INFRASTRUCTURE ONLY: it
 * pins the oracle to the definition of a local alignment, not to any
 * recurrence, and is meant for sequences of at most about 8 residues.
 *
 * Definition (paper Section II-B.1, with the affine gap model of Fig. 8):
 * a local alignment starts at 0-based positions (x, y) and is a string of
 * operations M (a residue of each sequence, scored s(a, b)), D (a query
 * residue against a gap) and I (a reference residue against a gap).  Its
 * score is the sum of the M scores plus, for every maximal run of k equal
 * gap operations, go + (k-1)*ge; an I run and a D run that touch are two
 * runs.  If the operations consume a_x..a_{i-1} and b_y..b_{j-1}, the
 * alignment ends at (i-1, j-1).  S is the best score over all alignments,
 * or 0.  End rule: among alignments of score S, the smallest end column,
 * then the smallest end row.  Start rule: among alignments of score S that
 * end there, the largest start column, then the largest start row.
 *
 * Every alignment is enumerated explicitly; nothing is memoised.
 */
#include <stdint.h>

typedef struct {
    const uint8_t *a, *b;
    int64_t n, m;
    const int8_t *mat;
    int32_t alpha;
    int64_t go, ge;
    int phase;                 /* 1: find S and end; 2: find start */
    int64_t x0, y0;            /* current start */
    int64_t best, qend, rend;  /* phase 1 result */
    int64_t qstart, rstart;    /* phase 2 result */
    int64_t visited;
} brute_ctx;

enum { OP_NONE = 0, OP_M = 1, OP_I = 2, OP_D = 3 };

static void consider(brute_ctx *c, int64_t score, int64_t ie, int64_t je) {
    if (c->phase == 1) {
        if (score <= 0) return;
        if (score > c->best ||
            (score == c->best && (je < c->rend || (je == c->rend && ie < c->qend)))) {
            c->best = score; c->qend = ie; c->rend = je;
        }
    } else {
        if (score != c->best || ie != c->qend || je != c->rend) return;
        if (c->y0 > c->rstart || (c->y0 == c->rstart && c->x0 > c->qstart)) {
            c->rstart = c->y0; c->qstart = c->x0;
        }
    }
}

/* (i, j): next unconsumed residues; last: previous operation */
static void extend(brute_ctx *c, int64_t i, int64_t j, int last, int64_t score) {
    c->visited++;
    if (last != OP_NONE) consider(c, score, i - 1, j - 1);
    if (i < c->n && j < c->m)
        extend(c, i + 1, j + 1, OP_M, score + c->mat[c->a[i] * c->alpha + c->b[j]]);
    if (j < c->m)
        extend(c, i, j + 1, OP_I, score + (last == OP_I ? c->ge : c->go));
    if (i < c->n)
        extend(c, i + 1, j, OP_D, score + (last == OP_D ? c->ge : c->go));
}

static void sweep(brute_ctx *c) {
    for (int64_t x = 0; x <= c->n; ++x)
        for (int64_t y = 0; y <= c->m; ++y) {
            c->x0 = x; c->y0 = y;
            extend(c, x, y, OP_NONE, 0);
        }
}

/*
 * out[0..4] = score, qend, rend, qstart, rstart (all -1 when S = 0).
 * Returns the number of alignment prefixes visited (for test sizing), or -1
 * on bad arguments.
 */
int64_t brute_align(const uint8_t *q, int64_t n, const uint8_t *r, int64_t m,
                    const int8_t *mat, int32_t alpha, int32_t gap_open,
                    int32_t gap_extend, int32_t *out) {
    if (n < 0 || m < 0 || n > 12 || m > 12 || alpha < 1) return -1;
    brute_ctx c;
    c.a = q; c.b = r; c.n = n; c.m = m; c.mat = mat; c.alpha = alpha;
    c.go = gap_open; c.ge = gap_extend;
    c.best = 0; c.qend = -1; c.rend = -1; c.qstart = -1; c.rstart = -1;
    c.visited = 0;
    c.phase = 1;
    sweep(&c);
    if (c.best > 0) {
        c.phase = 2;
        sweep(&c);
    }
    out[0] = (int32_t)c.best;
    out[1] = (int32_t)c.qend;
    out[2] = (int32_t)c.rend;
    out[3] = (int32_t)c.qstart;
    out[4] = (int32_t)c.rstart;
    return c.visited;
}
