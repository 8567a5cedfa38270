/*
 * Second, independent oracle: one forward pass that carries each cell's
 * start position instead of running a reverse pass.  TEST INFRASTRUCTURE
 * ONLY; it cross-checks the start coordinates of sw_oracle.c on pairs too
 * long for brute-force enumeration.
 *
 * Same recurrence as Section II-B.1 / Fig. 8 (see sw_oracle.c), but every
 * H, E, F entry is a triple (score, rstart, qstart) compared
 * lexicographically: larger score, then larger rstart, then larger qstart.
 * The zero floor at DP cell (i, j) (1-based; a_1..a_i and b_1..b_j consumed)
 * is the empty alignment whose next residues are a_{i+1} and b_{j+1}, i.e.
 * start (qstart, rstart) = (i, j) in 0-based coordinates.  Moves inherit the
 * start of the entry they extend.  Because ties are broken toward the larger
 * start at every cell, the entry at the chosen end cell holds, among the
 * score-S alignments ending there, the largest rstart and then the largest
 * qstart: the start rule of the reverse-pass oracle.
 */
#include <stdint.h>
#include <stdlib.h>

#define T_NEG_INF (INT64_MIN / 4)

typedef struct {
    int64_t s, y, x;   /* score, rstart, qstart */
} cell;

static cell better(cell p, cell q) {
    if (p.s != q.s) return p.s > q.s ? p : q;
    if (p.y != q.y) return p.y > q.y ? p : q;
    return p.x >= q.x ? p : q;
}

static cell plus(cell p, int64_t d) {
    cell r = p;
    r.s = p.s + d;
    return r;
}

/* out[0..4] = score, qend, rend, qstart, rstart.  Returns 0, or -1/-3. */
int track_align(const uint8_t *q, int64_t n, const uint8_t *r, int64_t m,
                const int8_t *mat, int32_t alpha, int32_t gap_open,
                int32_t gap_extend, int32_t *out) {
    if (n < 0 || m < 0 || alpha < 1) return -1;
    out[0] = 0; out[1] = out[2] = out[3] = out[4] = -1;
    if (n == 0 || m == 0) return 0;
    cell *hp = (cell *)malloc(sizeof(cell) * (size_t)(m + 1));
    cell *hc = (cell *)malloc(sizeof(cell) * (size_t)(m + 1));
    cell *f = (cell *)malloc(sizeof(cell) * (size_t)(m + 1));
    if (!hp || !hc || !f) { free(hp); free(hc); free(f); return -3; }
    for (int64_t j = 0; j <= m; ++j) {
        hp[j].s = 0; hp[j].y = j; hp[j].x = 0;      /* empty alignment at (0, j) */
        f[j].s = T_NEG_INF; f[j].y = -1; f[j].x = -1;
    }
    int64_t best = 0, bi = -1, bj = -1;
    cell bstart = {0, -1, -1};
    for (int64_t i = 1; i <= n; ++i) {
        hc[0].s = 0; hc[0].y = 0; hc[0].x = i;
        cell e = {T_NEG_INF, -1, -1};
        for (int64_t j = 1; j <= m; ++j) {
            e = better(plus(hc[j - 1], gap_open), plus(e, gap_extend));
            f[j] = better(plus(hp[j], gap_open), plus(f[j], gap_extend));
            cell floor0 = {0, j, i};
            cell h = plus(hp[j - 1], mat[q[i - 1] * alpha + r[j - 1]]);
            h = better(h, e);
            h = better(h, f[j]);
            h = better(h, floor0);
            hc[j] = h;
            if (h.s > best || (h.s == best && h.s > 0 &&
                               (j - 1 < bj || (j - 1 == bj && i - 1 < bi)))) {
                best = h.s; bi = i - 1; bj = j - 1; bstart = h;
            }
        }
        cell *t = hp; hp = hc; hc = t;
    }
    free(hp); free(hc); free(f);
    if (best > 0) {
        out[0] = (int32_t)best; out[1] = (int32_t)bi; out[2] = (int32_t)bj;
        out[3] = (int32_t)bstart.x; out[4] = (int32_t)bstart.y;
    }
    return 0;
}
