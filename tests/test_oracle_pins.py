"""Pins of the CPU oracle to things other than itself.

The oracle (oracle/sw_oracle.c) is checked against
  * hand-worked examples (tests/golden/hand_examples.txt), including the two
    sequences of the paper's Fig. 2 with the scores of Section II-B.1;
  * brute-force enumeration of every local alignment (oracle/sw_brute.c),
    exhaustively on short pairs and at random up to 8 residues;
  * an independent forward pass that carries start positions
    (oracle/sw_track.c) on longer pairs;
  * closed forms and invariants: S >= 0, S <= smax * min(n, m), self-alignment
    scores, swap symmetry, monotonicity under appending residues, the global
    (end-to-end) affine score of the reported span equals S, and the go == ge
    special case equals textbook linear-gap Smith-Waterman.
The global-score and linear-gap checks use plain Python written here from the
textbook recurrences, not the oracle's code.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
DNA = {c: i for i, c in enumerate("ACGT")}


def enc(s):
    return np.array([DNA[c] for c in s], dtype=np.uint8)


def pm_matrix(match, mismatch, a=4):
    m = np.full((a, a), mismatch, dtype=np.int8)
    np.fill_diagonal(m, match)
    return m


SCORINGS = {"pm2": pm_matrix(2, -2), "dna3": pm_matrix(3, -3)}


def load_golden():
    rows = []
    with open(os.path.join(HERE, "golden", "hand_examples.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows.append((p[0], p[1], int(p[2]), int(p[3]), p[4], p[5], tuple(int(v) for v in p[6:11])))
    return rows


GOLDEN = load_golden()


@pytest.mark.parametrize("row", GOLDEN, ids=[r[0] for r in GOLDEN])
def test_hand_examples(row):
    name, sc, go, ge, q, r, expect = row
    mat = SCORINGS[sc]
    assert oracle.align(enc(q), enc(r), mat, go, ge) == expect
    assert oracle.track(enc(q), enc(r), mat, go, ge) == expect
    assert oracle.brute(enc(q), enc(r), mat, go, ge) == expect


GAPS = [(-6, -1), (-1, -1), (-2, -2), (-3, 0), (-1, 0), (0, 0), (-5, -2)]


def test_brute_exhaustive_short_dna():
    """Every DNA pair with lengths 1..3 under +3/-3 and two gap settings."""
    mat = SCORINGS["dna3"]
    seqs = [np.array(s, np.uint8) for L in (1, 2, 3) for s in itertools.product(range(4), repeat=L)]
    n = 0
    for go, ge in [(-6, -1), (-1, -1)]:
        for q in seqs:
            for r in seqs:
                b = oracle.brute(q, r, mat, go, ge)
                assert oracle.align(q, r, mat, go, ge) == b, (q, r, go, ge)
                n += 1
    assert n == 2 * len(seqs) ** 2


def test_brute_exhaustive_binary_ties():
    """All pairs of length 4 over a two-letter alphabet: ties everywhere."""
    mat = pm_matrix(2, -2, a=2)
    seqs = [np.array(s, np.uint8) for s in itertools.product(range(2), repeat=4)]
    for go, ge in [(-1, -1), (-3, -1), (0, 0), (-2, 0)]:
        for q in seqs:
            for r in seqs:
                assert oracle.align(q, r, mat, go, ge) == oracle.brute(q, r, mat, go, ge), (q, r, go, ge)


@pytest.mark.parametrize("go,ge", GAPS)
def test_brute_random_dna(go, ge):
    rng = np.random.default_rng(1000 + 17 * go - ge)
    mat = SCORINGS["dna3"] if go != -1 else SCORINGS["pm2"]
    for _ in range(60):
        n, m = rng.integers(1, 8, size=2)
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        if rng.random() < 0.5:  # share a segment so gaps and long matches occur
            k = min(n, m) // 2
            r[:k] = q[n - k:]
        assert oracle.align(q, r, mat, go, ge) == oracle.brute(q, r, mat, go, ge), (q, r)


def test_brute_random_protein():
    s, _ = wl.load_blosum62()
    mat = s.astype(np.int8)
    rng = np.random.default_rng(7)
    for _ in range(80):
        n, m = rng.integers(1, 7, size=2)
        q = rng.integers(0, 20, n).astype(np.uint8)
        r = rng.integers(0, 20, m).astype(np.uint8)
        if rng.random() < 0.5:
            r[: min(n, m)] = q[: min(n, m)]
        for go, ge in [(-11, -1), (-2, -1)]:
            assert oracle.align(q, r, mat, go, ge) == oracle.brute(q, r, mat, go, ge), (q, r, go, ge)


def test_brute_random_asymmetric_matrix():
    """A non-symmetric matrix catches a transposed lookup s(b, a)."""
    rng = np.random.default_rng(11)
    for _ in range(120):
        mat = rng.integers(-4, 5, size=(3, 3)).astype(np.int8)
        n, m = rng.integers(1, 7, size=2)
        q = rng.integers(0, 3, n).astype(np.uint8)
        r = rng.integers(0, 3, m).astype(np.uint8)
        assert oracle.align(q, r, mat, -3, -1) == oracle.brute(q, r, mat, -3, -1), (mat, q, r)


def test_track_agrees_on_longer_pairs():
    """Forward start-tracking and the reverse pass pick the same start."""
    rng = np.random.default_rng(3)
    mat = SCORINGS["dna3"]
    s, _ = wl.load_blosum62()
    for t in range(3000):
        n, m = rng.integers(1, 200, size=2)
        if t % 3 == 2:
            A, M, go, ge = 20, s.astype(np.int8), -11, -1
        else:
            A, M = 4, mat
            go, ge = [(-6, -1), (-1, -1), (-2, 0)][(t // 3) % 3]
        q = rng.integers(0, A, n).astype(np.uint8)
        r = rng.integers(0, A, m).astype(np.uint8)
        if rng.random() < 0.4:
            k = min(n, m)
            off = rng.integers(0, m - k + 1)
            r[off:off + k] = q[:k]
        assert oracle.align(q, r, M, go, ge) == oracle.track(q, r, M, go, ge), (t, n, m)


def test_track_agrees_on_workload_sample():
    b = wl.gen_config(0, n_pairs=200)
    out = oracle.align_workload(b)
    for i in range(b.n_pairs):
        q, r = b.pair(i)
        assert tuple(out[i]) == oracle.track(q, r, b.matrix, b.gap_open, b.gap_extend)


# ------------------------------------------------------------- closed forms


def global_affine(q, r, mat, go, ge):
    """End-to-end (Needleman-Wunsch/Gotoh) score; plain Python, textbook."""
    n, m = len(q), len(r)
    NEG = -10 ** 9
    H = [[NEG] * (m + 1) for _ in range(n + 1)]
    E = [[NEG] * (m + 1) for _ in range(n + 1)]
    F = [[NEG] * (m + 1) for _ in range(n + 1)]
    H[0][0] = 0
    for j in range(1, m + 1):
        E[0][j] = go + (j - 1) * ge
        H[0][j] = E[0][j]
    for i in range(1, n + 1):
        F[i][0] = go + (i - 1) * ge
        H[i][0] = F[i][0]
        for j in range(1, m + 1):
            E[i][j] = max(H[i][j - 1] + go, E[i][j - 1] + ge)
            F[i][j] = max(H[i - 1][j] + go, F[i - 1][j] + ge)
            H[i][j] = max(H[i - 1][j - 1] + int(mat[q[i - 1], r[j - 1]]), E[i][j], F[i][j])
    return H[n][m]


def linear_sw_score(q, r, mat, g):
    """Textbook Smith-Waterman with a linear gap penalty g (Smith & Waterman 1981)."""
    n, m = len(q), len(r)
    prev = [0] * (m + 1)
    best = 0
    for i in range(1, n + 1):
        cur = [0] * (m + 1)
        for j in range(1, m + 1):
            cur[j] = max(0, prev[j - 1] + int(mat[q[i - 1], r[j - 1]]), prev[j] + g, cur[j - 1] + g)
            best = max(best, cur[j])
        prev = cur
    return best


def test_reported_span_global_score_equals_S():
    rng = np.random.default_rng(5)
    s, _ = wl.load_blosum62()
    for t in range(150):
        if t % 2:
            A, M, go, ge = 4, SCORINGS["dna3"], -6, -1
        else:
            A, M, go, ge = 20, s.astype(np.int8), -11, -1
        n, m = rng.integers(5, 60, size=2)
        q = rng.integers(0, A, n).astype(np.uint8)
        r = rng.integers(0, A, m).astype(np.uint8)
        if t % 3 == 0:
            k = min(n, m) // 2
            r[:k] = q[-k:]
        S, qe, re_, qs, rs = oracle.align(q, r, M, go, ge)
        if S == 0:
            continue
        assert 0 <= qs <= qe < n and 0 <= rs <= re_ < m
        assert global_affine(q[qs:qe + 1], r[rs:re_ + 1], M, go, ge) == S


def test_linear_gap_special_case():
    rng = np.random.default_rng(9)
    for t in range(150):
        g = -int(rng.integers(1, 4))
        M = SCORINGS["pm2"] if t % 2 else SCORINGS["dna3"]
        n, m = rng.integers(1, 50, size=2)
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        assert oracle.align(q, r, M, g, g)[0] == linear_sw_score(q, r, M, g)


def test_bounds_and_self_alignment():
    rng = np.random.default_rng(13)
    s, _ = wl.load_blosum62()
    M = SCORINGS["dna3"]
    for L in [1, 2, 7, 31, 32, 33, 100, 257]:
        q = rng.integers(0, 4, L).astype(np.uint8)
        assert oracle.align(q, q, M, -6, -1) == (3 * L, L - 1, L - 1, 0, 0)
        p = rng.integers(0, 20, L).astype(np.uint8)
        diag = int(np.sum(np.diag(s)[p]))
        assert oracle.align(p, p, s.astype(np.int8), -11, -1) == (diag, L - 1, L - 1, 0, 0)
    for _ in range(200):
        n, m = rng.integers(0, 80, size=2)
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        S = oracle.align(q, r, M, -6, -1)[0]
        assert 0 <= S <= 3 * min(n, m)


def test_swap_symmetry_and_monotonicity():
    rng = np.random.default_rng(17)
    s, _ = wl.load_blosum62()
    for t in range(200):
        A, M, go, ge = (4, SCORINGS["dna3"], -6, -1) if t % 2 else (20, s.astype(np.int8), -11, -1)
        n, m = rng.integers(1, 60, size=2)
        q = rng.integers(0, A, n).astype(np.uint8)
        r = rng.integers(0, A, m).astype(np.uint8)
        a = oracle.align(q, r, M, go, ge)
        b = oracle.align(r, q, M, go, ge)
        assert a[0] == b[0]
        extra = rng.integers(0, A, rng.integers(1, 10)).astype(np.uint8)
        assert oracle.align(np.concatenate([q, extra]), r, M, go, ge)[0] >= a[0]
        assert oracle.align(q, np.concatenate([extra, r]), M, go, ge)[0] >= a[0]


def test_unmutated_plant_scores_full_length():
    rng = np.random.default_rng(19)
    M = SCORINGS["dna3"]
    for _ in range(50):
        n = int(rng.integers(20, 150))
        m = n + int(rng.integers(0, 300))
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        off = int(rng.integers(0, m - n + 1))
        r[off:off + n] = q
        S, qe, re_, qs, rs = oracle.align(q, r, M, -6, -1)
        assert S >= 3 * n


def test_empty_inputs():
    M = SCORINGS["dna3"]
    e = np.zeros(0, np.uint8)
    q = enc("ACGT")
    assert oracle.align(e, q, M, -6, -1) == (0, -1, -1, -1, -1)
    assert oracle.align(q, e, M, -6, -1) == (0, -1, -1, -1, -1)
    assert oracle.align(e, e, M, -6, -1) == (0, -1, -1, -1, -1)


def test_invalid_inputs_rejected():
    M = SCORINGS["dna3"]
    with pytest.raises(oracle.OracleError):
        oracle.align(np.array([4], np.uint8), enc("A"), M, -6, -1)
    with pytest.raises(oracle.OracleError):
        oracle.align(enc("A"), enc("A"), M, 1, -1)
    # opening cheaper than extending is outside the recurrence's validity
    with pytest.raises(oracle.OracleError):
        oracle.align(enc("A"), enc("A"), M, 0, -1)
