"""Pins for the traceback oracle (oracle/sw_cigar.c), CPU only.

The CIGAR of a located local alignment is checked against things the
oracle's own recurrence does not produce: hand-worked alignments, an
independent scorer of the op string (substitution scores plus go + (k-1) ge
per maximal gap run), the lengths the ops consume, and brute-force
enumeration of every global alignment of tiny substrings.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as wl


def _enc(s, alphabet="ACGT"):
    return np.array([alphabet.index(c) for c in s], dtype=np.uint8)


def _runs(ops):
    return [(int(o) & 15, int(o) >> 4) for o in ops]


def score_ops(q, r, mat, go, ge, res, ops):
    """Independent scorer: walk the op string over the located substrings."""
    i, j = res[3], res[4]
    total = 0
    for code, k in _runs(ops):
        if code == 0:
            for _ in range(k):
                total += int(mat[q[i], r[j]])
                i += 1
                j += 1
        elif code == 1:
            total += go + (k - 1) * ge
            i += k
        else:
            total += go + (k - 1) * ge
            j += k
    return total, i, j


def test_fig2_example():
    # Fig. 2 scoring (+2/-2, gap -1): ATGCT / A-GCT, one query residue unmatched
    mat = wl.dna_matrix(2, -2)
    q, r = _enc("ATGCT"), _enc("AGCT")
    res = oracle.align(q, r, mat, -1, -1)
    assert res == (7, 4, 3, 0, 0)
    ops, g = oracle.cigar(q, r, mat, -1, -1, res)
    assert g == 7
    assert oracle.cigar_string(ops) == "1M1I3M"


def test_gap_placement_rule():
    # ACGT-ACGT / ACGTTACGT and ACG-TACGT / ACGTTACGT score 18 alike; the
    # walk back prefers M, so the deletion lands at the first of the two T's
    mat = wl.dna_matrix(3, -3)
    q, r = _enc("ACGTACGT"), _enc("ACGTTACGT")
    res = oracle.align(q, r, mat, -6, -1)
    assert res == (18, 7, 8, 0, 0)
    ops, g = oracle.cigar(q, r, mat, -6, -1, res)
    assert g == 18
    assert oracle.cigar_string(ops) == "3M1D5M"


def test_no_alignment_gives_no_ops():
    mat = wl.dna_matrix(3, -3)
    res = oracle.align(_enc("AAAA"), _enc("CCCC"), mat, -6, -1)
    assert res[0] == 0
    ops, g = oracle.cigar(_enc("AAAA"), _enc("CCCC"), mat, -6, -1, res)
    assert ops == [] and g == 0


@pytest.mark.parametrize("go,ge", [(-6, -1), (-1, -1), (0, 0), (-11, -1), (-3, -2)])
def test_random_pairs_score_and_span(go, ge):
    rng = np.random.default_rng(1000 + 13 * abs(go) + abs(ge))
    for kind in ("dna", "protein"):
        if kind == "dna":
            mat, A = wl.dna_matrix(3, -3), 4
        else:
            mat, A = wl.load_blosum62()[0].astype(np.int8), 20
        for _ in range(60):
            q = rng.integers(0, A, int(rng.integers(1, 60))).astype(np.uint8)
            r = rng.integers(0, A, int(rng.integers(1, 80))).astype(np.uint8)
            if rng.random() < 0.5 and len(r) > len(q):  # plant a copy
                at = int(rng.integers(0, len(r) - len(q) + 1))
                r[at:at + len(q)] = q
            res = oracle.align(q, r, mat, go, ge)
            ops, g = oracle.cigar(q, r, mat, go, ge, res)
            if res[0] == 0:
                assert ops == []
                continue
            assert g == res[0]
            total, i, j = score_ops(q, r, mat, go, ge, res, ops)
            assert total == res[0]
            assert (i, j) == (res[1] + 1, res[2] + 1)
            # runs are maximal: no two neighbours share an op
            codes = [c for c, _ in _runs(ops)]
            assert all(a != b for a, b in zip(codes, codes[1:]))


def _global_best(qa, rb, mat, go, ge):
    """Brute force: best score over every global alignment of qa, rb (op
    strings over M, I, D), scored with maximal runs."""
    n, m = len(qa), len(rb)
    best = None
    best_ops = []
    for nM in range(0, min(n, m) + 1):
        nI, nD = n - nM, m - nM
        for perm in set(itertools.permutations("M" * nM + "I" * nI + "D" * nD)):
            i = j = 0
            tot = 0
            prev = None
            for op in perm:
                if op == "M":
                    tot += int(mat[qa[i], rb[j]])
                    i += 1
                    j += 1
                elif op == "I":
                    tot += ge if prev == "I" else go
                    i += 1
                else:
                    tot += ge if prev == "D" else go
                    j += 1
                prev = op
            if best is None or tot > best:
                best, best_ops = tot, [perm]
            elif tot == best:
                best_ops.append(perm)
    return best, best_ops


def test_brute_force_tiny_spans():
    rng = np.random.default_rng(99)
    mat = wl.dna_matrix(3, -3)
    checked = 0
    for go, ge in ((-6, -1), (-2, -2), (-4, -1)):
        for _ in range(150):
            q = rng.integers(0, 4, int(rng.integers(1, 7))).astype(np.uint8)
            r = rng.integers(0, 4, int(rng.integers(1, 7))).astype(np.uint8)
            res = oracle.align(q, r, mat, go, ge)
            if res[0] == 0:
                continue
            qa, rb = q[res[3]:res[1] + 1], r[res[4]:res[2] + 1]
            if len(qa) + len(rb) > 9:
                continue
            best, opts = _global_best(qa, rb, mat, go, ge)
            assert best == res[0]
            ops, _ = oracle.cigar(q, r, mat, go, ge, res)
            text = "".join(("MID"[c]) * k for c, k in _runs(ops))
            assert tuple(text) in set(opts)
            checked += 1
    assert checked > 100


def test_batch_equals_single():
    b = wl.gen_config(0, n_pairs=120)
    res = oracle.align_workload(b)
    ops, off, n_ops = oracle.cigar_workload(b, res, threads=4)
    for p in range(b.n_pairs):
        q, r = b.pair(p)
        single, _ = oracle.cigar(q, r, b.matrix, b.gap_open, b.gap_extend, res[p])
        assert list(ops[off[p]:off[p] + n_ops[p]]) == single


# ---- the pins above catch plausible mistakes in the traceback oracle

import ctypes  # noqa: E402
import os  # noqa: E402
import subprocess  # noqa: E402

CIGAR_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                         "sw_cigar.c")

CIGAR_MUTANTS = {
    "gap_in_query_coded_as_D": ("if ((rc = push_op(rev, &nr, (int)(N + M), OP_I)) != OC_OK)",
                                "if ((rc = push_op(rev, &nr, (int)(N + M), OP_D)) != OC_OK)"),
    "open_test_inverted": ("            --j;\n            if (open) state = 0;",
                           "            --j;\n            if (!open) state = 0;"),
    "H_prefers_gap_over_M": ("if (i > 0 && j > 0) {\n                const int x",
                             "if (i > 0 && j > 0 && H[c] != E[c]) {\n                const int x"),
    "extend_charged_open": ("E[c] = max2(E[c - 1] + ge, H[c - 1] + go);",
                            "E[c] = max2(E[c - 1] + go, H[c - 1] + go);"),
    "diagonal_from_up": ("H[c] = max2(H[c - W - 1] + mat[x * A + y]",
                         "H[c] = max2(H[c - W] + mat[x * A + y]"),
    "transposed_lookup": ("H[c] = max2(H[c - W - 1] + mat[x * A + y]",
                          "H[c] = max2(H[c - W - 1] + mat[y * A + x]"),
}


def _compile_cigar(tmp_path, name, text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", str(c), "-o",
                    str(so)], check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    u8p, i8p, i32p = (ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int8),
                      ctypes.POINTER(ctypes.c_int32))
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_cigar.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i8p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32, i32p, u32p, ctypes.c_int32, i32p,
                                 ctypes.POINTER(ctypes.c_int64)]
    lib.oracle_cigar.restype = ctypes.c_int

    def cig(q, r, mat, go, ge, res):
        q = np.ascontiguousarray(q, np.uint8)
        r = np.ascontiguousarray(r, np.uint8)
        mat = np.ascontiguousarray(mat, np.int8)
        rr = np.ascontiguousarray(res, np.int32)
        cap = len(q) + len(r)
        ops = np.zeros(cap, np.uint32)
        n = ctypes.c_int32()
        g = ctypes.c_int64()
        rc = lib.oracle_cigar(q.ctypes.data_as(u8p), len(q), r.ctypes.data_as(u8p), len(r),
                              mat.ctypes.data_as(i8p), mat.shape[0], go, ge,
                              rr.ctypes.data_as(i32p), ops.ctypes.data_as(u32p), cap,
                              ctypes.byref(n), ctypes.byref(g))
        return rc, [int(x) for x in ops[:n.value]], int(g.value)

    return cig


def cigar_battery(cig) -> list[str]:
    fails = []
    m2, m3 = wl.dna_matrix(2, -2), wl.dna_matrix(3, -3)
    for name, q, r, mat, go, ge, want in (("fig2", "ATGCT", "AGCT", m2, -1, -1, "1M1I3M"),
                                          ("gap_rule", "ACGTACGT", "ACGTTACGT", m3, -6, -1,
                                           "3M1D5M")):
        res = oracle.align(_enc(q), _enc(r), mat, go, ge)
        rc, ops, _ = cig(_enc(q), _enc(r), mat, go, ge, res)
        if rc != 0 or oracle.cigar_string(ops) != want:
            fails.append(name)
    rng = np.random.default_rng(5)
    asym = rng.integers(-4, 3, size=(4, 4)).astype(np.int8)
    np.fill_diagonal(asym, 4)
    for mat, go, ge in ((m3, -6, -1), (m3, -3, -2), (asym, -5, -1)):
        for _ in range(80):
            q = rng.integers(0, 4, int(rng.integers(1, 40))).astype(np.uint8)
            r = rng.integers(0, 4, int(rng.integers(1, 50))).astype(np.uint8)
            res = oracle.align(q, r, mat, go, ge)
            if res[0] == 0:
                continue
            rc, ops, g = cig(q, r, mat, go, ge, res)
            if rc != 0:
                fails.append("rc")
                return fails
            try:
                total, i, j = score_ops(q, r, mat, go, ge, res, ops)
            except IndexError:  # the ops run past the located span
                total, i, j = None, -1, -1
            if g != res[0] or total != res[0] or (i, j) != (res[1] + 1, res[2] + 1):
                fails.append("score_span")
                return fails
    return fails


def test_cigar_pins_catch_mutants(tmp_path):
    src = open(CIGAR_SRC).read()
    assert cigar_battery(_compile_cigar(tmp_path, "orig", src)) == []
    for name, (a, b) in CIGAR_MUTANTS.items():
        assert src.count(a) == 1, name
        fails = cigar_battery(_compile_cigar(tmp_path, name, src.replace(a, b)))
        assert fails, f"mutant {name} passed every pin"
