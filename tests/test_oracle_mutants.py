"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a wrong index, a
transposed operand, a reversed tie-break) in a temporary copy of
oracle/sw_oracle.c, compiles it with gcc, and checks that the pin battery
below (hand examples, brute-force enumeration, closed forms) rejects it.  The
unmodified source must pass the same battery.  Everything runs on the CPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "sw_oracle.c")

MUTANTS = {
    "drop_zero_floor": ("h = max2(h, 0);", ""),
    "drop_E_term": ("h = max2(h, e);", ""),
    "drop_F_term": ("h = max2(h, f[j]);", ""),
    "swap_open_extend_E": ("e = max2(h_cur[j - 1] + go, e + ge);", "e = max2(h_cur[j - 1] + ge, e + go);"),
    "swap_open_extend_F": ("f[j] = max2(h_prev[j] + go, f[j] + ge);", "f[j] = max2(h_prev[j] + ge, f[j] + go);"),
    "F_from_diagonal": ("f[j] = max2(h_prev[j] + go,", "f[j] = max2(h_prev[j - 1] + go,"),
    "diag_from_up": ("int64_t h = h_prev[j - 1] +", "int64_t h = h_prev[j] +"),
    "transposed_lookup": ("mat[ai * alpha + bj_res]", "mat[bj_res * alpha + ai]"),
    "end_prefers_large_rend": ("(j - 1 < *bj ||", "(j - 1 > *bj ||"),
    "end_prefers_large_qend": ("i - 1 < *bi)", "i - 1 > *bi)"),
    "end_first_seen_only": ("(h == *best && h > 0 &&", "(0 && h > 0 &&"),
    "qstart_not_reflected": ("out[3] = (int32_t)(qe - k);", "out[3] = (int32_t)(k);"),
    "rstart_off_by_one": ("out[4] = (int32_t)(re - l);", "out[4] = (int32_t)(re - l + 1);"),
    "reverse_skips_last_residue": ("rc = forward_pass(q + qe, -1, qe + 1, r + re, -1, re + 1,",
                                   "rc = forward_pass(q + qe, -1, qe, r + re, -1, re + 1,"),
}


def _compile(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-pthread", str(c), "-o", str(so)],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    u8p, i8p, i32p = (ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int8),
                      ctypes.POINTER(ctypes.c_int32))
    lib.oracle_align.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, i8p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32, i32p]
    lib.oracle_align.restype = ctypes.c_int

    def align(q, r, mat, go, ge):
        q = np.ascontiguousarray(q, np.uint8)
        r = np.ascontiguousarray(r, np.uint8)
        mat = np.ascontiguousarray(mat, np.int8)
        out = np.zeros(5, np.int32)
        rc = lib.oracle_align(q.ctypes.data_as(u8p), len(q), r.ctypes.data_as(u8p), len(r),
                              mat.ctypes.data_as(i8p), mat.shape[0], go, ge, out.ctypes.data_as(i32p))
        return rc, tuple(int(v) for v in out)

    return align


def pin_battery(align) -> list[str]:
    """Return the names of the pins the given oracle function fails."""
    failures = []
    dna = {c: i for i, c in enumerate("ACGT")}
    enc = lambda s: np.array([dna[c] for c in s], np.uint8)  # noqa: E731
    pm2 = np.full((4, 4), -2, np.int8); np.fill_diagonal(pm2, 2)
    dna3 = wl.dna_matrix()
    mats = {"pm2": pm2, "dna3": dna3}
    with open(os.path.join(HERE, "golden", "hand_examples.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rc, got = align(enc(p[4]), enc(p[5]), mats[p[1]], int(p[2]), int(p[3]))
            if rc != 0 or got != tuple(int(v) for v in p[6:11]):
                failures.append(f"golden:{p[0]}")
    rng = np.random.default_rng(2024)
    for t in range(150):
        if t % 3 == 0:
            mat = rng.integers(-4, 5, size=(3, 3)).astype(np.int8)
            A, go, ge = 3, -3, -1
        else:
            mat, A = dna3, 4
            go, ge = [(-6, -1), (-2, -2), (-3, 0)][t % 3]
        n, m = rng.integers(1, 7, size=2)
        q = rng.integers(0, A, n).astype(np.uint8)
        r = rng.integers(0, A, m).astype(np.uint8)
        if t % 2:
            k = min(n, m) // 2
            r[:k] = q[n - k:]
        rc, got = align(q, r, mat, go, ge)
        if rc != 0 or got != oracle.brute(q, r, mat, go, ge):
            failures.append("brute")
            break
    for L in (1, 5, 40):
        q = rng.integers(0, 4, L).astype(np.uint8)
        rc, got = align(q, q, dna3, -6, -1)
        if rc != 0 or got != (3 * L, L - 1, L - 1, 0, 0):
            failures.append(f"self:{L}")
    return failures


def test_unmodified_oracle_passes_battery(tmp_path):
    align = _compile(tmp_path, "clean", open(SRC).read())
    assert pin_battery(align) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    align = _compile(tmp_path, name, text.replace(old, new))
    assert pin_battery(align), f"mutant {name} passed every pin"


def test_gap_boundary_value_is_irrelevant(tmp_path):
    """E[i][0] and F[0][j] set to 0 instead of -infinity change no output.

    With H >= 0 and go <= ge <= 0, a gap state seeded from a boundary value
    <= 0 stays <= 0 and never wins the maximum against the zero floor; the
    kernels rely on this to use a finite sentinel.
    """
    text = open(SRC).read()
    for old in ("int64_t e = NEG_INF;    /* E[i][0] = -inf */", "f[j] = NEG_INF;         /* F[0][j] = -inf */"):
        assert text.count(old) == 1
    text = text.replace("int64_t e = NEG_INF;    /* E[i][0] = -inf */", "int64_t e = 0;")
    text = text.replace("f[j] = NEG_INF;         /* F[0][j] = -inf */", "f[j] = 0;")
    align = _compile(tmp_path, "zero_boundary", text)
    rng = np.random.default_rng(77)
    s, _ = wl.load_blosum62()
    for t in range(300):
        A, M, go, ge = (4, wl.dna_matrix(), -6, -1) if t % 2 else (20, s.astype(np.int8), -11, -1)
        n, m = rng.integers(0, 40, size=2)
        q = rng.integers(0, A, n).astype(np.uint8)
        r = rng.integers(0, A, m).astype(np.uint8)
        rc, got = align(q, r, M, go, ge)
        assert rc == 0 and got == oracle.align(q, r, M, go, ge)
