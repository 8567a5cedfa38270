"""GPU parity of the packed 16-bit form of the batched kernel.

The packed form holds two DP cells per 32-bit word (scores scaled by 8, the
end cell tracked per column with a 3-bit row code).  It must give the same
five outputs as the scaled int32 form and the oracle, bit for bit, wherever
the plan takes it; these tests run both forms on the same batches (the int32
one with SW_PLAN_NO_S16X2) and check which form each plan took.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

from test_gpu_parity import EDGE, TUNINGS, assert_same, edge_batch, run_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


def both_forms(gpu_lib, ctx, b, expect, name, tuning=None, want_packed=True):
    got, info = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_BATCHED, tuning=tuning)
    assert info["arith"] == ("s16x2" if want_packed else "s32"), (name, info)
    assert_same(got, expect, f"{name} ({info['arith']})")
    got32, info32 = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_BATCHED,
                            flags=gpu_lib.SW_PLAN_NO_S16X2, tuning=tuning)
    assert info32["arith"] == "s32"
    assert_same(got32, expect, f"{name} (s32)")


def test_form_selection(gpu_lib, ctx):
    """DNA workloads fit the packed bound (32-bit profile words, scale 8);
    protein pairs take the byte profile (scale 4: 4 (11 x 400 + 22) <= 32767,
    s - go <= 22 < 32); a gap_open of -40 (s - go up to 51) or a mismatch
    below gap_open keeps the int32 form."""
    b0 = wl.gen_config(0, n_pairs=50)
    _, info = run_lib(gpu_lib, ctx, b0)
    assert info["arith"] == "s16x2"
    _, info = run_lib(gpu_lib, ctx, b0, flags=gpu_lib.SW_PLAN_NO_S16X2)
    assert info["arith"] == "s32"
    b2 = wl.gen_config(2).slice(0, 2000)
    _, info = run_lib(gpu_lib, ctx, b2)
    assert info["arith"] == "s16x2"
    b2w = wl.make_batch("protein-go40", [b2.pair(i)[0] for i in range(200)],
                        [b2.pair(i)[1] for i in range(200)], b2.matrix, -40, -1)
    got, info = run_lib(gpu_lib, ctx, b2w)
    assert info["arith"] == "s32"
    assert_same(got, oracle.align_workload(b2w), "protein go -40")
    fig2 = wl.make_batch("fig2", [b0.pair(i)[0] for i in range(b0.n_pairs)],
                         [b0.pair(i)[1] for i in range(b0.n_pairs)], wl.dna_matrix(2, -2), -1, -1)
    _, info = run_lib(gpu_lib, ctx, fig2)
    assert info["arith"] == "s32"  # s - go = -1 < 0


@pytest.mark.parametrize("tuning", TUNINGS, ids=[f"G{1 << t[0] if t[0] >= 0 else 'auto'}-cap{t[1]:g}"
                                                 for t in TUNINGS])
def test_edge_lengths_both_forms(gpu_lib, ctx, tuning):
    """Lengths around every tile edge under every lane-group width, both forms."""
    b = edge_batch("dna", 70 + max(tuning[0], 0), EDGE, EDGE[1::3])
    both_forms(gpu_lib, ctx, b, oracle.align_workload(b), f"edge tuning={tuning}", tuning)


def _periodic(unit, n):
    return np.resize(np.array(unit, np.uint8), n)


def test_tie_heavy_inputs(gpu_lib, ctx):
    """Periodic and constant sequences: many cells share the best score, so
    the end rule (smallest rend, then qend) and the start rule (largest
    rstart, then qstart) decide among many candidates in both sweeps."""
    rng = np.random.default_rng(101)
    qs, rs = [], []
    units = [[0], [0, 1], [0, 1, 2], [0, 0, 1], [2, 3, 2, 3, 1]]
    for n in (1, 7, 8, 9, 16, 17, 40, 64, 65, 130, 300):
        for m in (1, 8, 15, 33, 64, 200, 513):
            uq = units[int(rng.integers(len(units)))]
            ur = units[int(rng.integers(len(units)))]
            qs.append(_periodic(uq, n))
            rs.append(_periodic(ur, m))
    b = wl.make_batch("ties", qs, rs, wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(b)
    for tuning in ((1, 1e9), (2, 1e9), (4, 1e9), (5, 1e9), (-1, 0.5)):
        both_forms(gpu_lib, ctx, b, expect, f"ties {tuning}", tuning)
    # zero gap penalties: trailing gaps are free, so gap cells tie with their
    # neighbours (needs mismatch >= gap_open = 0 for the packed form)
    b0 = wl.make_batch("ties-free-gaps", qs, rs, wl.dna_matrix(2, 0), 0, 0)
    both_forms(gpu_lib, ctx, b0, oracle.align_workload(b0), "ties, gaps 0/0", (2, 1e9))


def test_hand_worked_examples(gpu_lib, ctx):
    """The small cases whose outputs were worked out by hand (end ties on
    rend and on qend, a start tie, no alignment, a gap in the best path)."""
    enc = {"A": 0, "C": 1, "G": 2, "T": 3}
    pairs = [("ACGTACGT", "ACGTTACGT"), ("AC", "ACAC"), ("ACAC", "AC"), ("ACGGGG", "AAGGGG"),
             ("AAAA", "CCCC"), ("ATGCT", "AGCT")]
    qs = [np.array([enc[c] for c in q], np.uint8) for q, _ in pairs]
    rs = [np.array([enc[c] for c in r], np.uint8) for _, r in pairs]
    b = wl.make_batch("hand", qs, rs, wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(b)
    assert expect[:5].tolist() == [[18, 7, 8, 0, 0], [6, 1, 1, 0, 0], [6, 1, 1, 0, 0],
                                   [12, 5, 5, 2, 2], [0, -1, -1, -1, -1]]
    both_forms(gpu_lib, ctx, b, expect, "hand-worked", (1, 1e9))


@pytest.mark.parametrize("lg", [1, 3])
def test_packed_bound_edges(gpu_lib, ctx, lg):
    """With 32-bit profile words (scale 8) the bound 8 (3 min(n, m) + 3 + 6)
    <= 32767 holds up to min(n, m) = 1362; from 1363 the byte profile (scale
    4) takes over, up to 2727 (a self-alignment there scores 8181, scaled
    32724); at 2728 the plan keeps int32.  Exact on every side."""
    rng = np.random.default_rng(53 + lg)
    for L, packed in ((1362, True), (1363, True), (2727, True), (2728, False)):
        qs, rs = [], []
        for extra in (0, 5, 700):
            q = rng.integers(0, 4, L).astype(np.uint8)
            r = np.concatenate([rng.integers(0, 4, extra).astype(np.uint8), q])
            qs.append(q)
            rs.append(r)
            qs.append(q.copy())
            rs.append(q.copy())
        b = wl.make_batch(f"bound-{L}", qs, rs, wl.dna_matrix(), -6, -1)
        expect = oracle.align_workload(b)
        assert expect[:, 0].max() == 3 * L
        both_forms(gpu_lib, ctx, b, expect, f"bound L={L}", (lg, 1e9), want_packed=packed)


def test_linear_gaps_packed(gpu_lib, ctx):
    """go == ge with s - go >= 0 takes the packed form without E and F."""
    for mat, g in ((wl.dna_matrix(), -3), (wl.dna_matrix(2, -2), -2)):
        src = wl.gen_config(1, n_pairs=300)
        b = wl.make_batch("lin-packed", [src.pair(i)[0] for i in range(src.n_pairs)],
                          [src.pair(i)[1] for i in range(src.n_pairs)], mat, g, g)
        expect = oracle.align_workload(b)
        for tuning in ((1, 1e9), (3, 1e9), (-1, 0.5)):
            both_forms(gpu_lib, ctx, b, expect, f"linear {g}", tuning)


def test_protein_short_pairs_and_larger_alphabets(gpu_lib, ctx):
    """BLOSUM62 (-11/-1) pairs take the packed form with the byte profile (a
    profile of 32-bit words for 21 residue codes leaves fewer than two blocks
    per SM); an 8-letter alphabet with small scores takes the 32-bit words.
    Both forms exact on both."""
    src = wl.gen_config(2, n_pairs=400)
    qs = [src.pair(i)[0][:300] for i in range(src.n_pairs)]
    rs = [src.pair(i)[1] for i in range(src.n_pairs)]
    b = wl.make_batch("protein-short", qs, rs, src.matrix, src.gap_open, src.gap_extend)
    expect = oracle.align_workload(b)
    for tuning in ((1, 1e9), (2, 1e9), (5, 1e9), (-1, 0.5)):
        both_forms(gpu_lib, ctx, b, expect, f"protein short {tuning}", tuning)
    lin = wl.make_batch("protein-linear", qs, rs, src.matrix, -6, -6)
    both_forms(gpu_lib, ctx, lin, oracle.align_workload(lin), "protein linear -6", (3, 1e9))
    rng = np.random.default_rng(61)
    mat = rng.integers(-3, 5, size=(8, 8)).astype(np.int8)
    np.fill_diagonal(mat, 6)
    qs8 = [rng.integers(0, 8, int(rng.integers(1, 300))).astype(np.uint8) for _ in range(300)]
    rs8 = [rng.integers(0, 8, int(rng.integers(1, 700))).astype(np.uint8) for _ in range(300)]
    b8 = wl.make_batch("alphabet-8", qs8, rs8, mat, -5, -2)
    expect8 = oracle.align_workload(b8)
    _, info8 = run_lib(gpu_lib, ctx, b8)
    for tuning in ((1, 1e9), (3, 1e9), (-1, 0.5)):
        both_forms(gpu_lib, ctx, b8, expect8, f"alphabet 8 {tuning}", tuning,
                   want_packed=info8["arith"] == "s16x2")


@pytest.mark.parametrize("k", [1, 2, 3])
def test_full_workloads_packed_vs_int32(gpu_lib, ctx, k):
    """The 100k- and 200k-pair DNA and the 20k-pair protein workloads in the
    benchmark's launch form: the packed form equals the int32 form on every
    pair and the oracle on a sample."""
    b = wl.gen_config(k)
    got, info = run_lib(gpu_lib, ctx, b, flags=gpu_lib.SW_PLAN_GRAPH)
    assert info["arith"] == "s16x2"
    got32, info32 = run_lib(gpu_lib, ctx, b, flags=gpu_lib.SW_PLAN_GRAPH | gpu_lib.SW_PLAN_NO_S16X2)
    assert info32["arith"] == "s32"
    assert_same(got, got32, f"config{k} packed vs int32")
    idx = np.random.default_rng(k).choice(b.n_pairs, min(2000, b.n_pairs), replace=False)
    assert_same(got[idx], oracle.align_workload(b, idx=idx), f"config{k} sample")


def test_out_of_range_residues_clamped(gpu_lib, ctx):
    """Residue codes at or above the alphabet size are clamped to
    alphabet_size - 1 on the device (the documented unchecked behaviour):
    every form equals the oracle on the clamped sequences."""
    rng = np.random.default_rng(67)
    qs, rs = [], []
    for _ in range(300):
        q = rng.integers(0, 4, int(rng.integers(1, 260))).astype(np.uint8)
        r = rng.integers(0, 4, int(rng.integers(1, 700))).astype(np.uint8)
        k = min(len(q), len(r))
        if rng.random() < 0.5:
            r[:k] = q[:k]
        q[rng.random(len(q)) < 0.1] = rng.integers(4, 256)
        r[rng.random(len(r)) < 0.1] = rng.integers(4, 256)
        qs.append(q)
        rs.append(r)
    raw = wl.make_batch("raw-codes", qs, rs, wl.dna_matrix(), -6, -1)
    clamped = wl.make_batch("clamped", [np.minimum(q, 3) for q in qs],
                            [np.minimum(r, 3) for r in rs], wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(clamped)
    both_forms(gpu_lib, ctx, raw, expect, "raw codes", (2, 1e9))
    got, _ = run_lib(gpu_lib, ctx, raw, mode=gpu_lib.SW_MODE_PLAIN)
    assert_same(got, expect, "raw codes, plain")
