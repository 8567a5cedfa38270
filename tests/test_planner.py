"""Host-side planning, checked without a GPU through sw_plan_preview: which
arithmetic form and profile a batch takes, which lane-group width each pair
gets, and the order of the kernel's queues."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def lib():
    import paper_2208_12350_gb300 as swgb
    swgb.load()
    return swgb


def _batch(lens_q, lens_r, matrix, go, ge, seed=0, A=4):
    rng = np.random.default_rng(seed)
    qs = [rng.integers(0, A, n).astype(np.uint8) for n in lens_q]
    rs = [rng.integers(0, A, m).astype(np.uint8) for m in lens_r]
    return wl.make_batch("planner", qs, rs, matrix, go, ge)


def preview(lib, b, **kw):
    return lib.sw_plan_preview(b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend, **kw)


def test_form_selection(lib):
    """Small alphabets take the packed form with 32-bit profile words,
    BLOSUM62 the byte profile (its 32-bit profile leaves one block per SM),
    and each bound's edge moves the batch to the next form."""
    dna = wl.gen_config(0, n_pairs=200)
    assert preview(lib, dna)[0] == "s16x2"
    assert preview(lib, dna, flags=lib.SW_PLAN_NO_S16X2)[0] == "int32"
    prot = wl.gen_config(2, n_pairs=300)
    assert preview(lib, prot)[0] == "s16x2-byte-profile"
    assert preview(lib, prot, flags=lib.SW_PLAN_NO_S16X2)[0] == "int32-int8-profile"
    go40 = wl.make_batch("go40", [prot.pair(i)[0] for i in range(50)],
                         [prot.pair(i)[1] for i in range(50)], prot.matrix, -40, -1)
    assert preview(lib, go40)[0] == "int32-int8-profile"  # s - go up to 51 > 31
    fig2 = _batch([100] * 5, [300] * 5, wl.dna_matrix(2, -2), -1, -1)
    assert preview(lib, fig2)[0] == "int32"  # mismatch below gap_open
    for L, kind in ((1362, "s16x2"), (1363, "s16x2-byte-profile"),
                    (2727, "s16x2-byte-profile"), (2728, "int32")):
        b = _batch([L, 50], [L + 10, 60], wl.dna_matrix(), -6, -1)
        assert preview(lib, b)[0] == kind, L


def test_every_pair_planned_once_longest_first(lib):
    """Every pair has one lane-group width (or the plain kernel), each width
    class's queue positions are a permutation, and a queue hands pairs out
    longest first by the planner's estimate, which grows with the pair's
    strips and with its columns (strips x (columns + a fixed cost per strip
    start)): no pair is queued after one it dominates in both."""
    b = wl.gen_config(3, n_pairs=3000)
    for tuning in ((-1, 0.5), (1, 0.05), (2, 1e9), (3, 0.25)):
        kind, lg, rank = preview(lib, b, narrow_log2g=tuning[0], cap_fraction=tuning[1])
        assert kind == "s16x2"
        assert np.all((lg >= 1) & (lg <= 5))
        n = np.diff(b.q_offsets)
        m = np.diff(b.r_offsets)
        for g in np.unique(lg):
            sel = np.flatnonzero(lg == g)
            assert np.array_equal(np.sort(rank[sel]), np.arange(len(sel)))
            G = 1 << int(g)
            order = sel[np.argsort(rank[sel])]
            strips = np.ceil(n[order] / (16 * G)).astype(np.int64)
            cols = (m[order] + G - 1 + 3) // 4 * 4
            # for every queue position, the most columns among the later pairs
            # with at least as many strips must not exceed its own, and a later
            # pair with more strips must not have as many columns
            for lvl in np.unique(strips):
                later_max = np.maximum.accumulate(
                    np.where(strips >= lvl, cols, -1)[::-1])[::-1]
                nxt = np.append(later_max[1:], -1)
                at = strips == lvl
                assert np.all(nxt[at] <= cols[at]), (tuning, g, int(lvl))
                more = np.maximum.accumulate(np.where(strips > lvl, cols, -1)[::-1])[::-1]
                nxt_more = np.append(more[1:], -1)
                assert np.all(nxt_more[at] < cols[at]), (tuning, g, int(lvl))


def test_half_width_tails(lib):
    """With a bulk width G and no cap in effect, a packed-form pair whose last
    strip of 16 G rows would be at most half used takes G / 2; the byte
    profile (protein) and the int32 form keep one width."""
    lens = list(range(100, 301, 7))
    b = _batch(lens, [600] * len(lens), wl.dna_matrix(), -6, -1, seed=3)
    kind, lg, _ = preview(lib, b, narrow_log2g=3, cap_fraction=1e9)
    assert kind == "s16x2"
    n = np.array(lens)
    tail = n % 128
    expect = np.where((tail > 0) & (tail <= 64), 2, 3)
    assert np.array_equal(lg, expect)
    _, lg32, _ = preview(lib, b, narrow_log2g=3, cap_fraction=1e9, flags=lib.SW_PLAN_NO_S16X2)
    assert np.all(lg32 == 3)
    s62, _ = wl.load_blosum62()
    bp = _batch(lens, [600] * len(lens), s62.astype(np.int8), -11, -1, seed=4, A=20)
    kindp, lgp, _ = preview(lib, bp, narrow_log2g=3, cap_fraction=1e9)
    assert kindp == "s16x2-byte-profile" and np.all(lgp == 3)


def test_long_pairs_go_to_wider_groups(lib):
    """Pairs whose sweep at the bulk width exceeds the cap (a fraction of the
    mean load per group) go to the narrowest wider class that fits, the
    widest when none does; the bulk keeps its width.  One SM: 192 groups of
    2 lanes; 2,000 pairs of 100 x 400 (sweep 4 x 404 steps) and three of
    3,000 / 5,000 / 8,000 x 4,000 (mean load about 27,000 steps)."""
    lens_q = [100] * 2000 + [3000, 5000, 8000]
    lens_r = [400] * 2000 + [4000, 4000, 4000]
    b = _batch(lens_q, lens_r, wl.dna_matrix(), -6, -1, seed=5)
    _, lg, _ = preview(lib, b, narrow_log2g=1, cap_fraction=1.0, sm_count=1)
    assert np.all(lg[:2000] == 1)
    assert list(lg[2000:]) == [5, 5, 5]
    _, lg_nocap, _ = preview(lib, b, narrow_log2g=1, cap_fraction=1e9, sm_count=1)
    assert np.all(lg_nocap == 1)


@pytest.mark.parametrize("lg_bulk", [0, 1, 2, 3, 4, 5])
def test_every_fixed_bulk_width(lib, lg_bulk):
    """Every bulk width sw_ctx_set_tuning accepts, up to 32 lanes, with pairs
    above the cap: the bulk keeps its width (0 means the narrowest, 2
    lanes), a pair above the cap takes a class no narrower than the bulk
    and at most 32 lanes wide (at the widest bulk width it stays there)."""
    lens_q = [100] * 600 + [3000, 5000, 8000]
    lens_r = [400] * 600 + [4000, 4000, 4000]
    b = _batch(lens_q, lens_r, wl.dna_matrix(), -6, -1, seed=8)
    bulk = max(lg_bulk, 1)
    for cap in (0.25, 1.0, 1e9):
        _, lg, rank = preview(lib, b, narrow_log2g=lg_bulk, cap_fraction=cap, sm_count=1)
        assert np.all((lg[:600] == bulk) | (lg[:600] == bulk - 1))  # half-width tails
        assert np.all((lg[600:] >= bulk) & (lg[600:] <= 5))
        for g in np.unique(lg):  # each class's queue positions are a permutation
            sel = np.flatnonzero(lg == g)
            assert np.array_equal(np.sort(rank[sel]), np.arange(len(sel)))
    _, lg, _ = preview(lib, b, narrow_log2g=lg_bulk, cap_fraction=0.25, sm_count=1)
    assert list(lg[600:]) == [5, 5, 5]


def test_pairs_beyond_the_batched_bounds_take_the_plain_kernel(lib):
    """Scores beyond the scaled int32 key and lengths beyond 65,471 residues
    go to the one-block-per-pair kernel; empty pairs stay on the batched path."""
    mat = np.full((4, 4), -90, np.int8)
    np.fill_diagonal(mat, 120)
    b = _batch([300, 50, 2100, 0], [400, 60, 2100, 10], mat, -200, -30, seed=6)
    _, lg, rank = preview(lib, b)
    assert list(lg == -1) == [True, False, True, False]
    assert sorted(rank[lg == -1]) == [0, 1]
    big = _batch([300, 300], [65471, 65472], wl.dna_matrix(), -6, -1, seed=7)
    _, lgb, _ = preview(lib, big)
    assert lgb[0] >= 1 and lgb[1] == -1


def test_preview_rejects_bad_arguments(lib):
    b = wl.gen_config(0, n_pairs=4)
    with pytest.raises(lib.SwError):
        preview(lib, b, narrow_log2g=6)
    with pytest.raises(lib.SwError):
        lib.sw_plan_preview(b.q_offsets, b.r_offsets, b.matrix, 0, -1)


def test_default_plans_take_the_measured_best_widths(lib):
    """Without autotuning, the planner's own choice (its simulated schedule,
    with each strip start charged to the whole warp) lands where measurement
    on a GB300 put the best plans: on the 100k DNA workload 8-lane bulk groups
    with 4-lane tails (2,228 GCUPS, against 1,995 for the all-2-lane plan the
    planner chose without the strip charge), on the 20k protein workload
    8-lane groups (1,922), and on the 200k skewed DNA workload 8- and 4-lane
    groups (2,073).  A change to the cost model that moves these plans must
    be re-measured."""
    sms = 152
    b1 = wl.gen_config(1)
    _, lg, _ = preview(lib, b1, sm_count=sms)
    h = np.bincount(lg[lg >= 0], minlength=6)
    assert h[3] >= 0.4 * b1.n_pairs and h[2] + h[3] == b1.n_pairs, h.tolist()
    b2 = wl.gen_config(2)
    _, lg, _ = preview(lib, b2, sm_count=sms)
    h = np.bincount(lg[lg >= 0], minlength=6)
    assert h[3] >= 0.95 * b2.n_pairs and h[1] == h[2] == 0, h.tolist()
    b3 = wl.gen_config(3)
    _, lg, _ = preview(lib, b3, sm_count=sms)
    h = np.bincount(lg[lg >= 0], minlength=6)
    assert h[2] + h[3] >= 0.99 * b3.n_pairs and h[1] == 0, h.tolist()


def test_small_batches_take_wide_groups(lib):
    """Batches too small to fill the GPU: the planner's simulation picks the
    widths a sweep of fixed tunings on a GB300 measured best (identical
    outputs under every tuning): 1,000 pairs of the 1k DNA workload on
    32-lane groups (0.099 ms, against 0.109 at the best of 2, 4 and 8
    lanes), 4,000 on 16-lane groups (0.148 ms, against 0.207), and a
    20,000-pair slice of the 100k DNA workload on 16-lane bulk groups with
    8-lane tails (1.203 ms, against 1.282)."""
    for n, want in ((1000, {5}), (4000, {4})):
        b = wl.gen_config(0, n_pairs=n)
        _, lg, _ = preview(lib, b, sm_count=152)
        assert set(np.unique(lg).tolist()) == want, np.bincount(lg, minlength=6).tolist()
    b = wl.gen_config(1, n_pairs=20000)
    _, lg, _ = preview(lib, b, sm_count=152)
    h = np.bincount(lg, minlength=6)
    assert h[4] >= 0.5 * b.n_pairs and h[3] + h[4] == b.n_pairs, h.tolist()
