"""GPU traceback (sw_traceback) equals the CPU oracle's CIGAR, op for op.

Positions come from the batched path (themselves checked against the
oracle elsewhere); the traceback of every aligned pair must then equal
oracle.cigar_batch on the same positions, bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


def gpu_cigars(swgb, ctx, b):
    import torch
    dev = torch.device("cuda:0")
    al = swgb.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                      b.gap_extend, mode=swgb.SW_MODE_BATCHED, ctx=ctx)
    al.run()
    res = al.results()  # (n, 5)
    res5 = np.ascontiguousarray(res.T)
    off = swgb.sw_cigar_capacity(res5)
    ops = torch.zeros(max(1, int(off[-1])), dtype=torch.int32, device=dev)
    n_ops = torch.full((b.n_pairs,), -1, dtype=torch.int32, device=dev)
    swgb.sw_traceback(ctx, al.q, b.q_offsets, al.r, b.r_offsets, b.matrix, b.gap_open,
                      b.gap_extend, res5, off, ops, n_ops)
    out = (ops.cpu().numpy().view(np.uint32), off, n_ops.cpu().numpy())
    al.close()
    return res, out


def assert_same_cigars(b, res, got):
    ops, off, n_ops = got
    eops, eoff, en = oracle.cigar_workload(b, res)
    assert np.array_equal(off, eoff)
    bad = np.flatnonzero(n_ops != en)
    assert len(bad) == 0, f"{len(bad)} pairs differ in op count; first {bad[0]}"
    for p in range(b.n_pairs):
        a = ops[off[p]:off[p] + n_ops[p]]
        e = eops[eoff[p]:eoff[p] + en[p]]
        if not np.array_equal(a, e):
            raise AssertionError(f"pair {p}: got {oracle.cigar_string(a)} "
                                 f"expected {oracle.cigar_string(e)}")


@pytest.mark.parametrize("k,n", [(0, 1000), (1, 1500), (2, 800), (3, 1500)])
def test_workloads(gpu_lib, ctx, k, n):
    b = wl.gen_config(k, n_pairs=n)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


def test_large_batch_sampled(gpu_lib, ctx):
    """A batch large enough that the host splits its preparation over worker
    threads; every 23rd pair checked against the oracle op for op."""
    b = wl.gen_config(1, n_pairs=40000)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    ops, off, n_ops = got
    idx = np.arange(0, b.n_pairs, 23)
    assert np.array_equal(res[idx], oracle.align_workload(b, idx=idx))
    eops, eoff, en = oracle.cigar_workload(b.subset(idx), res[idx])
    for k, p in enumerate(idx):
        assert n_ops[p] == en[k], f"pair {p}"
        a = ops[off[p]:off[p] + n_ops[p]]
        e = eops[eoff[k]:eoff[k] + en[k]]
        assert np.array_equal(a, e), f"pair {p}"


@pytest.mark.parametrize("go,ge", [(-1, -1), (0, 0), (-20, -3), (-16383, -1)])
def test_gap_settings(gpu_lib, ctx, go, ge):
    base = wl.gen_config(1, n_pairs=300)
    b = wl.make_batch("gaps", [base.pair(i)[0] for i in range(base.n_pairs)],
                      [base.pair(i)[1] for i in range(base.n_pairs)], base.matrix, go, ge)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    assert_same_cigars(b, res, got)


def test_long_spans_many_strips(gpu_lib, ctx):
    """Planted copies up to thousands of residues long, indels inside: spans
    on both sides of the one-strip path's 512-row limit (longer ones take
    the general kernel's 128-row strips)."""
    rng = np.random.default_rng(41)
    qs, rs = [], []
    for L in (129, 255, 256, 511, 512, 513, 520, 1000, 3000):
        q = rng.integers(0, 4, L).astype(np.uint8)
        mut = q.copy()
        for pos in rng.choice(L, size=max(1, L // 50), replace=False):
            mut[pos] = (mut[pos] + 1) % 4
        mut = np.delete(mut, rng.choice(L, size=max(1, L // 200), replace=False))
        r = np.concatenate([rng.integers(0, 4, 37).astype(np.uint8), mut,
                            rng.integers(0, 4, 11).astype(np.uint8)])
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("long", qs, rs, wl.dna_matrix(), -6, -1)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


def test_errors(gpu_lib, ctx):
    import torch
    b = wl.gen_config(0, n_pairs=50)
    res = oracle.align_workload(b)
    res5 = np.ascontiguousarray(res.T)
    off = gpu_lib.sw_cigar_capacity(res5)
    q = torch.from_numpy(b.q_seqs).cuda()
    r = torch.from_numpy(b.r_seqs).cuda()
    ops = torch.zeros(int(off[-1]) + 1, dtype=torch.int32, device="cuda")
    n_ops = torch.zeros(b.n_pairs, dtype=torch.int32, device="cuda")
    short = off.copy()
    short[1:] -= np.arange(1, b.n_pairs + 1)  # one op short for every pair
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_traceback(ctx, q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                             b.gap_extend, res5, short, ops, n_ops)
    assert e.value.code == gpu_lib.SW_ERANGE
    bad = res5.copy()
    p = int(np.flatnonzero(res[:, 0] > 0)[0])
    bad[2, p] = int(b.r_offsets[p + 1] - b.r_offsets[p])  # rend past the reference
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_traceback(ctx, q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                             b.gap_extend, bad, gpu_lib.sw_cigar_capacity(bad), ops, n_ops)
    assert e.value.code == gpu_lib.SW_ERANGE


def _planted(rng, lengths, A):
    """A planted copy of each query with substitutions and one indel away
    from its ends, so that the located span is (about) the whole query."""
    qs, rs = [], []
    for L in lengths:
        q = rng.integers(0, A, L).astype(np.uint8)
        mut = q.copy()
        if L > 24:
            mid = np.arange(8, L - 8)
            for pos in rng.choice(mid, size=max(1, L // 25), replace=False):
                mut[pos] = (mut[pos] + 1) % A
            mut = np.delete(mut, int(rng.integers(8, L - 8)))
        r = np.concatenate([rng.integers(0, A, 13).astype(np.uint8), mut,
                            rng.integers(0, A, 7).astype(np.uint8)])
        qs.append(q)
        rs.append(r)
    return qs, rs


def test_every_width_and_row_count(gpu_lib, ctx):
    """Spans at and just past every fast-path size R x G (R = 10, 12, 14, 16
    rows per lane, G = 1..32 lanes), so every (width, rows) class runs."""
    sizes = sorted({R << lg for R in (10, 12, 14, 16) for lg in range(6)})
    lengths = [L for s in sizes for L in (s - 1, s, s + 1) if 1 <= L <= 520]
    qs, rs = _planted(np.random.default_rng(7), lengths, 4)
    b = wl.make_batch("classes", qs, rs, wl.dna_matrix(), -6, -1)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


@pytest.mark.parametrize("A", [20, 32])
def test_large_alphabets(gpu_lib, ctx, A):
    """BLOSUM62 (a 40 KB profile per block) and a 32-letter alphabet (64 KB:
    the kernel's shared-memory limit raised for the launch)."""
    rng = np.random.default_rng(100 + A)
    if A == 20:
        mat = np.asarray(wl.load_blosum62()[0], dtype=np.int8)
        go, ge = -11, -1
    else:
        mat = rng.integers(-9, 10, size=(A, A)).astype(np.int8)
        np.fill_diagonal(mat, 12)
        go, ge = -10, -2
    lengths = [int(x) for x in rng.integers(5, 400, size=120)]
    qs, rs = _planted(rng, lengths, A)
    b = wl.make_batch(f"alpha{A}", qs, rs, mat, go, ge)
    res, got = gpu_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)
