"""GPU traceback from results already on the device (sw_traceback_device,
sw_cigar_capacity_device) equals the CPU oracle's CIGAR op for op, and the
host-prepared call's output bit for bit.

The span classification, sort and choice-word layout run as kernels here,
so every case of the host-prepared call's tests runs again through them:
the four workloads, every (width, rows) class at its size limits, spans past
the one-strip limit (general path), gap settings, large alphabets, and the
range errors, which the device must find and report by pair.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_cigar import _planted, assert_same_cigars

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


def device_cigars(swgb, ctx, b, check_host=True):
    """Aligns b, then traces back from the device results through the device
    call (offsets computed on the device too); returns the results and the
    ops, offsets and counts on the host."""
    import torch
    dev = torch.device("cuda:0")
    al = swgb.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                      b.gap_extend, mode=swgb.SW_MODE_BATCHED, ctx=ctx)
    al.run()
    res = al.results()
    qo = torch.from_numpy(np.asarray(b.q_offsets, dtype=np.int64)).to(dev)
    ro = torch.from_numpy(np.asarray(b.r_offsets, dtype=np.int64)).to(dev)
    coff = torch.full((b.n_pairs + 1,), -5, dtype=torch.int64, device=dev)
    swgb.sw_cigar_capacity_device(al.out, coff)
    off = coff.cpu().numpy()
    res5 = np.ascontiguousarray(res.T)
    assert np.array_equal(off, swgb.sw_cigar_capacity(res5))
    ops = torch.zeros(max(1, int(off[-1])), dtype=torch.int32, device=dev)
    n_ops = torch.full((b.n_pairs,), -1, dtype=torch.int32, device=dev)
    swgb.sw_traceback_device(ctx, al.q, qo, al.r, ro, b.matrix, b.gap_open, b.gap_extend,
                             al.out, coff, ops, n_ops)
    got = (ops.cpu().numpy().view(np.uint32), off, n_ops.cpu().numpy())
    if check_host:
        hops = torch.zeros_like(ops)
        hn = torch.full_like(n_ops, -1)
        swgb.sw_traceback(ctx, al.q, b.q_offsets, al.r, b.r_offsets, b.matrix, b.gap_open,
                          b.gap_extend, res5, off, hops, hn)
        hn = hn.cpu().numpy()
        assert np.array_equal(hn, got[2])
        hops = hops.cpu().numpy().view(np.uint32)
        for p in range(b.n_pairs):
            assert np.array_equal(hops[off[p]:off[p] + hn[p]], got[0][off[p]:off[p] + hn[p]]), p
    al.close()
    return res, got


@pytest.mark.parametrize("k,n", [(0, 1000), (1, 1500), (2, 800), (3, 1500)])
def test_workloads(gpu_lib, ctx, k, n):
    b = wl.gen_config(k, n_pairs=n)
    res, got = device_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


def test_every_width_and_row_count(gpu_lib, ctx):
    sizes = sorted({R << lg for R in (10, 12, 14, 16) for lg in range(6)})
    lengths = [L for s in sizes for L in (s - 1, s, s + 1) if 1 <= L <= 520]
    qs, rs = _planted(np.random.default_rng(8), lengths, 4)
    b = wl.make_batch("classes", qs, rs, wl.dna_matrix(), -6, -1)
    res, got = device_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


def test_long_spans_general_path(gpu_lib, ctx):
    """Spans on both sides of the one-strip limit: the longer ones are
    listed by the device for the general kernel."""
    rng = np.random.default_rng(43)
    lengths = [129, 511, 512, 513, 700, 1000, 2500, 40, 513, 3000]
    qs, rs = _planted(rng, lengths, 4)
    b = wl.make_batch("long", qs, rs, wl.dna_matrix(), -6, -1)
    res, got = device_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


@pytest.mark.parametrize("go,ge", [(-1, -1), (-20, -3), (-16383, -1)])
def test_gap_settings(gpu_lib, ctx, go, ge):
    base = wl.gen_config(1, n_pairs=300)
    b = wl.make_batch("gaps", [base.pair(i)[0] for i in range(base.n_pairs)],
                      [base.pair(i)[1] for i in range(base.n_pairs)], base.matrix, go, ge)
    res, got = device_cigars(gpu_lib, ctx, b)
    assert_same_cigars(b, res, got)


@pytest.mark.parametrize("A", [20, 32])
def test_large_alphabets(gpu_lib, ctx, A):
    rng = np.random.default_rng(200 + A)
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
    res, got = device_cigars(gpu_lib, ctx, b)
    assert np.array_equal(res, oracle.align_workload(b))
    assert_same_cigars(b, res, got)


def test_large_batch_twice(gpu_lib, ctx):
    """40,000 pairs, twice on the same context (the planning workspace and
    the choice words come back from the pool); every 29th pair against the
    oracle, all pairs against the host-prepared call."""
    b = wl.gen_config(1, n_pairs=40000)
    idx = np.arange(0, b.n_pairs, 29)
    for _ in range(2):
        res, got = device_cigars(gpu_lib, ctx, b)
        ops, off, n_ops = got
        eops, eoff, en = oracle.cigar_workload(b.subset(idx), res[idx])
        for k, p in enumerate(idx):
            assert n_ops[p] == en[k], f"pair {p}"
            assert np.array_equal(ops[off[p]:off[p] + n_ops[p]], eops[eoff[k]:eoff[k] + en[k]])


def test_unaligned_and_empty(gpu_lib, ctx):
    """Pairs with score 0 (and empty sequences) get no ops; a batch of none
    of them enqueues nothing but the cleared counts."""
    import torch
    qs = [np.array([0, 0, 0], np.uint8), np.zeros(0, np.uint8), np.array([1, 2], np.uint8)]
    rs = [np.array([3, 3, 3], np.uint8), np.array([1, 1], np.uint8), np.zeros(0, np.uint8)]
    b = wl.make_batch("zero", qs, rs, wl.dna_matrix(), -6, -1)
    res = oracle.align_workload(b)
    assert np.all(res[:, 0] == 0)
    dev = torch.device("cuda:0")
    res_d = torch.from_numpy(np.ascontiguousarray(res.T)).to(dev)
    qo = torch.from_numpy(b.q_offsets).to(dev)
    ro = torch.from_numpy(b.r_offsets).to(dev)
    coff = torch.zeros(b.n_pairs + 1, dtype=torch.int64, device=dev)
    gpu_lib.sw_cigar_capacity_device(res_d, coff)
    assert coff.cpu().numpy().tolist() == [0] * (b.n_pairs + 1)
    q = torch.from_numpy(np.concatenate(qs)).to(dev)
    r = torch.from_numpy(np.concatenate(rs)).to(dev)
    ops = torch.zeros(1, dtype=torch.int32, device=dev)
    n_ops = torch.full((b.n_pairs,), 9, dtype=torch.int32, device=dev)
    gpu_lib.sw_traceback_device(ctx, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend, res_d,
                                coff, ops, n_ops)
    assert n_ops.cpu().numpy().tolist() == [0] * b.n_pairs


def test_errors_found_on_the_device(gpu_lib, ctx):
    import torch
    dev = torch.device("cuda:0")
    b = wl.gen_config(0, n_pairs=60)
    res = oracle.align_workload(b)
    res5 = np.ascontiguousarray(res.T)
    off = gpu_lib.sw_cigar_capacity(res5)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    qo = torch.from_numpy(b.q_offsets).to(dev)
    ro = torch.from_numpy(b.r_offsets).to(dev)
    ops = torch.zeros(int(off[-1]) + 1, dtype=torch.int32, device=dev)
    n_ops = torch.zeros(b.n_pairs, dtype=torch.int32, device=dev)
    aligned = np.flatnonzero(res[:, 0] > 0)
    p0, p1 = int(aligned[3]), int(aligned[7])

    def call(res_h, off_h, qo_d=qo):
        gpu_lib.sw_traceback_device(ctx, q, qo_d, r, ro, b.matrix, b.gap_open, b.gap_extend,
                                    torch.from_numpy(np.ascontiguousarray(res_h)).to(dev),
                                    torch.from_numpy(off_h).to(dev), ops, n_ops)

    short = off.copy()
    short[p1 + 1:] -= 1  # pair p1 one op short
    short[p0 + 1:] -= 1  # and pair p0: the smaller index is named
    with pytest.raises(gpu_lib.SwError) as e:
        call(res5, short)
    assert e.value.code == gpu_lib.SW_ERANGE and f"pair {p0} " in str(e.value)
    bad = res5.copy()
    bad[2, p1] = int(b.r_offsets[p1 + 1] - b.r_offsets[p1])  # rend past the reference
    with pytest.raises(gpu_lib.SwError) as e:
        call(bad, gpu_lib.sw_cigar_capacity(bad))
    assert e.value.code == gpu_lib.SW_ERANGE and f"pair {p1} " in str(e.value)
    dec = b.q_offsets.copy()
    dec[5] = dec[4] - 1  # pair 4 has a negative length
    with pytest.raises(gpu_lib.SwError) as e:
        call(res5, off, torch.from_numpy(dec).to(dev))
    assert e.value.code == gpu_lib.SW_ERANGE and "pair 4 " in str(e.value)
    # the context still serves a good call afterwards
    call(res5, off)
    got = (ops.cpu().numpy().view(np.uint32), off, n_ops.cpu().numpy())
    assert_same_cigars(b, res, got)


def test_refuses_stream_capture(gpu_lib, ctx):
    """The call waits for its classification kernels, so on a stream being
    captured it refuses before enqueueing anything."""
    import torch
    dev = torch.device("cuda", 0)
    b = wl.gen_config(0, n_pairs=16)
    res = oracle.align_workload(b)
    res5 = np.ascontiguousarray(res.T)
    off = gpu_lib.sw_cigar_capacity(res5)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    qo = torch.from_numpy(b.q_offsets).to(dev)
    ro = torch.from_numpy(b.r_offsets).to(dev)
    res_d = torch.from_numpy(res5).to(dev)
    off_d = torch.from_numpy(off).to(dev)
    ops = torch.zeros(int(off[-1]) + 1, dtype=torch.int32, device=dev)
    n_ops = torch.zeros(b.n_pairs, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    caught = None
    with torch.cuda.graph(g, stream=stream):
        try:
            gpu_lib.sw_traceback_device(ctx, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend,
                                        res_d, off_d, ops, n_ops, stream)
        except gpu_lib.SwError as e:
            caught = e
        n_ops.add_(0)  # something to capture
    assert caught is not None and caught.code == gpu_lib.SW_EINVAL
    # outside the capture the same call works
    gpu_lib.sw_traceback_device(ctx, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend, res_d,
                                off_d, ops, n_ops, stream)
    stream.synchronize()
    got = (ops.cpu().numpy().view(np.uint32), off, n_ops.cpu().numpy())
    assert_same_cigars(b, res, got)
