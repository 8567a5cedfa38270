"""The one-shot call with device offsets: planned on the device, asynchronous.

sw_align_batch / sw_align_batch_ex read the offsets on the device, plan the
batch there (route, lane-group width, longest-first radix sort, queue
tables) and run the kernels, without reading anything back.  Every output is
compared with the CPU oracle bit for bit (exact integer path, tolerance 0):
the full 100k DNA, 20k protein and 200k skewed workloads, edge lengths
under every bulk width, pairs beyond the slots' reach and beyond the scaled
score bound (plain kernel), empty sequences and bad offsets.  A test also
shows that the call returns while the device is still busy with earlier work
on the same stream, i.e. that it never waits for the device.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

from test_gpu_parity import EDGE, TUNINGS, assert_same, edge_batch  # noqa: E402


def _dev(b):
    import torch
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(b.q_seqs if b.q_seqs.size else np.zeros(16, np.uint8)).to(dev)
    r = torch.from_numpy(b.r_seqs if b.r_seqs.size else np.zeros(16, np.uint8)).to(dev)
    qo = torch.from_numpy(b.q_offsets).to(dev)
    ro = torch.from_numpy(b.r_offsets).to(dev)
    return q, r, qo, ro


def one_shot(swgb, b, ctx=None, mode=None, stream=None, out=None):
    import torch
    q, r, qo, ro = _dev(b)
    if out is None:
        out = torch.full((5, max(1, b.n_pairs)), -9, dtype=torch.int32, device=q.device)
    if ctx is None:
        swgb.sw_align_batch(q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend, out, stream)
    else:
        swgb.sw_align_batch_ex(ctx, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend,
                               swgb.SW_MODE_AUTO if mode is None else mode, out, stream)
    torch.cuda.synchronize()
    return out[:, :b.n_pairs].T.contiguous().cpu().numpy()


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_full_workloads_one_shot(gpu_lib, k):
    """Workloads 0-3 at full size through sw_align_batch (default context)."""
    b = wl.gen_config(k)
    got = one_shot(gpu_lib, b)
    expect = oracle.align_workload(b)
    assert_same(got, expect, f"one-shot config{k}")
    dctx = gpu_lib.sw_default_ctx(0)
    assert gpu_lib.sw_ctx_status(dctx) == 0


@pytest.mark.parametrize("tuning", TUNINGS, ids=[f"G{1 << t[0] if t[0] >= 0 else 'auto'}-cap{t[1]:g}"
                                                 for t in TUNINGS])
def test_edge_lengths_every_bulk_width(gpu_lib, ctx, tuning):
    b = edge_batch("dna", 17 + tuning[0], EDGE, EDGE[::3])
    expect = oracle.align_workload(b)
    gpu_lib.sw_ctx_set_tuning(ctx, *tuning)
    try:
        got = one_shot(gpu_lib, b, ctx=ctx)
    finally:
        gpu_lib.sw_ctx_set_tuning(ctx, -1, 0.5)
    assert_same(got, expect, f"one-shot edge dna tuning={tuning}")
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_edge_lengths_protein_and_plain_mode(gpu_lib, ctx):
    b = edge_batch("protein", 15, EDGE[::2], EDGE[1::3])
    expect = oracle.align_workload(b)
    assert_same(one_shot(gpu_lib, b, ctx=ctx), expect, "one-shot edge protein")
    assert_same(one_shot(gpu_lib, b, ctx=ctx, mode=gpu_lib.SW_MODE_PLAIN), expect,
                "one-shot edge protein, plain mode")
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_long_pairs_beyond_the_slots_and_the_packed_bound(gpu_lib, ctx):
    """Pairs up to the maximum length: the packed route up to its bound, the
    int32 route beyond it, wider groups for long sequences and the plain
    kernel beyond the widest group's slot (longer sequence > ~16,400)."""
    rng = np.random.default_rng(29)
    qs, rs = [], []
    for n, m in [(1362, 1400), (1363, 1400), (3000, 3000), (9000, 9500), (16000, 300),
                 (300, 17000), (20000, 20000), (1, 65535), (65535, 40), (12000, 12000)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m, 2500)
        r[m - k:] = q[n - k:]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("one-shot-long", qs, rs, wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(b)
    assert_same(one_shot(gpu_lib, b, ctx=ctx), expect, "one-shot long pairs")
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_wide_scores_and_linear_gaps(gpu_lib, ctx):
    rng = np.random.default_rng(31)
    mat = np.full((4, 4), -90, np.int8)
    np.fill_diagonal(mat, 120)
    qs, rs = [], []
    for n, m in [(300, 400), (60, 80), (1200, 900), (5, 7)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        r[:n // 2] = q[:n // 2]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("one-shot-wide", qs, rs, mat, -200, -30)
    assert_same(one_shot(gpu_lib, b, ctx=ctx), oracle.align_workload(b), "one-shot wide scores")
    lin = wl.gen_config(1, n_pairs=3000)
    lin.gap_open, lin.gap_extend = -3, -3
    assert_same(one_shot(gpu_lib, lin, ctx=ctx), oracle.align_workload(lin), "one-shot linear")
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_empty_sequences_and_bad_offsets(gpu_lib, ctx):
    """Empty sequences give the no-alignment outputs; offsets that decrease,
    go negative or span more than the maximum length give them too and set
    the context's status bit, without touching the other pairs."""
    import torch
    base = wl.gen_config(0, n_pairs=8)
    qs = [base.pair(i)[0] for i in range(8)] + [np.zeros(0, np.uint8)] * 2
    rs = [base.pair(i)[1] for i in range(8)] + [np.zeros(0, np.uint8), base.pair(0)[1]]
    b = wl.make_batch("empty", qs, rs, base.matrix, base.gap_open, base.gap_extend)
    expect = oracle.align_workload(b)
    assert_same(one_shot(gpu_lib, b, ctx=ctx), expect, "empty sequences")
    assert gpu_lib.sw_ctx_status(ctx) == 0

    dev = torch.device("cuda", 0)
    qo = b.q_offsets.copy()
    ro = b.r_offsets.copy()
    # pair 2: query offsets decrease; pair 5: a reference span above the
    # maximum length (the buffer below is long enough for every offset used)
    qo_bad = qo.copy()
    qo_bad[3] = qo_bad[2] - 5
    ro_bad = ro.copy()
    ro_bad[6:] += 70000
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.zeros(int(ro_bad[-1]) + 16, dtype=torch.uint8, device=dev)
    rh = np.zeros(int(ro_bad[-1]) + 16, np.uint8)
    for i in range(b.n_pairs):
        if i != 5:
            s = b.pair(i)[1]
            rh[ro_bad[i]:ro_bad[i] + len(s)] = s
    r.copy_(torch.from_numpy(rh))
    out = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device=dev)
    gpu_lib.sw_align_batch_ex(ctx, q, torch.from_numpy(qo_bad).to(dev), r,
                              torch.from_numpy(ro_bad).to(dev), b.matrix, b.gap_open,
                              b.gap_extend, gpu_lib.SW_MODE_AUTO, out)
    torch.cuda.synchronize()
    got = out.T.cpu().numpy()
    none = np.array([0, -1, -1, -1, -1], np.int32)
    for i in range(b.n_pairs):
        if i in (2, 5):
            assert np.array_equal(got[i], none), (i, got[i])
        elif i != 3:  # pair 3 starts where the bad offset was planted
            assert np.array_equal(got[i], expect[i]), (i, got[i], expect[i])
    assert gpu_lib.sw_ctx_status(ctx) & gpu_lib.STATUS_BAD_OFFSETS


def test_call_returns_without_waiting_for_the_device(gpu_lib, ctx):
    """Enqueued behind a long device-side wait on the same stream, the call
    returns while that wait is still running: it reads nothing back and
    never synchronises.  The results are correct afterwards."""
    import torch
    b = wl.gen_config(1, n_pairs=20000)
    q, r, qo, ro = _dev(b)
    out = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device=q.device)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        torch.cuda._sleep(400_000_000)  # about 0.2 s of device time at 2 GHz
        gpu_lib.sw_align_batch_ex(ctx, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend,
                                  gpu_lib.SW_MODE_AUTO, out, s)
        still_busy = not s.query()
    s.synchronize()
    assert still_busy, "the one-shot call waited for the device"
    assert_same(out.T.cpu().numpy(), oracle.align_workload(b), "one-shot behind a wait")


def test_overlapping_calls_on_two_streams(gpu_lib, ctx):
    """Calls on different streams use workspaces of their own."""
    import torch
    b1 = wl.gen_config(1, n_pairs=6000)
    b2 = wl.gen_config(2, n_pairs=3000)
    d1, d2 = _dev(b1), _dev(b2)
    o1 = torch.full((5, b1.n_pairs), -9, dtype=torch.int32, device=d1[0].device)
    o2 = torch.full((5, b2.n_pairs), -9, dtype=torch.int32, device=d1[0].device)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        gpu_lib.sw_align_batch_ex(ctx, d1[0], d1[2], d1[1], d1[3], b1.matrix, b1.gap_open,
                                  b1.gap_extend, gpu_lib.SW_MODE_AUTO, o1, s1)
        gpu_lib.sw_align_batch_ex(ctx, d2[0], d2[2], d2[1], d2[3], b2.matrix, b2.gap_open,
                                  b2.gap_extend, gpu_lib.SW_MODE_AUTO, o2, s2)
    torch.cuda.synchronize()
    assert_same(o1.T.cpu().numpy(), oracle.align_workload(b1), "stream 1")
    assert_same(o2.T.cpu().numpy(), oracle.align_workload(b2), "stream 2")
    assert gpu_lib.sw_ctx_status(ctx) == 0


@pytest.mark.parametrize("k", [1, 2])
def test_page_locked_host_inputs_read_in_place(gpu_lib, ctx, k):
    """Where the device reads host memory coherently, the call takes the
    page-locked host buffers of the sequences and offsets themselves."""
    import torch
    swgb = gpu_lib
    if not swgb.sw_ctx_host_in_place(ctx):
        pytest.skip("this device does not read page-locked host memory in place")
    b = wl.gen_config(k, n_pairs=20000)
    swgb.sw_ctx_status(ctx)  # (read and cleared: earlier tests set bits on purpose)
    qh = torch.from_numpy(b.q_seqs).pin_memory()
    rh = torch.from_numpy(b.r_seqs).pin_memory()
    qoh = torch.from_numpy(b.q_offsets).pin_memory()
    roh = torch.from_numpy(b.r_offsets).pin_memory()
    out = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device="cuda")
    swgb.sw_align_batch_ex(ctx, qh, qoh, rh, roh, b.matrix, b.gap_open, b.gap_extend,
                           swgb.SW_MODE_AUTO, out)
    torch.cuda.synchronize()
    got = out.T.contiguous().cpu().numpy()
    assert np.array_equal(got, one_shot(swgb, b, ctx=ctx))
    idx = np.arange(0, b.n_pairs, 11)
    assert np.array_equal(got[idx], oracle.align_workload(b, idx=idx))
    assert swgb.sw_ctx_status(ctx) == 0
