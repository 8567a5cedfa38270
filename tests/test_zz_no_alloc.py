"""The allocation-free entry point gives the same results as the planned path.

sw_align_batch_static exists for callers that cannot allocate device memory
while they align (their device memory is owned by another allocator or
arena, or they cannot afford the synchronisation of cudaMalloc/cudaFree).
This test calls it through the C ABI twice in a row on one stream - the
second call reuses the fixed scratch left by the first - and compares every
output with sw_plan_create + sw_plan_execute on the same inputs.  The path is
exact integer arithmetic, so the comparison is bit for bit (tolerance 0).
The batch includes queries longer than one row strip, so the strip-boundary
scratch is exercised, and pairs beyond the scaled score bound.

It lives in a file of its own that pytest collects last and does not depend
on any other test having run.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _batch():
    """DNA pairs of the 1,000-pair workload plus long queries (several strips)."""
    base = wl.gen_config(0, n_pairs=600)
    rng = np.random.default_rng(4242)
    qs = [base.pair(i)[0] for i in range(base.n_pairs)]
    rs = [base.pair(i)[1] for i in range(base.n_pairs)]
    for n, m in [(700, 900), (1500, 400), (1025, 1025), (2000, 3000), (0, 50), (40, 0)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m) // 2
        if k:
            r[:k] = q[:k]
        qs.append(q)
        rs.append(r)
    return wl.make_batch("static-mix", qs, rs, base.matrix, base.gap_open, base.gap_extend)


def test_static_entry_matches_planned_path(gpu_lib):
    import torch
    swgb = gpu_lib
    b = _batch()
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    stream = torch.cuda.Stream(device=dev)

    ctx = swgb.sw_ctx_create(0)
    plan = swgb.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend)
    ref = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device=dev)
    swgb.sw_plan_execute(plan, q, r, ref, stream)
    stream.synchronize()
    expect = ref.cpu().numpy()
    swgb.sw_plan_destroy(plan)
    swgb.sw_ctx_destroy(ctx)

    for call in range(2):
        out = torch.full((5, b.n_pairs), -7 - call, dtype=torch.int32, device=dev)
        swgb.sw_align_batch_static(q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                                   b.gap_extend, out, stream)
        stream.synchronize()
        got = out.cpu().numpy()
        bad = np.flatnonzero(np.any(got != expect, axis=0))
        assert len(bad) == 0, (f"call {call}: {len(bad)} pairs differ, first {int(bad[0])}: "
                               f"{got[:, bad[0]].tolist()} vs {expect[:, bad[0]].tolist()}")
        # no kernel of the call found its reverse pass inconsistent
        assert swgb.sw_static_status(stream) == 0


def _long_pairs(seed, shapes):
    rng = np.random.default_rng(seed)
    qs, rs = [], []
    for n, m in shapes:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m) // 3
        if k:
            off = int(rng.integers(0, m - k + 1))
            r[off:off + k] = q[n - k:]
        qs.append(q)
        rs.append(r)
    return wl.make_batch(f"static-long-{seed}", qs, rs, wl.dna_matrix(), -6, -1)


def test_static_entry_large_then_small_batch(gpu_lib):
    """A large batch of long pairs, then a smaller batch of other long pairs:
    the second call must not read the strip-boundary words or tables that
    the first left in the shared array (each call writes what it reads)."""
    import torch
    swgb = gpu_lib
    dev = torch.device("cuda", 0)
    big = _long_pairs(71, [(int(n), int(m)) for n, m in
                           np.random.default_rng(5).integers(200, 3000, size=(300, 2))])
    small = _long_pairs(72, [(2500, 1800), (900, 2900), (1700, 1700), (3000, 600), (40, 2000)])
    ctx = swgb.sw_ctx_create(0)
    stream = torch.cuda.Stream(device=dev)
    try:
        for b in (big, small, big, small):
            q = torch.from_numpy(b.q_seqs).to(dev)
            r = torch.from_numpy(b.r_seqs).to(dev)
            plan = swgb.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                       b.gap_extend)
            ref = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device=dev)
            swgb.sw_plan_execute(plan, q, r, ref, stream)
            stream.synchronize()
            swgb.sw_plan_destroy(plan)
            out = torch.full((5, b.n_pairs), -3, dtype=torch.int32, device=dev)
            swgb.sw_align_batch_static(q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                                       b.gap_extend, out, stream)
            stream.synchronize()
            assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy()), b.name
            assert swgb.sw_static_status(stream) == 0
    finally:
        swgb.sw_ctx_destroy(ctx)


def test_static_entry_refuses_stream_capture(gpu_lib):
    """The call copies its tables from host memory it frees on return, so
    it refuses a capturing stream before enqueueing anything."""
    import torch
    swgb = gpu_lib
    dev = torch.device("cuda", 0)
    b = wl.gen_config(0, n_pairs=16)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    out = torch.zeros((5, b.n_pairs), dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    caught = None
    with torch.cuda.graph(g, stream=stream):
        try:
            swgb.sw_align_batch_static(q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                                       b.gap_extend, out, stream)
        except swgb.SwError as e:
            caught = e
        out.add_(0)  # something to capture
    assert caught is not None and caught.code == swgb.SW_EINVAL


def test_static_entry_matches_on_wide_scores(gpu_lib):
    """Pairs beyond the scaled bound take the plain kernel inside the same call."""
    import torch
    swgb = gpu_lib
    rng = np.random.default_rng(99)
    mat = np.full((4, 4), -90, np.int8)
    np.fill_diagonal(mat, 120)
    qs, rs = [], []
    for n, m in [(300, 400), (60, 80), (1200, 900)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        r[:n // 2] = q[:n // 2]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("static-wide", qs, rs, mat, -200, -30)
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    ctx = swgb.sw_ctx_create(0)
    plan = swgb.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend)
    ref = torch.zeros((5, b.n_pairs), dtype=torch.int32, device=dev)
    swgb.sw_plan_execute(plan, q, r, ref)
    torch.cuda.synchronize()
    swgb.sw_plan_destroy(plan)
    swgb.sw_ctx_destroy(ctx)
    for _ in range(2):
        out = torch.full((5, b.n_pairs), -5, dtype=torch.int32, device=dev)
        swgb.sw_align_batch_static(q, b.q_offsets, r, b.r_offsets, b.matrix, b.gap_open,
                                   b.gap_extend, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
        assert swgb.sw_static_status() == 0


def test_static_entry_rejects_oversize_batches(gpu_lib):
    import torch
    swgb = gpu_lib
    dev = torch.device("cuda", 0)
    out = torch.zeros((5, 1), dtype=torch.int32, device=dev)
    seq = torch.zeros(16, dtype=torch.uint8, device=dev)
    n = swgb.SW_STATIC_MAX_PAIRS + 1
    offs = np.zeros(n + 1, np.int64)
    with pytest.raises(swgb.SwError) as e:
        swgb.sw_align_batch_static(seq, offs, seq, offs, wl.dna_matrix(), -6, -1, out)
    assert e.value.code == swgb.SW_ERANGE and "split the batch" in str(e.value)
    # 70 pairs with queries longer than any row strip and 65,000-residue
    # references need about 70 x 2 x 65,000 boundary words, above the fixed
    # scratch
    k = 70
    qo = np.arange(k + 1, dtype=np.int64) * 2000
    ro = np.arange(k + 1, dtype=np.int64) * 65000
    qs = torch.zeros(int(qo[-1]), dtype=torch.uint8, device=dev)
    rs = torch.zeros(int(ro[-1]), dtype=torch.uint8, device=dev)
    assert 2 * 65000 * k > swgb.SW_STATIC_MAX_BOUNDARY_WORDS
    with pytest.raises(swgb.SwError) as e:
        swgb.sw_align_batch_static(qs, qo, rs, ro, wl.dna_matrix(), -6, -1,
                                   torch.zeros((5, k), dtype=torch.int32, device=dev))
    assert e.value.code == swgb.SW_ERANGE and "boundary words" in str(e.value)
