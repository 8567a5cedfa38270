"""GPU parity: every output of the CUDA path equals the CPU oracle, bit for bit.

The path is exact integer max-plus arithmetic, so the tolerance is zero on
all five outputs (score, qend, rend, qstart, rstart).  Inputs come from the
seeded generators in `workloads`; expected values from `oracle` only.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def run_lib(swgb, ctx, b, mode=None, flags=0, tuning=None):
    if tuning is not None:
        swgb.sw_ctx_set_tuning(ctx, *tuning)
    try:
        al = swgb.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                          b.gap_extend, mode=swgb.SW_MODE_AUTO if mode is None else mode,
                          flags=flags, ctx=ctx)
        al.run()
        got = al.results()
        info = al.info()
        al.close()
    finally:
        if tuning is not None:
            swgb.sw_ctx_set_tuning(ctx, -1, 0.5)
    assert swgb.sw_ctx_status(ctx) == 0
    return got, info


def assert_same(got, expect, name):
    bad = np.flatnonzero(np.any(got != expect, axis=1))
    if len(bad):
        i = int(bad[0])
        raise AssertionError(f"{name}: {len(bad)} pairs differ; first pair {i}: "
                             f"got {got[i].tolist()} expected {expect[i].tolist()}")


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_config0_full(gpu_lib, ctx, mode):
    b = wl.gen_config(0)
    expect = oracle.align_workload(b)
    m = gpu_lib.SW_MODE_BATCHED if mode == "batched" else gpu_lib.SW_MODE_PLAIN
    got, _ = run_lib(gpu_lib, ctx, b, mode=m)
    assert_same(got, expect, f"config0/{mode}")


@pytest.mark.parametrize("k", [1, 2, 3])
def test_full_configs_batched_graph(gpu_lib, ctx, k):
    """Workloads 1-3 at full size, in the launch form the benchmark times."""
    b = wl.gen_config(k)
    got, info = run_lib(gpu_lib, ctx, b, flags=gpu_lib.SW_PLAN_GRAPH)
    expect = oracle.align_workload(b)
    assert_same(got, expect, f"config{k}")
    assert info["plain_pairs"] == 0  # all pairs inside the scaled path's bound


def test_config1_plain_sampled(gpu_lib, ctx):
    """The plain one-block-per-pair form on the full 100k-pair batch, sampled."""
    b = wl.gen_config(1)
    got, _ = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_PLAIN)
    idx = np.random.default_rng(0).choice(b.n_pairs, 3000, replace=False)
    expect = oracle.align_workload(b, idx=idx)
    assert_same(got[idx], expect, "config1/plain sample")


EDGE = [0, 1, 2, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513,
        1023, 1024, 1025]


def edge_batch(kind, seed, lens_q, lens_r, plant=True):
    rng = np.random.default_rng(seed)
    A = 4 if kind == "dna" else 20
    qs, rs = [], []
    for n in lens_q:
        for m in lens_r:
            q = rng.integers(0, A, n).astype(np.uint8)
            r = rng.integers(0, A, m).astype(np.uint8)
            if plant and n and m and rng.random() < 0.5:
                k = min(n, m)
                off = int(rng.integers(0, m - k + 1))
                r[off:off + k] = q[:k]
            qs.append(q)
            rs.append(r)
    if kind == "dna":
        return wl.make_batch("edge-dna", qs, rs, wl.dna_matrix(), -6, -1)
    s, _ = wl.load_blosum62()
    return wl.make_batch("edge-protein", qs, rs, s.astype(np.int8), -11, -1)


# (the last two: pairs above the cap at the widest bulk widths, where no
# wider class is left)
TUNINGS = [(lg, 1e9) for lg in range(6)] + [(0, 0.05), (1, 0.3), (-1, 0.5), (4, 0.05), (5, 0.05)]


@pytest.mark.parametrize("tuning", TUNINGS, ids=[f"G{1 << t[0] if t[0] >= 0 else 'auto'}-cap{t[1]:g}"
                                                 for t in TUNINGS])
def test_edge_lengths_all_group_widths(gpu_lib, ctx, tuning):
    """Lengths around every tile edge, under every lane-group width.

    (lg, 1e9) puts every pair on groups of 2^lg lanes; a small cap fraction
    spreads the pairs over several width classes in one launch.
    """
    b = edge_batch("dna", 7 + tuning[0], EDGE, EDGE[::3])
    expect = oracle.align_workload(b)
    got, _ = run_lib(gpu_lib, ctx, b, tuning=tuning)
    assert_same(got, expect, f"edge dna tuning={tuning}")


def test_edge_lengths_protein(gpu_lib, ctx):
    b = edge_batch("protein", 5, EDGE[::2], EDGE[1::3])
    expect = oracle.align_workload(b)
    for tuning in ((5, 1e9), (0, 1e9), (-1, 0.5)):
        got, _ = run_lib(gpu_lib, ctx, b, tuning=tuning)
        assert_same(got, expect, f"edge protein tuning={tuning}")
    got, _ = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_PLAIN)
    assert_same(got, expect, "edge protein plain")


def test_long_sequences_and_maximum_length(gpu_lib, ctx):
    """Long tail beyond the workloads, up to the documented maximum length."""
    rng = np.random.default_rng(23)
    qs, rs = [], []
    for n, m in [(4000, 65535), (65535, 300), (3000, 3000), (1, 65535), (65535, 1)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m, 2000)
        r[m - k:] = q[n - k:]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("long", qs, rs, wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(b)
    got, _ = run_lib(gpu_lib, ctx, b)
    assert_same(got, expect, "long batched")


@pytest.mark.parametrize("lg", [1, 5])
def test_batched_length_limit(gpu_lib, ctx, lg):
    """Sequences up to 65,471 residues take the batched kernel (its end key
    keeps the column in 16 bits on the pad columns a lane's last row computes
    before its first), one more takes the plain kernel; exact either side,
    with the start far from the end (a long reverse sweep) and with a best
    cell near the last column."""
    rng = np.random.default_rng(31 + lg)
    qs, rs = [], []
    for n, m in [(300, 65471), (300, 65472), (65471, 200), (65472, 200)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m, 150)
        r[m - k:] = q[:k]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("limit", qs, rs, wl.dna_matrix(), -6, -1)
    expect = oracle.align_workload(b)
    got, info = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_AUTO, tuning=(lg, 1e9))
    assert_same(got, expect, f"length limit G{1 << lg}")
    assert info["plain_pairs"] == 2


def test_wide_scores_use_plain_path(gpu_lib, ctx):
    """Scores beyond the scaled int32 key range go to the general int32 kernel."""
    rng = np.random.default_rng(29)
    mat = np.full((4, 4), -90, np.int8)
    np.fill_diagonal(mat, 120)
    qs, rs = [], []
    for n, m in [(300, 400), (1200, 1300), (50, 60), (2100, 2100)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        r[:n // 2] = q[:n // 2]
        qs.append(q)
        rs.append(r)
    b = wl.make_batch("wide", qs, rs, mat, -200, -30)
    expect = oracle.align_workload(b)
    got, info = run_lib(gpu_lib, ctx, b)
    assert info["plain_pairs"] == 3  # 50 x 60 stays under the bound
    assert_same(got, expect, "wide")
    assert expect[:, 0].max() > 32766


@pytest.mark.parametrize("go,ge", [(-1, -1), (0, 0), (-3, 0), (-16383, -1), (-20000, -5)])
def test_gap_settings(gpu_lib, ctx, go, ge):
    b = wl.gen_config(0, n_pairs=200)
    b = wl.make_batch("gaps", [b.pair(i)[0] for i in range(b.n_pairs)],
                      [b.pair(i)[1] for i in range(b.n_pairs)], b.matrix, go, ge)
    expect = oracle.align_workload(b)
    for mode in (gpu_lib.SW_MODE_BATCHED, gpu_lib.SW_MODE_PLAIN):
        got, _ = run_lib(gpu_lib, ctx, b, mode=mode)
        assert_same(got, expect, f"gaps {go},{ge} mode {mode}")


def test_asymmetric_matrix_and_small_alphabet(gpu_lib, ctx):
    rng = np.random.default_rng(31)
    mat = rng.integers(-5, 6, size=(3, 3)).astype(np.int8)
    mat[0, 0] = 5
    qs = [rng.integers(0, 3, int(rng.integers(0, 200))).astype(np.uint8) for _ in range(300)]
    rs = [rng.integers(0, 3, int(rng.integers(0, 400))).astype(np.uint8) for _ in range(300)]
    b = wl.make_batch("asym", qs, rs, mat, -4, -2)
    expect = oracle.align_workload(b)
    got, _ = run_lib(gpu_lib, ctx, b)
    assert_same(got, expect, "asym")


def test_largest_alphabet_with_wide_scores(gpu_lib, ctx):
    """32 residue codes with scores outside the int8 profile's range: the
    int32 profile of so large an alphabet does not fit in shared memory, so
    every pair takes the plain kernel, still exact."""
    rng = np.random.default_rng(37)
    mat = rng.integers(-100, 101, size=(32, 32)).astype(np.int8)
    np.fill_diagonal(mat, 100)
    qs = [rng.integers(0, 32, int(rng.integers(0, 120))).astype(np.uint8) for _ in range(200)]
    rs = [rng.integers(0, 32, int(rng.integers(0, 300))).astype(np.uint8) for _ in range(200)]
    b = wl.make_batch("a32", qs, rs, mat, -50, -5)
    expect = oracle.align_workload(b)
    got, info = run_lib(gpu_lib, ctx, b)
    assert_same(got, expect, "alphabet 32, wide scores")
    assert info["plain_pairs"] == b.n_pairs
    # the same alphabet with int8-range scores fits and takes the batched path
    mat8 = np.clip(mat, -20, 20).astype(np.int8)
    b8 = wl.make_batch("a32i8", qs, rs, mat8, -10, -2)
    got8, info8 = run_lib(gpu_lib, ctx, b8)
    assert_same(got8, oracle.align_workload(b8), "alphabet 32, int8 profile")
    assert info8["group_pairs"] > 0


def test_graph_replay_and_repeat(gpu_lib, ctx):
    import torch
    b = wl.gen_config(0, n_pairs=500)
    expect = oracle.align_workload(b)
    al = gpu_lib.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                         b.gap_extend, flags=gpu_lib.SW_PLAN_GRAPH, ctx=ctx)
    s = torch.cuda.Stream()
    for _ in range(3):
        al.out.fill_(-9)
        with torch.cuda.stream(s):
            al.run(stream=s)
        s.synchronize()
        assert_same(al.results(), expect, "graph replay")
    al.close()


def test_one_shot_device_offsets(gpu_lib):
    import torch
    b = wl.gen_config(2, n_pairs=300)
    expect = oracle.align_workload(b)
    dev = torch.device("cuda", 0)
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    qo = torch.from_numpy(b.q_offsets).to(dev)
    ro = torch.from_numpy(b.r_offsets).to(dev)
    out = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device=dev)
    gpu_lib.sw_align_batch(q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend, out)
    torch.cuda.synchronize()
    assert_same(out.T.cpu().numpy(), expect, "one-shot")


def test_self_alignment_closed_form_at_scale(gpu_lib, ctx):
    """S = 3L, ends (L-1, L-1), starts (0, 0) for DNA self-alignment."""
    rng = np.random.default_rng(37)
    lens = rng.integers(1, 3000, 400)
    qs = [rng.integers(0, 4, L).astype(np.uint8) for L in lens]
    b = wl.make_batch("self", qs, qs, wl.dna_matrix(), -6, -1)
    got, _ = run_lib(gpu_lib, ctx, b)
    L = lens.astype(np.int32)
    expect = np.stack([3 * L, L - 1, L - 1, np.zeros_like(L), np.zeros_like(L)], axis=1)
    assert_same(got, expect, "self")


def test_invalid_arguments_rejected(gpu_lib, ctx):
    b = wl.gen_config(0, n_pairs=4)
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, 0, -1)
    assert e.value.code == gpu_lib.SW_EINVAL
    bad = b.q_offsets.copy()
    bad[2] = bad[1] - 1
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_plan_create(ctx, bad, b.r_offsets, b.matrix, -6, -1)
    assert e.value.code == gpu_lib.SW_ERANGE
    big = np.array([0, 70000], np.int64)
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_plan_create(ctx, big, np.array([0, 5], np.int64), b.matrix, -6, -1)
    assert e.value.code == gpu_lib.SW_ERANGE


def test_check_residues(gpu_lib):
    import torch
    dev = torch.device("cuda", 0)
    s = torch.tensor([0, 1, 2, 3, 4, 7, 1, 0, 200], dtype=torch.uint8, device=dev)
    bad = torch.zeros(1, dtype=torch.int64, device=dev)
    gpu_lib.sw_check_residues(s, s.numel(), 4, bad)
    torch.cuda.synchronize()
    assert int(bad.item()) == 3


def _with_gaps(b, go, ge, matrix=None, name="regapped"):
    return wl.make_batch(name, [b.pair(i)[0] for i in range(b.n_pairs)],
                         [b.pair(i)[1] for i in range(b.n_pairs)],
                         b.matrix if matrix is None else matrix, go, ge)


@pytest.mark.parametrize("tuning", TUNINGS, ids=[f"G{1 << t[0] if t[0] >= 0 else 'auto'}-cap{t[1]:g}"
                                                 for t in TUNINGS])
def test_linear_gaps_take_the_linear_kernel(gpu_lib, ctx, tuning):
    """gap_open == gap_extend runs the instantiation without E and F; it must
    equal the Gotoh oracle (which keeps E and F) on DNA with the paper's
    Fig. 2 scoring (+2/-2, gap -1) and on protein with BLOSUM62 and gap -4,
    with lengths spanning several strips, under every lane-group width."""
    dna = _with_gaps(wl.gen_config(1, n_pairs=400), -1, -1,
                     matrix=wl.dna_matrix(2, -2), name="fig2-scoring")
    prot = _with_gaps(wl.gen_config(2, n_pairs=300), -4, -4, name="blosum-linear")
    for b in (dna, prot):
        expect = oracle.align_workload(b)
        got, info = run_lib(gpu_lib, ctx, b, mode=gpu_lib.SW_MODE_BATCHED, tuning=tuning)
        assert info["group_pairs"] == b.n_pairs
        assert_same(got, expect, f"{b.name} tuning {tuning}")


@pytest.mark.parametrize("k", [0, 2])
def test_ends_only_plans(gpu_lib, ctx, k):
    """SW_PLAN_ENDS_ONLY: score, qend, rend equal the oracle's; the start
    outputs are left untouched (batched, plain, graph and host-buffer forms)."""
    import torch
    b = wl.gen_config(k, n_pairs=600)
    expect = oracle.align_workload(b)
    for mode in (gpu_lib.SW_MODE_BATCHED, gpu_lib.SW_MODE_PLAIN):
        flags = gpu_lib.SW_PLAN_ENDS_ONLY | gpu_lib.SW_PLAN_GRAPH
        al = gpu_lib.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                             b.gap_extend, mode=mode, flags=flags, ctx=ctx)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            al.run(stream=s)
        s.synchronize()
        got = al.results()
        assert_same(got[:, :3], expect[:, :3], f"ends only, mode {mode}")
        assert np.all(got[:, 3:] == -7), "start outputs were written"
        qh = torch.from_numpy(b.q_seqs).pin_memory()
        rh = torch.from_numpy(b.r_seqs).pin_memory()
        oh = torch.full((5, b.n_pairs), -9, dtype=torch.int32).pin_memory()
        gpu_lib.sw_plan_execute_host(al.plan, qh, rh, oh, s)
        host = oh.numpy().T
        assert_same(host[:, :3], expect[:, :3], f"ends only, host buffers, mode {mode}")
        assert np.all(host[:, 3:] == -9)
        al.close()
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_host_buffer_execution_pinned_and_pageable(gpu_lib, ctx):
    """sw_plan_execute_host on page-locked inputs (read in place when the
    device reads host memory over a coherent link) and on pageable inputs
    (copied): the same outputs as the oracle either way, repeated runs too."""
    import torch
    b = wl.gen_config(1, n_pairs=3000)
    expect = oracle.align_workload(b)
    plan = gpu_lib.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                  b.gap_extend, gpu_lib.SW_MODE_BATCHED, gpu_lib.SW_PLAN_GRAPH)
    try:
        pinned = (torch.from_numpy(b.q_seqs).pin_memory(), torch.from_numpy(b.r_seqs).pin_memory())
        pageable = (torch.from_numpy(b.q_seqs.copy()), torch.from_numpy(b.r_seqs.copy()))
        for q, r in (pinned, pageable, pinned):
            out = torch.full((5, b.n_pairs), -9, dtype=torch.int32).pin_memory()
            for _ in range(2):
                gpu_lib.sw_plan_execute_host(plan, q, r, out)
            assert_same(out.numpy().T, expect, f"host buffers, pinned={q.is_pinned()}")
    finally:
        gpu_lib.sw_plan_destroy(plan)
    assert isinstance(gpu_lib.sw_ctx_host_in_place(ctx), bool)


def test_host_input_transport_switch(gpu_lib):
    """sw_ctx_set_host_in_place: page-locked inputs copied to the device
    (0) or read in place where the device can (1) give the same outputs, for
    the plan's host-buffer call and the one-shot call; the setting reads
    back, and never claims in-place reads a device cannot do."""
    import torch
    b = wl.gen_config(2, n_pairs=800)
    expect = oracle.align_workload(b)
    ctx = gpu_lib.sw_ctx_create(0)
    try:
        able = gpu_lib.sw_ctx_host_in_place(ctx)
        plan = gpu_lib.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                      b.gap_extend, gpu_lib.SW_MODE_BATCHED, gpu_lib.SW_PLAN_GRAPH)
        qh = torch.from_numpy(b.q_seqs).pin_memory()
        rh = torch.from_numpy(b.r_seqs).pin_memory()
        qoh = torch.from_numpy(b.q_offsets).pin_memory()
        roh = torch.from_numpy(b.r_offsets).pin_memory()
        try:
            for enable in (False, True, False):
                gpu_lib.sw_ctx_set_host_in_place(ctx, enable)
                assert gpu_lib.sw_ctx_host_in_place(ctx) == (enable and able)
                out = torch.full((5, b.n_pairs), -9, dtype=torch.int32).pin_memory()
                gpu_lib.sw_plan_execute_host(plan, qh, rh, out)
                assert_same(out.numpy().T, expect, f"host buffers, in place={enable}")
                if enable and able:
                    # (the one-shot call takes host buffers only when it reads
                    # them in place; otherwise its inputs must be on the device)
                    dout = torch.full((5, b.n_pairs), -9, dtype=torch.int32, device="cuda")
                    gpu_lib.sw_align_batch_ex(ctx, qh, qoh, rh, roh, b.matrix, b.gap_open,
                                              b.gap_extend, gpu_lib.SW_MODE_AUTO, dout)
                    torch.cuda.synchronize()
                    assert_same(dout.cpu().numpy().T, expect, "one-shot, inputs in place")
        finally:
            gpu_lib.sw_plan_destroy(plan)
        assert gpu_lib.load().sw_ctx_set_host_in_place(ctx, 2) == gpu_lib.SW_EINVAL
        assert gpu_lib.sw_ctx_host_in_place(ctx) is False
    finally:
        gpu_lib.sw_ctx_destroy(ctx)
