"""2-bit packed DNA input: the same results as one byte per residue."""
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


def test_unpack_round_trip(gpu_lib):
    import torch
    rng = np.random.default_rng(11)
    for n in (1, 2, 3, 4, 5, 4097, 100003):
        codes = rng.integers(0, 4, n).astype(np.uint8)
        packed = torch.from_numpy(gpu_lib.sw_pack_2bit(codes)).cuda()
        out = torch.full((n + 8,), 0xEE, dtype=torch.uint8, device="cuda")
        gpu_lib.sw_unpack_2bit(packed, n, out)
        got = out.cpu().numpy()
        assert np.array_equal(got[:n], codes)
        assert np.all(got[n:] == 0xEE), "wrote past the end"


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_packed_plans_equal_oracle(gpu_lib, ctx, mode):
    import torch
    b = wl.gen_config(1, n_pairs=2000)
    expect = oracle.align_workload(b)
    m = gpu_lib.SW_MODE_BATCHED if mode == "batched" else gpu_lib.SW_MODE_PLAIN
    qp = gpu_lib.sw_pack_2bit(b.q_seqs)
    rp = gpu_lib.sw_pack_2bit(b.r_seqs)
    flags = gpu_lib.SW_PLAN_PACKED_2BIT | gpu_lib.SW_PLAN_GRAPH
    plan = gpu_lib.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                  b.gap_extend, m, flags)
    try:
        q = torch.from_numpy(qp).cuda()
        r = torch.from_numpy(rp).cuda()
        out = torch.full((5, b.n_pairs), -7, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        for _ in range(2):  # graph capture, then replay
            with torch.cuda.stream(s):
                gpu_lib.sw_plan_execute(plan, q, r, out, s)
            s.synchronize()
            assert np.array_equal(out.T.cpu().numpy(), expect)
        # host buffers: a quarter of the bytes cross to the device
        qh = torch.from_numpy(qp).pin_memory()
        rh = torch.from_numpy(rp).pin_memory()
        oh = torch.zeros((5, b.n_pairs), dtype=torch.int32).pin_memory()
        gpu_lib.sw_plan_execute_host(plan, qh, rh, oh, s)
        assert np.array_equal(oh.numpy().T, expect)
        assert gpu_lib.sw_plan_info(plan)["launches"] == 3
    finally:
        gpu_lib.sw_plan_destroy(plan)
    assert gpu_lib.sw_ctx_status(ctx) == 0


def test_packed_needs_small_alphabet(gpu_lib, ctx):
    b = wl.gen_config(2, n_pairs=10)
    with pytest.raises(gpu_lib.SwError) as e:
        gpu_lib.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                               b.gap_extend, gpu_lib.SW_MODE_AUTO, gpu_lib.SW_PLAN_PACKED_2BIT)
    assert e.value.code == gpu_lib.SW_EINVAL
