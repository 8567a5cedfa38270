"""Measured autotuner: candidates timed on the GPU, choice cached as JSON.

Whatever tuning wins, results stay bit-exact: tuning changes only how pairs
are spread over lane groups, never the arithmetic of a pair.
"""
import json

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def test_autotune_cache_miss_then_hit(gpu_lib, tmp_path):
    import torch
    swgb = gpu_lib
    b = wl.gen_config(3, n_pairs=6000)
    dev = torch.device("cuda:0")
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    out = torch.empty((5, b.n_pairs), dtype=torch.int32, device=dev)
    ctx = swgb.sw_ctx_create(0)
    cache = tmp_path / "tune.json"
    try:
        first = swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                                 q, r, out, cache_path=str(cache))
        torch.cuda.synchronize()
        assert cache.exists()
        doc = json.loads(cache.read_text())
        assert len(doc["entries"]) == 1
        assert doc["entries"][0]["narrow_log2g"] == first["narrow_log2g"]
        assert first["ms"] > 0
        # the candidates' runs left exact results in out
        idx = np.arange(0, b.n_pairs, 13)
        got = out.cpu().numpy().T
        assert np.array_equal(got[idx], oracle.align_workload(b, idx=idx))

        # a second call with the same kind of batch reads the cache
        ctx2 = swgb.sw_ctx_create(0)
        try:
            out.zero_()
            second = swgb.sw_autotune(ctx2, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                      b.gap_extend, q, r, out, cache_path=str(cache))
            assert second == first
            assert not out.any().item()  # nothing ran
            # a plan made after tuning uses the cached choice and stays exact
            a = swgb.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                             b.gap_extend, mode=swgb.SW_MODE_BATCHED, ctx=ctx2)
            a.run()
            res = a.results()
            a.close()
            assert np.array_equal(res[idx], oracle.align_workload(b, idx=idx))
        finally:
            swgb.sw_ctx_destroy(ctx2)

        # another batch gets its own entry
        b2 = wl.gen_config(1, n_pairs=3000)
        q2 = torch.from_numpy(b2.q_seqs).to(dev)
        r2 = torch.from_numpy(b2.r_seqs).to(dev)
        out2 = torch.empty((5, b2.n_pairs), dtype=torch.int32, device=dev)
        swgb.sw_autotune(ctx, b2.q_offsets, b2.r_offsets, b2.matrix, b2.gap_open, b2.gap_extend,
                         q2, r2, out2, cache_path=str(cache))
        doc = json.loads(cache.read_text())
        assert len(doc["entries"]) == 2
        assert len({e["key"] for e in doc["entries"]}) == 2
    finally:
        swgb.sw_ctx_destroy(ctx)


def test_autotune_with_plan_flags(gpu_lib, tmp_path):
    """sw_autotune_ex plans its candidates with the caller's ENDS_ONLY /
    NO_S16X2 bits: each flag set gets its own cache entry, and the ends-only
    candidates leave exact score/end outputs (no start outputs written)."""
    import torch
    swgb = gpu_lib
    b = wl.gen_config(1, n_pairs=4000)
    dev = torch.device("cuda:0")
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    out = torch.full((5, b.n_pairs), -7, dtype=torch.int32, device=dev)
    ctx = swgb.sw_ctx_create(0)
    cache = tmp_path / "tune.json"
    idx = np.arange(0, b.n_pairs, 17)
    expect = oracle.align_workload(b, idx=idx)
    try:
        swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                         q, r, out, cache_path=str(cache), flags=swgb.SW_PLAN_ENDS_ONLY)
        got = out.cpu().numpy().T
        assert np.array_equal(got[idx, :3], expect[:, :3])
        assert np.all(got[:, 3:] == -7)
        swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                         q, r, out, cache_path=str(cache), flags=swgb.SW_PLAN_NO_S16X2)
        swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                         q, r, out, cache_path=str(cache))
        assert np.array_equal(out.cpu().numpy().T[idx], expect)
        doc = json.loads(cache.read_text())
        assert len(doc["entries"]) == 3
        assert len({e["key"] for e in doc["entries"]}) == 3
    finally:
        swgb.sw_ctx_destroy(ctx)


@pytest.mark.parametrize("arith,rows,blocks", [(0, 16, 0), (1, 16, 0), (1, 32, 0), (-1, 32, 0),
                                               (-1, 16, 2), (0, 16, 1)])
def test_kernel_forms_exact(gpu_lib, arith, rows, blocks):
    """Each kernel form the autotuner chooses between - the packed 16-bit
    form with 16 or 32 rows per lane, and the scaled int32 form, with as many
    resident blocks per SM as fit or fewer - gives the oracle's results on a
    batch that spans one-strip, multi-strip and long-cap pairs."""
    import torch
    swgb = gpu_lib
    b = wl.gen_config(1, n_pairs=1500)
    ctx = swgb.sw_ctx_create(0)
    try:
        swgb.sw_ctx_set_form(ctx, arith, rows, blocks)
        t = swgb.sw_ctx_get_tuning(ctx)
        assert t["rows"] == rows and t["blocks_per_sm"] == blocks
        a = swgb.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                         b.gap_extend, mode=swgb.SW_MODE_BATCHED, ctx=ctx)
        info = swgb.sw_plan_info(a.plan)
        assert info["arith"] == ("s32" if arith == 0 else "s16x2")
        assert info["rows"] == (16 if arith == 0 else rows)
        a.run()
        res = a.results()
        a.close()
        idx = np.arange(0, b.n_pairs, 7)
        assert np.array_equal(res[idx], oracle.align_workload(b, idx=idx))
    finally:
        swgb.sw_ctx_destroy(ctx)


def test_autotune_records_form(gpu_lib, tmp_path):
    """The autotuner's choice includes the kernel form; a cache hit restores it."""
    import torch
    swgb = gpu_lib
    b = wl.gen_config(1, n_pairs=2000)
    dev = torch.device("cuda:0")
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    out = torch.empty((5, b.n_pairs), dtype=torch.int32, device=dev)
    cache = tmp_path / "tune.json"
    ctx = swgb.sw_ctx_create(0)
    ctx2 = swgb.sw_ctx_create(0)
    try:
        first = swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                 b.gap_extend, q, r, out, cache_path=str(cache))
        assert first["arith"] in ("auto", "s32", "s16x2") and first["rows"] in (16, 32)
        e = json.loads(cache.read_text())["entries"][0]
        assert {e["arith"], e["rows"]} <= {-1, 0, 1, 16, 32} and e["blocks_per_sm"] in (0, 2)
        swgb.sw_ctx_set_form(ctx2, 0, 16)
        second = swgb.sw_autotune(ctx2, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                  b.gap_extend, q, r, out, cache_path=str(cache))
        assert second == first
        assert swgb.sw_ctx_get_tuning(ctx2) == swgb.sw_ctx_get_tuning(ctx)
    finally:
        swgb.sw_ctx_destroy(ctx)
        swgb.sw_ctx_destroy(ctx2)


def test_damaged_cache_entry_is_measured_again(gpu_lib, tmp_path):
    """A cache entry the context rejects (here a lane-group width of 2^99,
    as a torn write could leave) counts as a miss: the batch is measured,
    the results stay exact, and the file keeps one valid entry for it.
    Processes tuning at once write through temporary files of their own,
    so no other file is left beside the cache."""
    import torch
    swgb = gpu_lib
    b = wl.gen_config(1, n_pairs=2000)
    dev = torch.device("cuda:0")
    q = torch.from_numpy(b.q_seqs).to(dev)
    r = torch.from_numpy(b.r_seqs).to(dev)
    out = torch.empty((5, b.n_pairs), dtype=torch.int32, device=dev)
    ctx = swgb.sw_ctx_create(0)
    cache = tmp_path / "tune.json"
    try:
        swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                         q, r, out, cache_path=str(cache))
        text = cache.read_text()
        doc = json.loads(text)
        key = doc["entries"][0]["key"]
        bad = text.replace(f'"narrow_log2g": {doc["entries"][0]["narrow_log2g"]},',
                           '"narrow_log2g": 99,')
        assert bad != text
        cache.write_text(bad)
        out.zero_()
        again = swgb.sw_autotune(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open,
                                 b.gap_extend, q, r, out, cache_path=str(cache))
        assert -1 <= again["narrow_log2g"] <= 5 and again["ms"] > 0
        torch.cuda.synchronize()
        idx = np.arange(0, b.n_pairs, 7)
        assert np.array_equal(out.cpu().numpy().T[idx], oracle.align_workload(b, idx=idx))
        doc = json.loads(cache.read_text())
        mine = [e for e in doc["entries"] if e["key"] == key]
        assert len(mine) == 1 and -1 <= mine[0]["narrow_log2g"] <= 5
        assert sorted(p.name for p in tmp_path.iterdir()) == ["tune.json"]
    finally:
        swgb.sw_ctx_destroy(ctx)
