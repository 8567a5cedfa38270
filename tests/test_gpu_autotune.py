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
