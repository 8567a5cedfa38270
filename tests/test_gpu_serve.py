"""Serving loop: continuous batching gives the same results alone and in a mix.

Requests (DNA pairs drawn like the 100k-pair workload, protein pairs like the
20k-pair workload) are submitted one at a time and waited for (alone), then
all at once so that they overlap on the GPU (in the mix).  Every result must
be identical between the two, and equal to the CPU oracle (tolerance 0: the
path is exact integer arithmetic).
"""
import threading
import time

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu


def _requests(k=24, seed=5):
    reqs = wl.serving_requests(k, rate_per_s=1000.0, seed=seed, max_pairs=300)
    return [r.batch for r in reqs]


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


def test_alone_equals_mix_equals_oracle(gpu_lib, ctx):
    swgb = gpu_lib
    batches = _requests()
    srv = swgb.sw_server_create(ctx, 1 << 30, streams=6, staging_bytes=1 << 28)
    try:
        alone = []
        for b in batches:
            rid = swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets,
                                        b.matrix, b.gap_open, b.gap_extend)
            alone.append(swgb.sw_server_wait(srv, rid, b.n_pairs))
        ids = [swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                     b.gap_open, b.gap_extend) for b in batches]
        seen_overlap = 0
        for _ in range(200):
            st = swgb.sw_server_stats(srv)
            seen_overlap = max(seen_overlap, st["in_flight"])
            if st["completed"] >= 2 * len(batches):
                break
            time.sleep(0.001)
        mix = [swgb.sw_server_wait(srv, rid, b.n_pairs) for rid, b in zip(ids, batches)]
    finally:
        swgb.sw_server_destroy(srv)
    for i, b in enumerate(batches):
        assert np.array_equal(alone[i], mix[i]), f"request {i} differs alone vs mix"
        assert np.array_equal(mix[i], oracle.align_workload(b)), f"request {i} differs from oracle"
    assert seen_overlap >= 1


def test_budget_limits_admission_and_rejects_oversize(gpu_lib, ctx):
    swgb = gpu_lib
    batches = _requests(12, seed=9)
    # a tight budget: requests must wait for memory to free up, yet all finish
    need = max(int(b.q_seqs.nbytes + b.r_seqs.nbytes) for b in batches)
    budget = max(1 << 20, 3 * need + (4 << 20))
    srv = swgb.sw_server_create(ctx, budget, streams=8, staging_bytes=1 << 26)
    try:
        ids = [swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                     b.gap_open, b.gap_extend) for b in batches]
        outs = [swgb.sw_server_wait(srv, rid, b.n_pairs) for rid, b in zip(ids, batches)]
        st = swgb.sw_server_stats(srv)
        assert st["device_bytes_peak"] <= budget
        for b, o in zip(batches, outs):
            assert np.array_equal(o, oracle.align_workload(b))
        big = wl.gen_config(1, n_pairs=20000)
        with pytest.raises(swgb.SwError) as e:
            swgb.sw_server_submit(srv, big.q_seqs, big.q_offsets, big.r_seqs, big.r_offsets,
                                  big.matrix, big.gap_open, big.gap_extend)
        assert e.value.code == swgb.SW_EBUDGET
    finally:
        swgb.sw_server_destroy(srv)


def test_wait_is_bounded(gpu_lib, ctx):
    swgb = gpu_lib
    b = wl.gen_config(1, n_pairs=3000)
    srv = swgb.sw_server_create(ctx, 1 << 30, streams=2)
    try:
        rid = swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                    b.gap_open, b.gap_extend)
        # a zero timeout either finds the request done or says SW_ETIMEOUT;
        # after a timeout the request is still there to wait for
        try:
            early = swgb.sw_server_wait(srv, rid, b.n_pairs, timeout_ms=0)
        except swgb.SwError as e:
            assert e.code == swgb.SW_ETIMEOUT
            early = None
        if early is None:
            out = swgb.sw_server_wait(srv, rid, b.n_pairs, timeout_ms=60000)
            idx = np.arange(0, b.n_pairs, 97)
            assert np.array_equal(out[idx], oracle.align_workload(b, idx=idx))
        # a finished request's results are handed out once
        with pytest.raises(swgb.SwError):
            swgb.sw_server_wait(srv, rid, b.n_pairs, timeout_ms=0)
    finally:
        swgb.sw_server_destroy(srv)


def test_concurrent_clients(gpu_lib, ctx):
    """Several host threads submit and wait at once."""
    swgb = gpu_lib
    batches = _requests(16, seed=21)
    srv = swgb.sw_server_create(ctx, 1 << 30, streams=4)
    results = [None] * len(batches)
    errors = []

    def client(lo, hi):
        try:
            for i in range(lo, hi):
                b = batches[i]
                rid = swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets,
                                            b.matrix, b.gap_open, b.gap_extend)
                results[i] = swgb.sw_server_wait(srv, rid, b.n_pairs)
        except Exception as e:  # pragma: no cover - reported below
            errors.append(e)

    th = [threading.Thread(target=client, args=(4 * k, 4 * k + 4)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    swgb.sw_server_destroy(srv)
    assert not errors, errors
    for b, o in zip(batches, results):
        assert np.array_equal(o, oracle.align_workload(b))


def test_queued_requests_merge_into_one_launch(gpu_lib, ctx):
    """With one stream slot busy on a large request, the requests queued
    behind it run as merged launches: one per scoring, DNA and protein kept
    apart, results still exact."""
    swgb = gpu_lib
    big = wl.gen_config(1, n_pairs=60000)
    small = _requests(12, seed=33)
    srv = swgb.sw_server_create(ctx, 4 << 30, streams=1, staging_bytes=1 << 28)
    try:
        rid_big = swgb.sw_server_submit(srv, big.q_seqs, big.q_offsets, big.r_seqs,
                                        big.r_offsets, big.matrix, big.gap_open, big.gap_extend)
        ids = [swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                     b.gap_open, b.gap_extend) for b in small]
        outs = [swgb.sw_server_wait(srv, rid, b.n_pairs) for rid, b in zip(ids, small)]
        out_big = swgb.sw_server_wait(srv, rid_big, big.n_pairs)
        launches = swgb.sw_server_launches(srv)["launches"]
    finally:
        swgb.sw_server_destroy(srv)
    kinds = {b.name.split("-")[-1] for b in small}
    # the large request alone, then at most a few merged launches
    assert launches <= 1 + 2 * len(kinds), launches
    assert launches < 1 + len(small)
    for b, o in zip(small, outs):
        assert np.array_equal(o, oracle.align_workload(b))
    idx = np.arange(0, big.n_pairs, 211)
    assert np.array_equal(out_big[idx], oracle.align_workload(big, idx=idx))


def test_resident_pools_equal_oracle(gpu_lib, ctx):
    """Sequences uploaded once as resident pools; requests name pair ranges
    (some overlapping, some at the pools' ends), mixed with staged requests,
    from several client threads: every result equals the oracle's."""
    swgb = gpu_lib
    dna = wl.gen_config(1, n_pairs=6000)
    prot = wl.gen_config(2, n_pairs=2000)
    exp = {"dna": oracle.align_workload(dna), "protein": oracle.align_workload(prot)}
    srv = swgb.sw_server_create(ctx, 2 << 30, streams=6, staging_bytes=1 << 28)
    rng = np.random.default_rng(77)
    jobs = []
    for k in range(60):
        kind = "dna" if k % 2 == 0 else "protein"
        total = dna.n_pairs if kind == "dna" else prot.n_pairs
        n = int(min(total, max(1, np.exp(rng.uniform(0, np.log(1500))))))
        first = int(rng.integers(0, total - n + 1)) if k % 7 else total - n
        jobs.append((kind, first, n))
    staged = _requests(8, seed=88)
    results, errors = {}, []
    try:
        pid = {"dna": swgb.sw_server_add_pool(srv, dna.q_seqs, dna.q_offsets, dna.r_seqs,
                                              dna.r_offsets, dna.matrix, dna.gap_open,
                                              dna.gap_extend),
               "protein": swgb.sw_server_add_pool(srv, prot.q_seqs, prot.q_offsets, prot.r_seqs,
                                                  prot.r_offsets, prot.matrix, prot.gap_open,
                                                  prot.gap_extend)}

        def client(c):
            try:
                mine = []
                for k in range(c, len(jobs), 4):
                    kind, first, n = jobs[k]
                    mine.append((k, swgb.sw_server_submit_pool(srv, pid[kind], first, n), n))
                for k in range(c, len(staged), 4):
                    b = staged[k]
                    mine.append((-1 - k, swgb.sw_server_submit(
                        srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                        b.gap_open, b.gap_extend), b.n_pairs))
                for k, rid, n in mine:
                    results[k] = swgb.sw_server_wait(srv, rid, n)
            except Exception as e:  # pragma: no cover - reported below
                errors.append(e)

        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert swgb.sw_ctx_status(ctx) == 0
    finally:
        swgb.sw_server_destroy(srv)
    assert not errors, errors
    for k, (kind, first, n) in enumerate(jobs):
        assert np.array_equal(results[k], exp[kind][first:first + n]), (k, kind, first, n)
    for k, b in enumerate(staged):
        assert np.array_equal(results[-1 - k], oracle.align_workload(b))


def test_pool_errors(gpu_lib, ctx):
    swgb = gpu_lib
    b = wl.gen_config(0, n_pairs=50)
    srv = swgb.sw_server_create(ctx, 8 << 20, streams=2, staging_bytes=1 << 24)
    try:
        pid = swgb.sw_server_add_pool(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                      b.gap_open, b.gap_extend)
        with pytest.raises(swgb.SwError) as e:
            swgb.sw_server_submit_pool(srv, pid, 40, 20)
        assert e.value.code == swgb.SW_ERANGE
        with pytest.raises(swgb.SwError) as e:
            swgb.sw_server_submit_pool(srv, pid + 5, 0, 1)
        assert e.value.code == swgb.SW_EINVAL
        big = wl.gen_config(1, n_pairs=20000)  # 16 MB of residues: above the budget
        with pytest.raises(swgb.SwError) as e:
            swgb.sw_server_add_pool(srv, big.q_seqs, big.q_offsets, big.r_seqs, big.r_offsets,
                                    big.matrix, big.gap_open, big.gap_extend)
        assert e.value.code == swgb.SW_EBUDGET
        rid = swgb.sw_server_submit_pool(srv, pid, 10, 30)
        out = swgb.sw_server_wait(srv, rid, 30)
        assert np.array_equal(out, oracle.align_workload(b.slice(10, 40)))
    finally:
        swgb.sw_server_destroy(srv)
