"""Multi-rank path on the CPU: LPT sharding of a batch across ranks, each
rank aligning its shard (here with the CPU oracle, as no GPU is present),
and the all-gather of the results, run as world-size-2 gloo process groups.
The gathered results must equal a single-process run over the whole batch.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workloads as wl
from paper_2208_12350_gb300 import shard


def test_lpt_partition_balances_and_covers():
    b = wl.gen_config(3, n_pairs=5000)
    costs = shard.pair_costs(b.q_offsets, b.r_offsets)
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(b.n_pairs))
        loads = np.array([costs[p].sum() for p in parts])
        # LPT bound: no rank exceeds the mean by more than the largest pair
        assert loads.max() - loads.mean() <= costs.max()
    # deterministic
    a = shard.lpt_partition(costs, 4)
    c = shard.lpt_partition(costs, 4)
    assert all(np.array_equal(x, y) for x, y in zip(a, c))


def test_shard_batch_repacks_pairs():
    b = wl.gen_config(0, n_pairs=50)
    idx = np.array([3, 7, 8, 40])
    q, qo, r, ro = shard.shard_batch(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, idx)
    for k, i in enumerate(idx):
        assert np.array_equal(q[qo[k]:qo[k + 1]], b.pair(i)[0])
        assert np.array_equal(r[ro[k]:ro[k + 1]], b.pair(i)[1])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = wl.gen_config(0, n_pairs=300)
        parts = shard.lpt_partition(shard.pair_costs(b.q_offsets, b.r_offsets), world)
        mine = parts[rank]
        q, qo, r, ro = shard.shard_batch(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, mine)
        res = oracle.align_batch(q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend, threads=1)
        full = shard.gather_results(mine, res, b.n_pairs)
        if rank == 0:
            np.save(out_path, full)
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shard_and_gather(tmp_path):
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    b = wl.gen_config(0, n_pairs=300)
    assert np.array_equal(got, oracle.align_workload(b))
