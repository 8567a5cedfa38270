"""Multi-GPU sharding of a batch: pairs are independent, so a batch splits
across ranks with no exchange on the data path.

``lpt_partition`` assigns pairs to ranks by greedy longest-processing-time
over the cell count n*m (largest pair first, each to the least-loaded rank;
ties to the lower rank), so every rank gets about the same DP work.
``shard_batch`` cuts a rank's pairs out of the CSR arrays.  After each rank
has aligned its shard on its own GPU, ``gather_results`` brings the (n, 5)
results to every rank in the batch's order with one all-gather of 20 bytes
per pair (any torch.distributed backend: NCCL on GPUs, gloo on CPU).

Host-side logic only; it launches nothing on a GPU.
"""
from __future__ import annotations

import heapq

import numpy as np


def pair_costs(q_offsets, r_offsets) -> np.ndarray:
    """DP cells n*m of each pair (int64)."""
    q = np.diff(np.asarray(q_offsets, dtype=np.int64))
    r = np.diff(np.asarray(r_offsets, dtype=np.int64))
    return q * r


def lpt_partition(costs, world: int) -> list[np.ndarray]:
    """Indices of the pairs each rank takes, each list in ascending order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.int64)
    order = np.lexsort((np.arange(len(costs)), -costs))  # largest first, then index
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(i))
        heapq.heappush(heap, (load + int(costs[i]), r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_batch(q_seqs, q_offsets, r_seqs, r_offsets, idx):
    """(q_seqs, q_offsets, r_seqs, r_offsets) of the pairs idx, repacked."""
    q_offsets = np.asarray(q_offsets, dtype=np.int64)
    r_offsets = np.asarray(r_offsets, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)

    def cut(seqs, off):
        lens = off[idx + 1] - off[idx]
        new_off = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(lens, out=new_off[1:])
        out = np.empty(int(new_off[-1]), dtype=np.uint8)
        for k, i in enumerate(idx):
            out[new_off[k]:new_off[k + 1]] = seqs[off[i]:off[i + 1]]
        return out, new_off

    q, qo = cut(np.asarray(q_seqs, dtype=np.uint8), q_offsets)
    r, ro = cut(np.asarray(r_seqs, dtype=np.uint8), r_offsets)
    return q, qo, r, ro


def gather_results(local_idx, local_res, n_total: int, group=None, device=None) -> np.ndarray:
    """(n_total, 5) int32 results on every rank from each rank's (idx, res)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    idx = torch.as_tensor(np.asarray(local_idx, dtype=np.int64), device=device)
    res = torch.as_tensor(np.asarray(local_res, dtype=np.int32).reshape(-1, 5), device=device)
    counts = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([len(idx)], dtype=torch.int64, device=device), group=group)
    top = int(max(int(c.item()) for c in counts))
    pad_idx = torch.full((top,), -1, dtype=torch.int64, device=device)
    pad_res = torch.zeros((top, 5), dtype=torch.int32, device=device)
    pad_idx[:len(idx)] = idx
    pad_res[:len(idx)] = res
    all_idx = [torch.empty_like(pad_idx) for _ in range(world)]
    all_res = [torch.empty_like(pad_res) for _ in range(world)]
    dist.all_gather(all_idx, pad_idx, group=group)
    dist.all_gather(all_res, pad_res, group=group)
    out = np.full((n_total, 5), np.iinfo(np.int32).min, dtype=np.int32)
    for gi, gr in zip(all_idx, all_res):
        gi = gi.cpu().numpy()
        keep = gi >= 0
        out[gi[keep]] = gr.cpu().numpy()[keep]
    if np.any(out[:, 0] == np.iinfo(np.int32).min):
        raise RuntimeError("gather_results: some pairs were on no rank")
    return out
