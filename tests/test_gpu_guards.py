"""Guard canaries: no kernel writes outside its buffers, at any size.

Out-of-bounds writes often show only at full size (paper Section VI-D), and
the sanitizer is not available here, so every device buffer gets a guard
region of a known pattern on both sides and is checked after each run,
without trapping or asserting on the device:

* the five output arrays are caller-owned: the test places them between
  margins of a pattern and checks the margins on the host;
* plans made with SW_PLAN_GUARDS wrap the pair and class tables, the queue
  heads, the strip-boundary scratch and the host-call staging, and the
  one-shot call with guards on wraps every workspace part (tables, sort
  buffers, slots); a check kernel after the alignment kernels sets bit 2 of
  the context's status word if any guard word changed.

Runs workloads 1-3 at full size, the edge-length and maximum-length batches,
in the planned, graph, host-buffer and one-shot forms.  A negative control
breaks one guard word from the host and checks that the next run reports it.
"""
import numpy as np
import pytest

import oracle
import workloads as wl
from test_gpu_parity import EDGE, edge_batch

pytestmark = pytest.mark.gpu

MARGIN = 1024  # int32 words of pattern on each side of every output row
PATTERN = 0x5A5A5A5A


class GuardedOut:
    """Five output rows, each between MARGIN-word margins of PATTERN."""

    def __init__(self, n):
        import torch
        self.n = n
        self.stride = n + 2 * MARGIN
        self.buf = torch.full((5 * self.stride,), PATTERN, dtype=torch.int32, device="cuda")
        self.rows = [self.buf[k * self.stride + MARGIN:k * self.stride + MARGIN + n]
                     for k in range(5)]

    def margins_intact(self):
        h = self.buf.cpu().numpy()
        for k in range(5):
            lo = h[k * self.stride:k * self.stride + MARGIN]
            hi = h[k * self.stride + MARGIN + self.n:(k + 1) * self.stride]
            if not (np.all(lo == PATTERN) and np.all(hi == PATTERN)):
                return False
        return True

    def results(self):
        return np.stack([r.cpu().numpy() for r in self.rows], axis=1)


def long_batch():
    rng = np.random.default_rng(41)
    qs, rs = [], []
    for n, m in [(4000, 65535), (65535, 300), (3000, 3000), (1, 65535), (65535, 1),
                 (1363, 1500), (2500, 40)]:
        q = rng.integers(0, 4, n).astype(np.uint8)
        r = rng.integers(0, 4, m).astype(np.uint8)
        k = min(n, m, 2000)
        r[m - k:] = q[n - k:]
        qs.append(q)
        rs.append(r)
    return wl.make_batch("guard-long", qs, rs, wl.dna_matrix(), -6, -1)


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.sw_ctx_create(0)
    yield c
    gpu_lib.sw_ctx_destroy(c)


def planned_run(swgb, ctx, b, flags, host=False):
    import torch
    q = torch.from_numpy(b.q_seqs).cuda()
    r = torch.from_numpy(b.r_seqs).cuda()
    plan = swgb.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                               swgb.SW_MODE_AUTO, swgb.SW_PLAN_GUARDS | flags)
    try:
        if host:
            out = np.zeros((5, b.n_pairs), np.int32)
            swgb.sw_plan_execute_host(plan, b.q_seqs, b.r_seqs, out, None)
            res, intact = out.T.copy(), True
        else:
            g = GuardedOut(b.n_pairs)
            s = torch.cuda.Stream()
            for _ in range(2):  # graph plans: capture, then replay
                swgb.sw_plan_execute(plan, q, r, g.rows, s)
            s.synchronize()
            res, intact = g.results(), g.margins_intact()
    finally:
        swgb.sw_plan_destroy(plan)
    return res, intact, swgb.sw_ctx_status(ctx)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_full_workloads_guarded(gpu_lib, ctx, k):
    b = wl.gen_config(k)
    res, intact, status = planned_run(gpu_lib, ctx, b, gpu_lib.SW_PLAN_GRAPH)
    assert intact, "an output row's margin was overwritten"
    assert status == 0, f"status {status}: a guard word changed or a reverse pass lost its score"
    # the same results as an unguarded plan
    al = gpu_lib.Aligner(b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix, b.gap_open,
                         b.gap_extend, ctx=ctx)
    al.run()
    assert np.array_equal(res, al.results())
    al.close()


@pytest.mark.parametrize("which", ["edge", "long", "protein-edge"])
@pytest.mark.parametrize("form", ["planned", "pair-scratch", "host"])
def test_edge_and_maximum_lengths_guarded(gpu_lib, ctx, which, form):
    b = {"edge": lambda: edge_batch("dna", 3, EDGE, EDGE[::2]), "long": long_batch,
         "protein-edge": lambda: edge_batch("protein", 4, EDGE[::2], EDGE[1::2])}[which]()
    flags = gpu_lib.SW_PLAN_PAIR_SCRATCH if form == "pair-scratch" else 0
    res, intact, status = planned_run(gpu_lib, ctx, b, flags, host=form == "host")
    assert intact and status == 0, (intact, status)
    assert np.array_equal(res, oracle.align_workload(b))


@pytest.mark.parametrize("k", [1, 3])
def test_one_shot_workspace_guarded(gpu_lib, k):
    import torch
    swgb = gpu_lib
    c = swgb.sw_ctx_create(0)
    try:
        swgb.sw_ctx_set_guards(c, True)
        for b in (wl.gen_config(k), edge_batch("dna", 9, EDGE, EDGE[1::2]), long_batch()):
            g = GuardedOut(b.n_pairs)
            q = torch.from_numpy(b.q_seqs).cuda()
            r = torch.from_numpy(b.r_seqs).cuda()
            qo = torch.from_numpy(b.q_offsets).cuda()
            ro = torch.from_numpy(b.r_offsets).cuda()
            swgb.sw_align_batch_ex(c, q, qo, r, ro, b.matrix, b.gap_open, b.gap_extend,
                                   swgb.SW_MODE_AUTO, g.rows)
            torch.cuda.synchronize()
            assert g.margins_intact(), b.name
            assert swgb.sw_ctx_status(c) == 0, b.name
            if b.n_pairs < 5000:
                assert np.array_equal(g.results(), oracle.align_workload(b)), b.name
    finally:
        swgb.sw_ctx_destroy(c)


def test_a_broken_guard_is_reported(gpu_lib, ctx):
    """Negative control: a guard word changed from the host between runs
    shows in the status word after the next run, and only then."""
    import torch
    swgb = gpu_lib
    b = wl.gen_config(0, n_pairs=300)
    q = torch.from_numpy(b.q_seqs).cuda()
    r = torch.from_numpy(b.r_seqs).cuda()
    plan = swgb.sw_plan_create(ctx, b.q_offsets, b.r_offsets, b.matrix, b.gap_open, b.gap_extend,
                               swgb.SW_MODE_AUTO, swgb.SW_PLAN_GUARDS)
    try:
        out = torch.zeros((5, b.n_pairs), dtype=torch.int32, device="cuda")
        swgb.sw_plan_execute(plan, q, r, out)
        assert swgb.sw_ctx_status(ctx) == 0
        swgb.sw_plan_poison_guard(plan, 1)
        swgb.sw_plan_execute(plan, q, r, out)
        assert swgb.sw_ctx_status(ctx) & swgb.STATUS_GUARD
        with pytest.raises(swgb.SwError):
            swgb.sw_plan_poison_guard(plan, 10 ** 6)
    finally:
        swgb.sw_plan_destroy(plan)
