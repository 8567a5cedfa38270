"""Benchmark: batched Smith-Waterman/Gotoh alignment on GB300.

One step = one pass of the whole hot path (forward DP, end-cell selection,
reverse DP, output) over the 100,000-pair DNA workload (query 100-300,
reference 200-1024, 30% planted; +3/-3, gap_open -6, gap_extend -1) with the
inputs resident in device memory.  The metric is GCUPS: forward cells
(sum of n*m) per second, whole job.  The same line reports the plain
one-block-per-pair launch on the same GPU, the end-to-end rate through the
host-buffer C-ABI call, the integer-pipe roofline of the batched kernel, and
the CPU oracle timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the workload grows to N times the per-GPU size and is
split across the ranks by longest-processing-time over n*m (weak scaling,
no collective on the data path); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "bit-exact GCUPS on 1 GB300, batched vs plain, % int-pipe roofline; serve p99 ms"
CONFIG = 1
OPS_PER_CELL = 6
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=CONFIG)
    ap.add_argument("--pairs", type=int, default=0,
                    help="only the first N pairs of the workload (0 = all); for profiler captures")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-pairs", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--gaps", type=int, nargs=2, metavar=("OPEN", "EXTEND"), default=None,
                    help="override the workload's gap costs (equal values take the linear-gap kernel)")
    ap.add_argument("--dna-scores", type=int, nargs=2, metavar=("MATCH", "MISMATCH"),
                    default=None, help="override a DNA workload's match/mismatch scores")
    ap.add_argument("--ends-only", action="store_true",
                    help="score and end cell only (no reverse pass)")
    ap.add_argument("--packed", action="store_true",
                    help="2-bit packed DNA input (expanded on the device inside each step)")
    ap.add_argument("--no-s16x2", action="store_true",
                    help="keep the batched kernel on scaled int32 arithmetic (one cell per "
                         "instruction) where the packed 16-bit form would apply")
    ap.add_argument("--no-cigar", action="store_true",
                    help="skip timing the traceback (CIGAR) of every aligned pair")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-serve-staged", action="store_true",
                    help="skip the serving sweep with per-request staged sequences")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the secondary workloads (1,000 DNA, 20k protein, 200k skewed DNA)")
    ap.add_argument("--config-steps", type=int, default=6,
                    help="timed steps of each secondary workload")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's own lane-group choice instead of measuring candidates")
    ap.add_argument("--tune-cache", default=os.path.join(ROOT, ".swgb_tune_cache.json"))
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per rate point")
    ap.add_argument("--serve-rate0", type=float, default=250.0, help="first offered rate, req/s")
    ap.add_argument("--serve-points", type=int, default=14)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    ap.add_argument("--serve-clients", type=int, default=4,
                    help="client threads submitting the Poisson arrival schedule")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ CPU oracle leg

def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(batch, n_pairs: int, threads: int, gpu_res=None, cols: int = 5) -> dict:
    """The CPU oracle timed on the first n_pairs pairs; with gpu_res, also
    whether the GPU's results for those pairs equal the oracle's."""
    import oracle
    oracle.build()
    sub = batch.slice(0, n_pairs)
    t0 = time.perf_counter()
    ref = oracle.align_workload(sub, threads=threads)
    dt = time.perf_counter() - t0
    cells = sub.cells
    out = {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": threads, "kind": "oracle",
           "sample": f"first {n_pairs} pairs of {batch.name} ({cells / 1e9:.3f} G forward cells), "
                     f"{dt:.2f} s on {threads} host threads",
           "seconds": dt, "pairs": n_pairs}
    if gpu_res is not None:
        a, b = ref[:, :cols], gpu_res[:n_pairs, :cols]
        out["gpu_identical_pairs"] = int(np.sum(np.all(a == b, axis=1)))
        out["gpu_identical"] = bool(np.array_equal(a, b))
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def single_core_rate(batch, multi: dict, target_s: float = 2.0) -> dict:
    """The oracle on one host thread, over the first pairs of the workload
    (about target_s seconds, sized from the multi-threaded run)."""
    per_pair_1 = multi["seconds"] * multi["cores"] / max(1, multi["pairs"])
    n1 = int(max(50, min(multi["pairs"], target_s / max(per_pair_1, 1e-9))))
    r = oracle_rate(batch, n1, 1)
    return {"value": r["value"], "unit": "GCUPS", "cores": 1, "sample": r["sample"]}


def auto_cpu_pairs(batch, threads: int, target_s: float = 12.0) -> int:
    """Pairs of the workload the oracle aligns in about target_s seconds here."""
    probe = min(2000, batch.n_pairs)
    r = oracle_rate(batch, probe, threads)
    per_pair = r["seconds"] / probe
    return int(max(probe, min(batch.n_pairs, target_s / per_pair)))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        mx = [num(r[2]) for r in rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# -------------------------------------------------------------- reference arm

def run_reference(args, rank):
    if rank != 0:
        return
    batch = wl.gen_config(args.config)
    threads = cpu_cores()
    n = args.cpu_pairs or max(500, auto_cpu_pairs(batch, threads, target_s=6.0) // 2)
    for _ in range(args.warmup):
        oracle_rate(batch, min(n, 500), threads)
    vals, secs, cells = [], 0.0, 0
    for _ in range(args.steps):
        r = oracle_rate(batch, n, threads)
        vals.append(r["value"])
        secs += r["seconds"]
        cells += batch.slice(0, n).cells
    value = cells / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": batch.name, "pairs_per_step": n, "threads": threads},
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": threads, "kind": "oracle",
                             "sample": f"first {n} pairs of {batch.name} per step",
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ ncu traffic

def profiled_traffic(batch, tune, arith="s16x2", flags=0, sms=152) -> tuple[int | None, bool]:
    """(DRAM bytes per launch of the group kernel from the committed ncu
    summary, whether the captured plan put the same number of pairs on each
    lane-group width as this run's tuning).  The bytes are None unless that
    capture was of this workload, this arithmetic and this kernel source (the
    counters are stale otherwise); a plan with other widths (the autotuner's
    choice can differ between boxes) keeps the figure and says so."""
    import hashlib
    import re
    form = "" if arith == "s16x2" else "s32_"
    path = os.path.join(ROOT, "profiles", f"sw_group_kernel_{form}{batch.name}.md")
    src = os.path.join(ROOT, "paper_2208_12350_gb300", "csrc", "kernel_group.cu")
    import paper_2208_12350_gb300 as swgb
    # captures are of the default plan (starts and ends, one byte per residue)
    if not os.path.exists(path) or flags & ~swgb.SW_PLAN_NO_S16X2:
        return None, False
    if tune is None:  # not autotuned: the planner's own choice
        tune = {"narrow_log2g": -1, "cap_fraction": 0.5}
    text = open(path).read()
    sha = re.search(r"kernel_sha256: ([0-9a-f]{64})", text)
    wid = re.search(r"widths: ([0-9,]+)", text)
    byt = re.search(r"dram_bytes_per_launch: (\d+)", text)
    if not (sha and wid and byt):
        return None, False
    if sha.group(1) != hashlib.sha256(open(src, "rb").read()).hexdigest():
        return None, False
    ar = re.search(r"arith: (\w+)", text)
    if (ar.group(1) if ar else "s32") != arith:
        return None, False
    _, lg, _ = swgb.sw_plan_preview(batch.q_offsets, batch.r_offsets, batch.matrix,
                                    batch.gap_open, batch.gap_extend, swgb.SW_MODE_BATCHED, flags,
                                    sms, tune["narrow_log2g"], tune["cap_fraction"])
    hist = np.bincount(lg[lg >= 0], minlength=6)[:6].tolist() + [int(np.sum(lg < 0))]
    return int(byt.group(1)), hist == [int(x) for x in wid.group(1).split(",")]


# ------------------------------------------------------------------- serving

def serve_sweep(swgb, ctx, pools, expect, args, resident: bool) -> dict:
    """Open-loop serving: Poisson arrivals of requests of floor(log-uniform
    [1, 4096]) pairs, half from the DNA workload and half from the protein
    workload, offered at rates growing x1.5 per point until one point past
    the first the server no longer keeps up with (served rate below 90% of
    offered), or p99 above 1 s.
    resident: both workloads are uploaded once as resident pools and each
    request names its pair range (sequences stay on the device); otherwise
    each request brings its sequences, staged at submission.  Latency =
    completion on the GPU (server clock) - scheduled arrival, so a late
    submitter counts against the server, as a real client would.  Every
    request's results are compared with the CPU oracle's results for those
    pairs (expect)."""
    import queue
    import threading
    reqs = wl.serving_requests(args.serve_requests, 1.0, pools=pools)
    budget = int(args.serve_budget_gb * (1 << 30))
    srv = swgb.sw_server_create(ctx, budget, streams=8, staging_bytes=2 << 30)
    identical = True
    pid = {}
    if resident:
        for kind, b in pools.items():
            pid[kind] = swgb.sw_server_add_pool(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets,
                                                b.matrix, b.gap_open, b.gap_extend)

    def check(rq, out):
        exp = expect[rq.kind][rq.first:rq.first + rq.batch.n_pairs]
        return bool(np.array_equal(out, exp))

    def submit(rq):
        b = rq.batch
        if resident:
            return swgb.sw_server_submit_pool(srv, pid[rq.kind], rq.first, b.n_pairs,
                                              timeout_ms=120000)
        return swgb.sw_server_submit(srv, b.q_seqs, b.q_offsets, b.r_seqs, b.r_offsets, b.matrix,
                                     b.gap_open, b.gap_extend, timeout_ms=120000)

    # warm-up: one at a time, then a burst that puts work on every stream slot
    # (their first launches allocate staging and workspace)
    for rq in reqs[:16]:
        out = swgb.sw_server_wait(srv, submit(rq), rq.batch.n_pairs, timeout_ms=120000)
        identical &= check(rq, out)
    for _ in range(2):
        burst = [(rq, submit(rq)) for rq in reqs[:64]]
        for rq, rid in burst:
            identical &= check(rq, swgb.sw_server_wait(srv, rid, rq.batch.n_pairs,
                                                       timeout_ms=120000))
    points = []
    n_sub = max(1, args.serve_clients)
    rate = args.serve_rate0
    misses = 0
    # the client side must not pause: collect once, then no cyclic GC during
    # the sweep (the earlier legs leave a large heap behind)
    import gc
    gc.collect()
    gc.disable()
    try:
        for _ in range(args.serve_points):
            n = min(len(reqs), max(200, int(rate * 20.0)))
            lc0 = swgb.sw_server_launches(srv)
            todo = reqs[:n]
            arrival = np.zeros(n, dtype=np.int64)
            ids: queue.Queue = queue.Queue()
            t0 = time.monotonic_ns() + 20_000_000
            for i, rq in enumerate(todo):
                arrival[i] = t0 + int(rq.arrival_s / rate * 1e9)

            def submitter(k):
                # client thread k submits requests k, k + S, ... at their
                # scheduled arrivals (the copy into the server's staging runs
                # outside the interpreter lock, so clients overlap)
                try:
                    for i in range(k, n, n_sub):
                        delay = (arrival[i] - time.monotonic_ns()) / 1e9
                        if delay > 0:
                            time.sleep(delay)
                        ids.put((i, submit(todo[i])))
                except Exception as e:  # surfaced by the waiter
                    ids.put((-1, e))

            ths = [threading.Thread(target=submitter, args=(k,)) for k in range(n_sub)]
            for th in ths:
                th.start()
            lat = np.zeros(n)
            done_last = 0
            cells = 0
            for _k in range(n):
                i, rid = ids.get()
                if i < 0:
                    raise rid
                rq = todo[i]
                out, done_ns = swgb.sw_server_wait(srv, rid, rq.batch.n_pairs, timeout_ms=120000,
                                                   return_done_ns=True)
                identical &= check(rq, out)
                lat[i] = (done_ns - arrival[i]) / 1e6
                done_last = max(done_last, done_ns)
                cells += rq.batch.cells
            for th in ths:
                th.join()
            lc1 = swgb.sw_server_launches(srv)
            span = (done_last - t0) / 1e9
            served = n / span
            pt = {"offered_rps": rate, "requests": n, "served_rps": served,
                  "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                  "gcups": cells / span / 1e9,
                  "launches": lc1["launches"] - lc0["launches"],
                  "plan_ms_per_launch": (lc1["plan_ms"] - lc0["plan_ms"]) /
                  max(1, lc1["launches"] - lc0["launches"])}
            points.append(pt)
            if pt["p99_ms"] > 1000.0:
                break
            if served < 0.9 * rate:
                # one point past the first rate not kept up with, so that the
                # saturation throughput is measured however close that miss was
                misses += 1
                if misses == 2:
                    break
            rate *= 1.5
        st = swgb.sw_server_stats(srv)
    finally:
        gc.enable()
        swgb.sw_server_destroy(srv)
    kept = [p for p in points if p["served_rps"] >= 0.9 * p["offered_rps"]
            and p["p99_ms"] <= 1000.0]
    best = kept[-1] if kept else None
    return {"p99_ms": best["p99_ms"] if best else None, "p50_ms": best["p50_ms"] if best else None,
            "at_rps": best["offered_rps"] if best else None,
            "max_sustained_rps": best["served_rps"] if best else None,
            "peak_gcups": max(p["gcups"] for p in points) if points else None,
            "oracle_identical": identical, "budget_gb": args.serve_budget_gb, "streams": 8,
            "client_threads": n_sub,
            "sequences": ("resident pools on the device (requests name pair ranges)" if resident
                          else "staged per request (each request brings its sequences)"),
            "device_bytes_peak": st["device_bytes_peak"],
            "requests": "Poisson arrivals; floor(log-uniform[1,4096]) pairs; 50% dna-100k, "
                        "50% protein-20k pairs; every result compared with the CPU oracle",
            "points": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in p.items()}
                       for p in points]}


# ------------------------------------------------------------------- our arm

def reverse_cells(res: np.ndarray) -> int:
    """Cells the reverse pass needs: rows 0..qend by columns rend..rstart."""
    ok = res[:, 0] > 0
    q = res[ok, 1].astype(np.int64) + 1
    c = (res[ok, 2] - res[ok, 4]).astype(np.int64) + 1
    return int(np.sum(q * c))


def time_plan(swgb, torch, plan, q, r, out, stream, steps, warmup, flush):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for _ in range(warmup):
        flush.add_(1)
        swgb.sw_plan_execute(plan, q, r, out, stream)
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.add_(1)  # larger than L2: every step starts with a cold L2
            ev[k][0].record(stream)
            swgb.sw_plan_execute(plan, q, r, out, stream)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def nominal_peak(sms: int, mhz: float | None, lanes_per_clk: int = 64) -> float | None:
    """Integer ALU lane-instructions per second (T/s) of the whole device at
    the sampled clock: lanes_per_clk per SM (64 = 4 sub-partitions x 16
    lanes of the ALU pipe that issues the max forms)."""
    return lanes_per_clk * sms * mhz * 1e6 / 1e12 if mhz else None


def roofline_fracs(ops_per_cell: int, max_ops_per_cell: int, cells_total: int, seconds: float,
                   sms: int, mhz: float | None) -> dict:
    """The alternative roofline fractions beside the measured-peak one:
    frac_nominal against 64 lanes/clk/SM at the sampled clock, frac_survey_128
    against 128 lanes/clk/SM, frac_max_only counting only the max-type
    algorithmic ops per cell (E, F, the three-way H max, the end key; the two
    adds issue on the FMA pipe) against 64 lanes/clk/SM."""
    nom = nominal_peak(sms, mhz)
    s128 = nominal_peak(sms, mhz, 128)
    ach = ops_per_cell * cells_total / seconds / 1e12
    ach_max = max_ops_per_cell * cells_total / seconds / 1e12
    return {"frac_nominal": ach / nom if nom else None,
            "frac_survey_128": ach / s128 if s128 else None,
            "frac_max_only": ach_max / nom if nom else None,
            "peak_nominal": nom, "max_ops_per_cell": max_ops_per_cell}


def time_one_shot(swgb, torch, batch, dev, stream, steps, warmup, in_place=False):
    """End to end through sw_align_batch: every step copies the sequences and
    offsets from page-locked host buffers to the device (in_place: passes the
    page-locked buffers themselves, which the kernels read over the coherent
    host link), plans on the device (no offset read-back, no host planning),
    runs both passes and copies the five result rows back; host-timed,
    synchronised at the end of each step."""
    qh = torch.from_numpy(batch.q_seqs).pin_memory()
    rh = torch.from_numpy(batch.r_seqs).pin_memory()
    qoh = torch.from_numpy(batch.q_offsets).pin_memory()
    roh = torch.from_numpy(batch.r_offsets).pin_memory()
    q = torch.empty_like(qh, device=dev)
    r = torch.empty_like(rh, device=dev)
    qo = torch.empty_like(qoh, device=dev)
    ro = torch.empty_like(roh, device=dev)
    out = torch.empty((5, batch.n_pairs), dtype=torch.int32, device=dev)
    oh = torch.empty((5, batch.n_pairs), dtype=torch.int32).pin_memory()

    def step():
        with torch.cuda.stream(stream):
            if in_place:
                swgb.sw_align_batch(qh, qoh, rh, roh, batch.matrix, batch.gap_open,
                                    batch.gap_extend, out, stream)
            else:
                q.copy_(qh, non_blocking=True)
                r.copy_(rh, non_blocking=True)
                qo.copy_(qoh, non_blocking=True)
                ro.copy_(roh, non_blocking=True)
                swgb.sw_align_batch(q, qo, r, ro, batch.matrix, batch.gap_open,
                                    batch.gap_extend, out, stream)
            oh.copy_(out, non_blocking=True)
        stream.synchronize()

    for _ in range(warmup):
        step()
    step_t = []
    t0 = time.perf_counter()
    for _ in range(steps):
        t1 = time.perf_counter()
        step()
        step_t.append(time.perf_counter() - t1)
    dt = time.perf_counter() - t0
    h2d = int(qh.numel() + rh.numel() + 8 * (qoh.numel() + roh.numel()))
    stats = {"min": min(step_t) * 1e3, "median": statistics.median(step_t) * 1e3,
             "max": max(step_t) * 1e3}
    return dt, oh.numpy().T.copy(), h2d, int(oh.numel() * 4), stats


def measure_config(swgb, torch, ctx, k, dev, stream, flush, steps, tune_cache, sms):
    """Secondary workload k: the batched form (autotuned, CUDA graph), the
    plain one-block-per-pair form, the roofline fractions, the clocks of the
    timed region and the whole workload compared with the oracle."""
    import oracle
    batch = wl.gen_config(k)
    q = torch.from_numpy(batch.q_seqs).to(dev)
    r = torch.from_numpy(batch.r_seqs).to(dev)
    out = torch.zeros((5, batch.n_pairs), dtype=torch.int32, device=dev)
    tune = swgb.sw_autotune(ctx, batch.q_offsets, batch.r_offsets, batch.matrix, batch.gap_open,
                            batch.gap_extend, q, r, out, cache_path=tune_cache, stream=stream)
    plan = swgb.sw_plan_create(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                               batch.gap_open, batch.gap_extend, swgb.SW_MODE_BATCHED,
                               swgb.SW_PLAN_GRAPH)
    info = swgb.sw_plan_info(plan)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    times = time_plan(swgb, torch, plan, q, r, out, stream, steps, 3, flush)
    clk = clocks.stop()
    swgb.sw_plan_destroy(plan)
    res = out.T.contiguous().cpu().numpy()
    t = sum(times) / len(times)
    cells = batch.cells
    rcells = reverse_cells(res)
    packed16 = info["arith"] == "s16x2"
    opc = OPS_PER_CELL // 2 if packed16 else OPS_PER_CELL
    pplan = swgb.sw_plan_create(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                                batch.gap_open, batch.gap_extend, swgb.SW_MODE_PLAIN, 0)
    out2 = torch.zeros_like(out)
    pt = time_plan(swgb, torch, pplan, q, r, out2, stream, max(2, steps // 2), 1, flush)
    swgb.sw_plan_destroy(pplan)
    plain_same = bool(torch.equal(out, out2))
    threads = cpu_cores()
    t0 = time.perf_counter()
    ref = oracle.align_workload(batch, threads=threads)
    odt = time.perf_counter() - t0
    same = np.all(ref == res, axis=1)
    v = cells / t / 1e9
    pv = cells * len(pt) / sum(pt) / 1e9
    mb_rate, _ = swgb.sw_microbench_int("viaddmax_s16x2" if packed16 else "viaddmax_s32",
                                        dev.index, 2048)
    entry = {"workload": batch.name, "pairs": batch.n_pairs, "forward_cells": cells,
             "reverse_cells": rcells, "arith": info["arith"], "rows": info["rows"], "tuning": tune,
             "batched_gcups": v, "ms_per_step": t * 1e3, "steps": len(times),
             "plain_gcups": pv, "plain_identical_outputs": plain_same,
             "batched_over_plain": v / pv,
             "frac": opc * (cells + rcells) / t / mb_rate if mb_rate else None,
             "oracle_identical_pairs": int(same.sum()), "oracle_identical": bool(same.all()),
             "oracle_gcups": cells / odt / 1e9, "oracle_threads": threads, "clocks": clk}
    entry.update(roofline_fracs(opc, 2 if packed16 else 4, cells + rcells, t, sms,
                                clk.get("sm_mhz")))
    return entry


def run_ours(args, rank, world, local):
    import torch
    import paper_2208_12350_gb300 as swgb
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    swgb.load()
    if world > 1:
        # weak scaling: a global workload of world x the per-GPU size, split by
        # longest-processing-time over n*m so every rank gets the same DP work
        from paper_2208_12350_gb300 import shard
        per = args.pairs or wl.CONFIGS[args.config]["n_pairs"]
        full = wl.gen_config(args.config, n_pairs=per * world)
        mine = shard.lpt_partition(shard.pair_costs(full.q_offsets, full.r_offsets), world)[rank]
        q_, qo_, r_, ro_ = shard.shard_batch(full.q_seqs, full.q_offsets, full.r_seqs,
                                             full.r_offsets, mine)
        batch = wl.Batch(full.name, q_, qo_, r_, ro_, full.matrix,
                         full.gap_open, full.gap_extend, full.planted[mine])
        del full
    else:
        batch = wl.gen_config(args.config, n_pairs=args.pairs or None)
    if args.dna_scores:
        batch.matrix = wl.dna_matrix(*args.dna_scores)
        batch.name += f"-dna{args.dna_scores[0]:+d}{args.dna_scores[1]:+d}"
    if args.gaps:
        batch.gap_open, batch.gap_extend = args.gaps
        batch.name += f"-gaps{args.gaps[0]}{args.gaps[1]}"
    flags = (swgb.SW_PLAN_ENDS_ONLY if args.ends_only else 0) | \
        (swgb.SW_PLAN_PACKED_2BIT if args.packed else 0) | \
        (swgb.SW_PLAN_NO_S16X2 if args.no_s16x2 else 0)
    # the input the plans read: one byte per residue, or 2-bit packed
    q_in = swgb.sw_pack_2bit(batch.q_seqs) if args.packed else batch.q_seqs
    r_in = swgb.sw_pack_2bit(batch.r_seqs) if args.packed else batch.r_seqs
    cells = batch.cells
    ctx = swgb.sw_ctx_create(local)
    sms = swgb.sw_ctx_sm_count(ctx)
    stream = torch.cuda.Stream(device=dev)
    q = torch.from_numpy(q_in).to(dev)
    r = torch.from_numpy(r_in).to(dev)
    out = torch.zeros((5, batch.n_pairs), dtype=torch.int32, device=dev)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # unpacked copies for the calls that take one byte per residue
    q8 = torch.from_numpy(batch.q_seqs).to(dev) if args.packed else q
    r8 = torch.from_numpy(batch.r_seqs).to(dev) if args.packed else r
    tune = None
    if not args.no_autotune:
        # measured choice of the lane-group widths (cached by GPU and batch shape)
        tune = swgb.sw_autotune(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                                batch.gap_open, batch.gap_extend, q8, r8, out,
                                cache_path=args.tune_cache, stream=stream, flags=flags)
        torch.cuda.synchronize()
    plan = swgb.sw_plan_create(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                               batch.gap_open, batch.gap_extend, swgb.SW_MODE_BATCHED,
                               swgb.SW_PLAN_GRAPH | flags)
    info = swgb.sw_plan_info(plan)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    times = time_plan(swgb, torch, plan, q, r, out, stream, args.steps, args.warmup, flush)
    barrier()
    clk = clocks.stop()
    t_total = sum(times)
    if world > 1:
        t = torch.tensor([t_total], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_total = float(t.item())
    res = out.T.contiguous().cpu().numpy()
    rcells = 0 if args.ends_only else reverse_cells(res)
    job_cells = cells
    if world > 1:
        c = torch.tensor([cells], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(c)
        job_cells = int(c.item())
    value = job_cells * args.steps / t_total / 1e9
    per_launch = t_total / args.steps

    # --- integer roofline of the batched kernel (events timed live above)
    # the packed 16-bit form does each of the 6 ops for two cells with one
    # instruction: 3 instruction slots per cell against the packed max's rate
    packed16 = info["arith"] == "s16x2"
    ops_per_cell = OPS_PER_CELL // 2 if packed16 else OPS_PER_CELL
    peak_op = "viaddmax_s16x2" if packed16 else "viaddmax_s32"
    ops = ops_per_cell * (cells + rcells)
    achieved = ops / per_launch / 1e12
    sm_mhz = clk.get("sm_mhz")
    mb_rate, _ = swgb.sw_microbench_int(peak_op, local, 2048)
    peak_measured = mb_rate / 1e12
    traffic, traffic_same_plan = profiled_traffic(batch, tune, info["arith"], flags, sms) \
        if batch.n_pairs == wl.CONFIGS[args.config]["n_pairs"] else (None, False)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_measured, "unit": "Tops/s",
            "frac": achieved / peak_measured if peak_measured else None, "traffic": traffic,
            **roofline_fracs(ops_per_cell, 2 if packed16 else 4, cells + rcells, per_launch,
                             sms, sm_mhz),
            "peak_kind": f"measured __{peak_op} issue rate, whole device, this run",
            "ops_per_cell": ops_per_cell, "cells_forward": cells, "cells_reverse": rcells,
            "traffic_unit": "DRAM bytes per launch (ncu, committed summary)",
            "traffic_same_plan": traffic_same_plan,
            "algorithmic_bytes": int(batch.q_seqs.nbytes + batch.r_seqs.nbytes + 20 * batch.n_pairs)}

    # --- plain one-block-per-pair comparator
    plain = None
    if not args.no_plain:
        pplan = swgb.sw_plan_create(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                                    batch.gap_open, batch.gap_extend, swgb.SW_MODE_PLAIN, flags)
        out2 = torch.zeros_like(out)
        pt = time_plan(swgb, torch, pplan, q, r, out2, stream, max(3, args.steps // 2), 1, flush)
        same = bool(torch.equal(out, out2))
        swgb.sw_plan_destroy(pplan)
        pv = cells * len(pt) / sum(pt) / 1e9
        plain = {"value": pv, "unit": "GCUPS", "ms_per_step": sum(pt) / len(pt) * 1e3,
                 "steps": len(pt), "identical_outputs": same}

    # --- end to end through the host-buffer C-ABI call
    qh = torch.from_numpy(q_in).pin_memory()
    rh = torch.from_numpy(r_in).pin_memory()
    oh = torch.zeros((5, batch.n_pairs), dtype=torch.int32).pin_memory()
    eplan = swgb.sw_plan_create(ctx, batch.q_offsets, batch.r_offsets, batch.matrix,
                                batch.gap_open, batch.gap_extend, swgb.SW_MODE_BATCHED,
                                swgb.SW_PLAN_GRAPH | flags)
    # the inputs' transport, chosen before the timed region by a short probe
    # of each (like the kernel tuning): read in place over the coherent host
    # link where the device can (fastest on an idle link), or copied by the
    # copy engines (steadier when the link is busy)
    probe = {}
    for tr in ([True, False] if swgb.sw_ctx_host_in_place(ctx) else [False]):
        swgb.sw_ctx_set_host_in_place(ctx, tr)
        for _ in range(max(2, args.warmup)):
            swgb.sw_plan_execute_host(eplan, qh, rh, oh, stream)
        tp = time.perf_counter()
        for _ in range(3):
            swgb.sw_plan_execute_host(eplan, qh, rh, oh, stream)
        probe["in_place" if tr else "copied"] = (time.perf_counter() - tp) / 3 * 1e3
    in_place = "in_place" in probe and probe["in_place"] <= probe.get("copied", float("inf"))
    swgb.sw_ctx_set_host_in_place(ctx, in_place)
    for _ in range(args.warmup):
        swgb.sw_plan_execute_host(eplan, qh, rh, oh, stream)
    barrier()
    step_t = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t1 = time.perf_counter()
        swgb.sw_plan_execute_host(eplan, qh, rh, oh, stream)
        step_t.append(time.perf_counter() - t1)
    barrier()
    e2e_t = time.perf_counter() - t0
    e2e_same = bool(np.array_equal(oh.numpy().T, res))
    swgb.sw_plan_destroy(eplan)
    swgb.sw_ctx_set_host_in_place(ctx, True)  # the device's default again
    e2e = {"value": job_cells * args.steps / e2e_t / 1e9, "unit": "GCUPS",
           "h2d_bytes_per_step": int(q_in.nbytes + r_in.nbytes),
           "d2h_bytes_per_step": int(5 * 4 * batch.n_pairs), "identical_outputs": e2e_same,
           "step_ms": {"min": min(step_t) * 1e3, "median": statistics.median(step_t) * 1e3,
                       "max": max(step_t) * 1e3},
           "inputs": ("page-locked host buffers read in place by the kernels over the "
                      "coherent host link" if in_place
                      else "page-locked host buffers copied to the device each step"),
           "transport_probe_ms": probe}

    swgb.sw_plan_destroy(plan)

    # --- end to end through the one-shot call, planning on the device inside
    # the timed region (fresh offsets uploaded every step)
    e2e_oneshot = None
    if not (args.packed or args.ends_only or args.no_s16x2 or world > 1):
        ot, ores, oh2d, od2h, ostats = time_one_shot(swgb, torch, batch, dev, stream, args.steps,
                                                     args.warmup)
        e2e_oneshot = {"value": job_cells * args.steps / ot / 1e9, "unit": "GCUPS",
                       "ms_per_step": ot / args.steps * 1e3, "step_ms": ostats,
                       "h2d_bytes_per_step": oh2d, "d2h_bytes_per_step": od2h,
                       "identical_outputs": bool(np.array_equal(ores, res)),
                       "call": "sw_align_batch (device offsets; planned on the device)",
                       "inputs": "page-locked host buffers copied to the device each step"}
        if swgb.sw_ctx_host_in_place(ctx):
            it, ires, ih2d, id2h, istats = time_one_shot(swgb, torch, batch, dev, stream,
                                                         args.steps, args.warmup, in_place=True)
            e2e_oneshot["in_place"] = {
                "value": job_cells * args.steps / it / 1e9, "unit": "GCUPS",
                "ms_per_step": it / args.steps * 1e3, "step_ms": istats,
                "h2d_bytes_per_step": ih2d, "d2h_bytes_per_step": id2h,
                "identical_outputs": bool(np.array_equal(ires, res)),
                "inputs": ("the page-locked host buffers themselves (sequences and "
                           "offsets), read by the planner and the kernels over the "
                           "coherent host link")}

    cigar = None
    if not args.no_cigar and not args.ends_only and world == 1:
        # traceback of every aligned pair: cells = the spans' global DP.  The
        # headline call takes the results where the alignment left them, on
        # the device (sw_traceback_device: spans classified by kernels); the
        # host-prepared call (sw_traceback, results on the host) beside it.
        res5 = np.ascontiguousarray(res.T)
        coff = swgb.sw_cigar_capacity(res5)
        res5_d = torch.from_numpy(res5).to(dev)
        qo_d = torch.from_numpy(np.ascontiguousarray(batch.q_offsets, dtype=np.int64)).to(dev)
        ro_d = torch.from_numpy(np.ascontiguousarray(batch.r_offsets, dtype=np.int64)).to(dev)
        coff_d = torch.empty(batch.n_pairs + 1, dtype=torch.int64, device=dev)
        swgb.sw_cigar_capacity_device(res5_d, coff_d, stream)
        stream.synchronize()
        same_offsets = bool(np.array_equal(coff_d.cpu().numpy(), coff))
        ops = torch.zeros(max(1, int(coff[-1])), dtype=torch.int32, device=dev)
        nops = torch.zeros(batch.n_pairs, dtype=torch.int32, device=dev)
        ok = res[:, 0] > 0
        span_cells = int(np.sum((res[ok, 1] - res[ok, 3] + 1).astype(np.int64) *
                                (res[ok, 2] - res[ok, 4] + 1)))

        def tb_device():
            swgb.sw_traceback_device(ctx, q8, qo_d, r8, ro_d, batch.matrix, batch.gap_open,
                                     batch.gap_extend, res5_d, coff_d, ops, nops, stream)

        def tb_host():
            swgb.sw_traceback(ctx, q8, batch.q_offsets, r8, batch.r_offsets, batch.matrix,
                              batch.gap_open, batch.gap_extend, res5, coff, ops, nops, stream)

        def time_calls(call, reps=3):
            call()
            torch.cuda.synchronize()
            dev_ms, host_ms = [], []
            t0 = time.perf_counter()
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                th = time.perf_counter()
                call()
                host_ms.append((time.perf_counter() - th) * 1e3)
                e1.record(stream)
                stream.synchronize()
                dev_ms.append(e0.elapsed_time(e1))
            dt = (time.perf_counter() - t0) / reps
            return {"value": span_cells / dt / 1e9, "unit": "GCUPS (span cells)",
                    "ms": dt * 1e3, "device_ms": statistics.median(dev_ms),
                    "call_host_ms": statistics.median(host_ms),
                    "device_value": span_cells / (statistics.median(dev_ms) * 1e-3) / 1e9}

        host_leg = time_calls(tb_host)
        host_ops = ops.cpu().numpy().view(np.uint32).copy()
        host_nops = nops.cpu().numpy().copy()
        ops.zero_()
        nops.zero_()
        dev_leg = time_calls(tb_device)
        # the CIGARs of a sample of pairs against the CPU oracle's
        import oracle
        idx = np.flatnonzero(ok)[::97]
        sub = batch.subset(idx)
        eops, eoff, en = oracle.cigar_workload(sub, res[idx])
        got_ops = ops.cpu().numpy().view(np.uint32)
        got_n = nops.cpu().numpy()
        same = all(int(got_n[p]) == int(en[k]) and np.array_equal(
            got_ops[coff[p]:coff[p] + got_n[p]], eops[eoff[k]:eoff[k] + en[k]])
            for k, p in enumerate(idx))
        host_leg["identical_to_device_call"] = bool(
            np.array_equal(host_nops, got_n) and np.array_equal(host_ops, got_ops))
        host_leg["call"] = ("sw_traceback: results and offsets on the host, spans classified "
                            "by host threads inside the call (the GPU idles meanwhile)")
        cigar = dict(dev_leg)
        cigar.update({
            "span_cells": span_cells, "pairs": int(ok.sum()), "ops": int(nops.sum().item()),
            "oracle_identical_sample": bool(same), "device_offsets_identical": same_offsets,
            "sample": f"{len(idx)} aligned pairs (every 97th) against the CPU oracle",
            "call": "sw_traceback_device: results, offsets and cigar offsets on the device",
            "host_inputs": host_leg,
            "note": "value: host-timed call + stream synchronisation, 3 calls after one "
                    "untimed; the device call waits for its three classification kernels and "
                    "reads back a summary before it enqueues the fill and walk; device_value: "
                    "CUDA events around the call on its stream; scratch from the context's pool"})

    overridden = bool(args.gaps or args.dna_scores or args.ends_only or args.pairs or args.packed)
    configs = None
    if not args.no_configs and rank == 0 and world == 1 and not overridden and args.config == 1:
        configs = {}
        for k in (0, 2, 3):
            configs[str(k)] = measure_config(swgb, torch, ctx, k, dev, stream, flush,
                                             args.config_steps, args.tune_cache, sms)

    serve = serve_staged = None
    if not args.no_serve and rank == 0 and world == 1 and not overridden:
        import oracle
        dna = batch if args.config == 1 else wl.gen_config(1)
        protein = wl.gen_config(2)
        pools = {"dna": dna, "protein": protein}
        expect = {k: oracle.align_workload(b, threads=cpu_cores()) for k, b in pools.items()}
        serve = serve_sweep(swgb, ctx, pools, expect, args, resident=True)
        if not args.no_serve_staged:
            serve_staged = serve_sweep(swgb, ctx, pools, expect, args, resident=False)
    swgb.sw_ctx_destroy(ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = cpu_cores()
        n = args.cpu_pairs or auto_cpu_pairs(batch, threads)
        cpu = oracle_rate(batch, n, threads, gpu_res=res, cols=3 if args.ends_only else 5)
        cpu["single_core"] = single_core_rate(batch, cpu)
        cpu["cpu_model"] = cpu_model()
        cpu.pop("seconds")
        cpu.pop("pairs")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_launch * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int16x2" if packed16 else "int32", "data": "synthetic",
                "config": {"workload": batch.name, "pairs": batch.n_pairs,
                           "forward_cells": cells, "mode": "batched persistent + CUDA graph",
                           "l2": "flushed between steps (512 MB write)", "sms": sms,
                           "input": "2-bit packed, expanded on the device" if args.packed
                           else "one byte per residue",
                           "shards": (f"{world} LPT shards of {world} x the per-GPU pairs"
                                      if world > 1 else None),
                           "tuning": tune, "arith": info["arith"], "rows_per_lane": info["rows"],
                           "group_pairs": info["group_pairs"]},
                "plain": plain,
                "batched_over_plain": (value / world) / plain["value"] if plain else None,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "e2e_oneshot": e2e_oneshot,
                "configs": configs, "serve": serve, "serve_staged": serve_staged, "cigar": cigar,
                "clocks": clk,
                "gpu_launches": info["launches"] * args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
