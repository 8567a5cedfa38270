"""The benchmark's output contract, checked on the CPU.

The reference arm (the CPU oracle timed on the host cores) prints one JSON
line with the keys every benchmark line carries; under torchrun only rank 0
works and prints.  The roofline's DRAM traffic is read from the committed
ncu summary only for the plan that was captured (same kernel source, same
number of pairs on each lane-group width, the default plan flags).
"""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_bench(extra_env=None, *args):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    return r


def test_reference_arm_line():
    r = _run_bench(None, "--impl", "reference", "--config", "0", "--steps", "2", "--warmup", "1",
                   "--cpu-pairs", "120")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "GCUPS" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "dna-1k" and d["config"]["pairs_per_step"] == 120
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "120" in cb["sample"] and cb["cpu_model"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == "GCUPS"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    r = _run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference",
                   "--config", "0", "--steps", "1", "--warmup", "1", "--cpu-pairs", "50")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


@pytest.fixture(scope="module")
def bench_mod():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    import paper_2208_12350_gb300 as swgb
    try:
        swgb.load()
    except Exception as e:  # the library is built by __graft_entry__.build()
        pytest.fail(f"libswgb.so does not load: {e}")
    return mod


def test_roofline_traffic_only_for_the_captured_kernel(bench_mod):
    """The committed ncu figure is used only for the kernel source and
    arithmetic it was captured with; a plan with other lane-group widths keeps
    it but is flagged."""
    import re
    import workloads as wl
    import paper_2208_12350_gb300 as swgb
    text = open(os.path.join(ROOT, "profiles", "sw_group_kernel_dna-100k.md")).read()
    want = int(re.search(r"dram_bytes_per_launch: (\d+)", text).group(1))
    b = wl.gen_config(1)
    sha_now = __import__("hashlib").sha256(open(os.path.join(
        ROOT, "paper_2208_12350_gb300", "csrc", "kernel_group.cu"), "rb").read()).hexdigest()
    captured = re.search(r"kernel_sha256: ([0-9a-f]{64})", text).group(1)
    # the capture runs the planner's own plan (the benchmark without autotuning)
    got, same = bench_mod.profiled_traffic(b, {"narrow_log2g": -1, "cap_fraction": 0.5},
                                           "s16x2", 0, 152)
    if sha_now == captured:
        assert got == want and same
        got1, same1 = bench_mod.profiled_traffic(b, {"narrow_log2g": 1, "cap_fraction": 0.5},
                                                 "s16x2", 0, 152)
        assert got1 == want and not same1  # another plan: kept, flagged
        # no autotuning: the planner's own plan, as captured
        assert bench_mod.profiled_traffic(b, None, "s16x2", 0, 152) == (want, True)
    else:
        assert got is None  # the kernel changed since the capture: stale counters
    # another arithmetic reads its own capture (never the packed form's)
    s32 = open(os.path.join(ROOT, "profiles", "sw_group_kernel_s32_dna-100k.md")).read()
    s32_bytes = int(re.search(r"dram_bytes_per_launch: (\d+)", s32).group(1))
    s32_sha = re.search(r"kernel_sha256: ([0-9a-f]{64})", s32).group(1)
    assert bench_mod.profiled_traffic(b, {"narrow_log2g": -1, "cap_fraction": 0.5}, "s32", 0,
                                      152)[0] == (s32_bytes if s32_sha == sha_now else None)
    # other plan flags: no traffic
    assert bench_mod.profiled_traffic(b, {"narrow_log2g": -1, "cap_fraction": 0.5}, "s16x2",
                                      swgb.SW_PLAN_ENDS_ONLY, 152)[0] is None


def test_single_core_oracle_rate(bench_mod):
    """The CPU baseline's single-thread figure: the oracle on one thread over
    a sample sized from the multi-threaded run."""
    import workloads as wl
    b = wl.gen_config(0)
    multi = bench_mod.oracle_rate(b, 60, 2)
    one = bench_mod.single_core_rate(b, multi, target_s=0.2)
    assert one["cores"] == 1 and one["unit"] == "GCUPS" and one["value"] > 0
    assert "1 host threads" in one["sample"]
    assert isinstance(bench_mod.cpu_model(), str) and bench_mod.cpu_model()
