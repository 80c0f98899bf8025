"""Host-side pieces of bench.py that need no GPU: argument defaults, the
roofline entry, the kernel-launch count, error summaries and workload
names."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_finish_within_minutes():
    a = bench.parse_args([])
    assert (a.gpus, a.steps, a.warmup) == (1, 3, 3)
    assert a.warmup >= 3 and a.workload == bench.DEFAULT_WORKLOAD and a.impl == "orqa"


def test_roofline_entry_uses_the_dominant_kernel():
    """frac divides the dominant kernel's share of the method's traffic floor
    (168 bytes per branch event for the unit kernel at 127 qubits, FP64) by
    its event time; frac_pass_model uses the pass-structure bytes; traffic
    is the per-branch-event DRAM ratio of a scoped capture, if measured on
    the current kernel."""
    prof = [{"name": "unit_local", "launches": 4, "ms": 40.0, "bytes": 4.0e10, "floor_bytes": 168.0 * 1e8},
            {"name": "bucket_scatter", "launches": 4, "ms": 10.0, "bytes": 2.0e10, "floor_bytes": 0.0},
            {"name": "expect", "launches": 0, "ms": 0.0, "bytes": 0.0, "floor_bytes": 0.0}]
    r = bench.roofline_entry(prof, 1, bench.DEFAULT_WORKLOAD)
    peak, _ = bench.measured_peaks()
    assert r["kernel"] == "unit_local" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 420.0) < 1e-9                      # 1.68e10 B / 40 ms
    assert abs(r["frac"] - round(420.0 / peak, 4)) < 1e-12
    assert abs(r["achieved_pass_model"] - 1000.0) < 1e-9          # 4e10 B / 40 ms
    assert abs(r["algorithmic_bytes_per_launch"] - 168.0 * 1e8 / 4) < 1e-3
    assert abs(r["share_of_kernel_time"] - 0.8) < 1e-12
    old = bench.UNIT_DRAM_BYTES_PER_BRANCH
    try:
        bench.UNIT_DRAM_BYTES_PER_BRANCH = None
        assert bench.roofline_entry(prof, 1)["traffic"] is None
        bench.UNIT_DRAM_BYTES_PER_BRANCH = 100.0
        r = bench.roofline_entry(prof, 1)
        assert abs(r["traffic"] - 100.0 * 1e8 / 4) < 1e-3          # 2.5e7 branch events per launch
        # the captured limiter of the unit kernel rides along, with its source
        assert r["limiter"]["source"].startswith("profiles/") and 0 < r["limiter"]["issue_active"] <= 1
    finally:
        bench.UNIT_DRAM_BYTES_PER_BRANCH = old


def test_kernel_launch_count():
    prof = [{"name": "rzz_layer", "launches": 2}, {"name": "rx_split", "launches": 2},
            {"name": "fine_scan", "launches": 5}, {"name": "bucket_scatter", "launches": 5},
            {"name": "unit_local", "launches": 5}, {"name": "expect", "launches": 2},
            {"name": "merge_assign", "launches": 1}, {"name": "merge_offsets", "launches": 1},
            {"name": "merge_scatter", "launches": 1}, {"name": "merge_reduce", "launches": 1},
            {"name": "truncate", "launches": 1}]
    # 2 + 2 + 15 + 5 + 5 + 4 + 4 merge + 1 truncate, + (2 + 5) pass bookkeeping, + (2 + 1 + 1) commits
    assert bench.kernel_launches(prof) == 38 + 7 + 4


def test_error_entry_and_names():
    e = bench.error_entry([1.0, 0.5, 0.25], [1.0, 0.5 + 1e-9])
    assert e["steps_compared"] == 2 and abs(e["max_abs"] - 1e-9) < 1e-15
    wl = bench.sweep_from_name("sweep_n=4_t=2_delta=1e-3")
    assert len(wl["problems"]) == 12 and wl["steps"] == 2 and wl["delta"] == 1e-3
    cfg = bench.workload_config(bench.W.workload("heavyhex"), "fp32")
    assert cfg["coefficients"] == "fp32" and cfg["n_qubits"] == 127 and "l2" in cfg
    host = bench.host_cpu()
    assert host["nproc"] >= 1 and host["model"]


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    import sys
    env = dict(os.environ)
    env.update(env_extra or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True,
                         text=True, env=env, cwd=ROOT, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_contract_line():
    """The reference arm times the CPU oracle on the arm's own metric and
    workload; one JSON line, no GPU needed."""
    lines = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--workload", "chain12"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "chain12"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs and prints the reference line."""
    assert _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "chain12"],
                      {"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_sweep_shards_partition_the_problems():
    """On N ranks the sweep's problems are split round-robin: every problem
    on exactly one rank, shard sizes within one, angles kept with their
    problems."""
    wl = bench.sweep_from_name("sweep_n=5_t=2_delta=1e-3")
    P = len(wl["problems"])
    assert bench.shard_sweep(wl, 0, 1) is wl
    for world in (2, 3, 4, 7):
        shards = [bench.shard_sweep(wl, r, world) for r in range(world)]
        seen = sorted(p for sh in shards for p in sh["problem_index"])
        assert seen == list(range(P))
        sizes = [len(sh["problems"]) for sh in shards]
        assert max(sizes) - min(sizes) <= 1
        for sh in shards:
            for k, p in enumerate(sh["problem_index"]):
                assert sh["problems"][k] == wl["problems"][p] and sh["theta"][k] == wl["theta"][p]


def test_clock_summary_from_nvidia_smi_lines():
    """The clocks entry: median SM clock under load, the maximum clock, and
    every throttle reason seen Active (nvidia-smi csv, noheader, nounits)."""
    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    cs = bench.ClockSampler(0)
    cs.proc = _Done()
    cs.lines = [
        "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "",
    ]
    assert cs.stop() == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]
