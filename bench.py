"""Benchmark: Heisenberg-picture kicked-Ising propagation on the 127-qubit
heavy-hex lattice through liborqa, reported as Pauli string-gate updates/s.

One step = one full evolution of sigma_z^62 through T Trotter steps (the ZZ
layer, the X layer with merge + truncation after every gate, and <M_t>
after each step), starting from the operator resident in HBM.  The update
count of a layer is the sum over its gates of |O| before the gate (144 ZZ
gates + 127 X gates per step), the convention behind the paper's per-gate
wall time (layer time / 271 gates).

    python bench.py [--gpus N --steps K --warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Under torchrun each rank runs its own replica of the workload on its own
GPU (replicas only: the single-observable path is not sharded), the
timings are max-reduced and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_13241_gb300 import workloads as W  # noqa: E402

# 127-qubit heavy-hex kicked Ising, theta_x = pi/4, 20 steps, delta = 3.5e-6:
# the live set peaks at 1.05e9 strings (at t = 9), about 40 bytes each
DEFAULT_WORKLOAD = "heavyhex_t=20_delta=3.5e-6"
METRIC = "Pauli string-gate updates/s"
UNIT = "string-gate updates/s"
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="orqa", choices=["orqa", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--capacity", type=float, default=0.0, help="string capacity (0: from workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="fp32: the precision form (FP32 coefficients, compensated pair updates)")
    ap.add_argument("--autotune", action="store_true",
                    help="sweep workloads: pick the launch tuning by measurement before warm-up")
    ap.add_argument("--compare-plain", action="store_true",
                    help="sweep workloads: also time the plain FP64 path, one problem after another")
    ap.add_argument("--truncation", default="absolute", choices=["absolute", "relative"],
                    help="relative: |c| <= delta * max|c| after every X gate (Eq. truncation1), gate by gate")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed evolutions: no norm invariants, delta sequence, end-to-end run or "
                         "sweep comparison (for profiler runs)")
    return ap.parse_args(argv)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def default_capacity(wl):
    """Strings per buffer (the workspace is ~196 B per unit of capacity at
    127 qubits).  Peaks measured for theta_x = pi/4 over 20 steps: 2.3e6 at
    delta = 1e-4, 2.0e7 at 3e-5, 1.5e8 at 1e-5, 5.5e8 at 5e-6; they grow
    about as delta^-1.8."""
    d = wl["delta"]
    if d <= 0.0:
        return int(2.5e7)
    est = 5.5e8 * (5e-6 / d) ** 1.8
    return int(min(max(1.35 * est, 1 << 21), 1.3e9))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_gpu_runner(wl, capacity, profile=True, fp32=False, relative=False):
    import numpy as np
    import torch
    from paper_2506_13241_gb300 import orqa as B

    n = wl["n"]
    ctx = B.Context(n, capacity, profile=profile, fp32=fp32, relative=relative)
    layers = [B.gate_array(layer) for layer in wl["layers"]]
    x_h, z_h = B.strings_from_labels([lab for lab, _ in wl["observable"]], n)
    c_h = np.array([c for _, c in wl["observable"]], dtype=np.float64)
    dev = torch.device("cuda", torch.cuda.current_device())
    x_d = torch.from_numpy(x_h.view(np.int64)).to(dev)
    z_d = torch.from_numpy(z_h.view(np.int64)).to(dev)
    c_d = torch.from_numpy(c_h).to(dev)
    # pinned host copies for the end-to-end arm
    x_p = torch.from_numpy(x_h.view(np.int64)).pin_memory()
    z_p = torch.from_numpy(z_h.view(np.int64)).pin_memory()
    c_p = torch.from_numpy(c_h).pin_memory()
    delta = wl["delta"]

    fp64 = {"one": 0, "two": 0, "branch": 0}  # pair updates and branch events of the timed steps

    def evolve(d=delta, steps=wl["steps"]):
        updates, mags, peak = 0, [], 0
        for _ in range(steps):
            for layer in layers:
                B.orqa_apply_layer(ctx.ctx, layer, d)
                s = B.orqa_counters(ctx.ctx)  # host counters only: no device work in the timed loop
                updates += s["string_gate_updates"]
                peak = max(peak, s["last_layer_peak"])
                fp64["one"] += s["pair_updates_one"]
                fp64["two"] += s["pair_updates_two"]
                fp64["branch"] += s["branch_events"]
            mags.append(B.orqa_expect(ctx.ctx))
        return updates, mags, peak

    def step_device(d=delta, steps=wl["steps"]):
        ctx.set_operator_device(x_d, z_d, c_d)
        return evolve(d, steps)

    def step_host():
        B.orqa_set_operator(ctx.ctx, x_p.numpy().view(np.uint64), z_p.numpy().view(np.uint64),
                            c_p.numpy())
        return evolve()

    def step_invariants():
        """One evolution with the norm bookkeeping: after every layer, sum c^2
        before minus sum c^2 after must equal the sum of c^2 the truncation
        removed (each gate is an orthogonal map on every pair of strings).
        Then the first steps at delta = 0, where sum c^2 must stay 1."""
        ctx.set_norm_tracking(True)
        ctx.set_operator_device(x_d, z_d, c_d)
        prev = B.orqa_stats(ctx.ctx)["sum_sq"]
        norm0 = prev
        worst, layers_checked, per_step = 0.0, 0, []
        for _ in range(wl["steps"]):
            for layer in layers:
                B.orqa_apply_layer(ctx.ctx, layer, delta)
                s = B.orqa_stats(ctx.ctx)
                worst = max(worst, abs(prev - s["sum_sq"] - s["dropped_sum_sq"]) / norm0)
                layers_checked += 1
                prev = s["sum_sq"]
            per_step.append(prev)
        ctx.set_operator_device(x_d, z_d, c_d)
        exact, exact_steps = 0.0, 0
        for _ in range(min(4, wl["steps"])):
            for layer in layers:
                B.orqa_apply_layer(ctx.ctx, layer, 0.0)
                exact = max(exact, abs(B.orqa_stats(ctx.ctx)["sum_sq"] - norm0) / norm0)
            exact_steps += 1
        ctx.set_norm_tracking(False)
        return {"max_rel_norm_gap": worst, "steps_checked": wl["steps"], "layers_checked": layers_checked,
                "sum_sq_per_step": per_step,
                "delta0_max_rel_norm_change": exact, "delta0_steps": exact_steps,
                "check": "|sum c^2 before - sum c^2 after - dropped sum c^2| / sum c^2 at t=0, per layer"}

    h2d = x_h.nbytes + z_h.nbytes + c_h.nbytes
    d2h = 8 * wl["steps"]
    return ctx, step_device, step_host, h2d, d2h, fp64, step_invariants


def run_gpu(args, wl, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    capacity = int(args.capacity) if args.capacity else default_capacity(wl)
    ctx, step_dev, step_host, h2d, d2h, fp64, step_inv = make_gpu_runner(wl, capacity,
                                                                         fp32=(args.precision == "fp32"),
                                                                         relative=(args.truncation == "relative"))
    stream = ctx.stream
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    invariants = None
    for k in range(args.warmup):
        if k == 0 and not args.no_extras and wl["delta"] > 0 and args.truncation == "absolute":
            invariants = step_inv()  # the first warm-up evolution checks the norm bookkeeping
        else:
            step_dev()
    torch.cuda.synchronize()
    ctx.profile_reset()
    fp64["one"] = fp64["two"] = fp64["branch"] = 0
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, total_updates, mags, peak = 0.0, 0, None, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            upd, mags, pk = step_dev()
            e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_updates += upd
        peak = max(peak, pk)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof = ctx.profile()
    fp64_ops = 2 * fp64["one"] + 6 * fp64["two"]
    branch_events = fp64["branch"]
    # end to end through the public API with host buffers
    e2e_s, e2e_updates = 0.0, 0
    for _ in range(max(1, min(args.steps, 2)) if not args.no_extras else 0):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upd, _, _ = step_host()
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        e2e_updates += upd
    deltas = None
    if not args.no_extras and wl["delta"] > 0 and args.truncation == "absolute":
        deltas = delta_sequence(wl, mags, step_dev)
    times, sums = reduce_over_ranks([total_ms, e2e_s], [total_updates, e2e_updates], "cuda")
    return dict(total_ms=times[0], updates=sums[0], mags=mags, peak=peak, clocks=clk,
                prof=prof, e2e_s=times[1], e2e_updates=sums[1], h2d=h2d, d2h=d2h,
                capacity=capacity, fp64_ops=fp64_ops, branch_events=branch_events,
                invariants=invariants, delta_sequence=deltas)


def delta_sequence(wl, mags, step_dev):
    """Parity beyond the oracle's reach: the same evolution at two larger
    thresholds (delta x 10/7 and x 20/7; 5e-6 and 1e-5 for delta = 3.5e-6).
    As delta falls the truncation error falls, so the differences between
    neighbouring thresholds should shrink step by step."""
    d0 = wl["delta"]
    seq = [d0, d0 * 10 / 7, d0 * 20 / 7]
    runs = [list(mags)]
    for d in seq[1:]:
        _, m, _ = step_dev(d)
        runs.append(m)
    near = [abs(a - b) for a, b in zip(runs[0], runs[1])]
    far = [abs(a - b) for a, b in zip(runs[1], runs[2])]
    return {"deltas": seq, "magnetization": runs, "max_abs_diff": [max(near), max(far)],
            "steps_closer_at_smaller_delta": sum(1 for a, b in zip(near, far) if a <= b),
            "steps": len(near)}


def reduce_over_ranks(times, counts, device="cpu"):
    """Replicas on N ranks: the slowest rank's times (max) and the work of
    all ranks (sum).  One rank: unchanged."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(times), list(counts)
    import torch
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    c = torch.tensor(list(counts), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), [int(round(v)) for v in c.tolist()]


def kernel_launches(prof):
    """Kernel launches behind the per-kind profile records: the scan is three
    kernels and the expectation two; every X layer adds one pass-bookkeeping
    kernel at its start and one per chunk pass, and every host-side commit
    (X layer, input merge, truncation) one small kernel."""
    n = {p["name"]: p["launches"] for p in prof}
    per_record = {"fine_scan": 3, "expect": 2}
    total = sum(v * per_record.get(k, 1) for k, v in n.items())
    total += n.get("rx_split", 0) + n.get("bucket_scatter", 0)                        # pass bookkeeping
    total += n.get("rx_split", 0) + n.get("merge_assign", 0) + n.get("truncate", 0)  # commits
    return total


def fp64_entry(prof, fp64_ops, sm_mhz):
    """FP64 view of the unit kernel: the pair updates need 2 (one member) or
    6 (both) FP64 operations; GB300 issues FP64 at 2 lanes per clock per SM."""
    local = [p for p in prof if p["name"] == "unit_local" and p["ms"] > 0]
    if not local:
        return None
    ms = local[0]["ms"]
    mhz = sm_mhz or 2070.0
    peak = 2.0 * 152 * mhz * 1e6
    achieved = fp64_ops / (ms * 1e-3)
    return {"kernel": "unit_local", "ops": fp64_ops, "achieved_ops_per_s": achieved,
            "peak_ops_per_s": peak, "frac": round(achieved / peak, 4),
            "peak_note": "2 FP64 lanes/clock/SM x 152 SMs x median SM clock (ncu peak_sustained)"}


# DRAM traffic of the unit kernel per branch event it processes, from one
# ncu capture scoped to that kernel (dram__bytes_read.sum +
# dram__bytes_write.sum over all its launches of one evolution of a
# few-GB heavy-hex case, divided by that evolution's branch events); the
# command and figures are in profiles/.  traffic = this ratio x the branch
# events of an average launch here.  Valid only while the kernel is
# unchanged: None until it has been measured on the current kernel.
UNIT_DRAM_BYTES_PER_BRANCH = 27.57
UNIT_DRAM_SOURCE = "profiles/unit_kernel_traffic_heavyhex_t8_delta3e-5.md"
# What bounds the unit kernel, from its ncu full capture (fractions of each
# unit's peak on the few-GB heavy-hex case; the same validity rule): issue
# slots and the ALU and FP64 pipes are busy, DRAM is not.
UNIT_LIMITER = {"issue_active": 0.672, "alu_pipe": 0.657, "fp64_pipe": 0.558, "dram_throughput": 0.086,
                "warps_active": 0.434, "source": "profiles/unit_kernel_heavyhex_t8_delta3e-5.md"}


def roofline_entry(prof, steps, workload=None, precision="fp64", n_qubits=127):
    """The dominant kernel against the measured HBM bandwidth.  `achieved`
    divides the kernel's share of the method's traffic floor (per X gate: 8
    bytes of z per string tested, and per branch event the string's record
    read, the child record and the parent's c written and a merge that
    meets and writes both once -- 4R + 8 = 168 bytes at 127 qubits in FP64)
    by the CUDA-event time of its launches; `frac_pass_model` does the same
    with the bytes of this implementation's pass structure."""
    peak_gbs, peak_src = measured_peaks()
    timed = [p for p in prof if p["launches"] > 0 and p["ms"] > 0]
    if not timed:
        return None
    dom = max(timed, key=lambda p: p["ms"])
    secs = dom["ms"] * 1e-3
    floor_b = dom.get("floor_bytes", 0.0)
    achieved = floor_b / secs / 1e9
    pass_achieved = dom["bytes"] / secs / 1e9
    entry = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
             "peak": peak_gbs, "peak_source": peak_src, "unit": "GB/s",
             "frac": round(achieved / peak_gbs, 4),
             "traffic": None, "traffic_source": None,
             "frac_pass_model": round(pass_achieved / peak_gbs, 4), "achieved_pass_model": round(pass_achieved, 1),
             "launches": dom["launches"], "avg_launch_ms": dom["ms"] / dom["launches"],
             "algorithmic_bytes_per_launch": floor_b / dom["launches"],
             "pass_model_bytes_per_launch": dom["bytes"] / dom["launches"],
             "share_of_kernel_time": round(dom["ms"] / sum(p["ms"] for p in timed), 4),
             "kernels": {p["name"]: {"launches": p["launches"], "ms": round(p["ms"], 3),
                                     "floor_GB/s": round(p.get("floor_bytes", 0.0) / (p["ms"] * 1e-3) / 1e9, 1),
                                     "pass_model_GB/s": round(p["bytes"] / (p["ms"] * 1e-3) / 1e9, 1)}
                         for p in timed}}
    if dom["name"] == "unit_local" and UNIT_DRAM_BYTES_PER_BRANCH and floor_b > 0:
        R = 16 * (1 if n_qubits <= 64 else 2) + (4 if precision == "fp32" else 8)
        per_branch = 4 * R + (4 if precision == "fp32" else 8)
        branches_per_launch = floor_b / per_branch / dom["launches"]
        entry["traffic"] = UNIT_DRAM_BYTES_PER_BRANCH * branches_per_launch
        entry["traffic_source"] = UNIT_DRAM_SOURCE + " (DRAM bytes per branch event x branch events per launch)"
        if precision == "fp64" and UNIT_LIMITER:
            entry["limiter"] = dict(UNIT_LIMITER)
    return entry


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

ORACLE_MAX_TERMS = 20_000_000  # keeps the std::map oracle within a few GB of host memory


def oracle_sample(wl, seconds: float, relative: bool = False):
    """Runs the oracle on the workload from its start, gate by gate, and stops
    after the gate that passes ``seconds`` (or when the operator outgrows
    ORACLE_MAX_TERMS), so the sample is bounded whatever the workload size.
    Returns (updates, seconds used, whole time steps done, gates done in the
    last partial step, <M_t> of the whole steps)."""
    import oracle
    n = wl["n"]
    op = oracle.Oracle(n)
    for lab, c in wl["observable"]:
        op.add_label(lab, c)
    updates, t_used, steps, mags, partial = 0, 0.0, 0, [], 0
    t0 = time.perf_counter()
    for t in range(wl["steps"]):
        partial = 0
        for layer in wl["layers"]:
            for g in layer:
                size = len(op)
                if time.perf_counter() - t0 >= seconds or size > ORACLE_MAX_TERMS:
                    return updates, time.perf_counter() - t0, steps, partial, mags
                updates += size
                if relative:
                    op.apply_rel(g, wl["delta"])
                else:
                    op.apply(g, wl["delta"])
                partial += 1
        mags.append(op.expect_zero())
        steps = t + 1
    return updates, time.perf_counter() - t0, steps, 0, mags


def host_cpu():
    """The host's CPU model (x86 'model name', else the Arm part fields) and
    logical core count."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read().splitlines()
        for key in ("model name", "CPU part"):
            vals = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith(key)]
            if vals:
                model = vals[0] if key == "model name" else "Arm CPU part %s" % vals[0]
                break
    except OSError:
        pass
    import platform
    return {"model": model or platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(wl, seconds, relative=False):
    upd, secs, steps, partial, mags = oracle_sample(wl, seconds, relative)
    return {"value": upd / secs if secs > 0 else None, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": "first %d of %d time steps of %s plus %d gates of the next (%d string-gate "
                      "updates, %.1f s)" % (steps, wl["steps"], wl["name"], partial, upd, secs),
            "magnetization": mags}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    seconds = min(20.0, max(2.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(wl, seconds)
    upd, secs, steps = 0, 0.0, 0
    partial = 0
    for _ in range(args.steps):
        u, s, st, partial, _ = oracle_sample(wl, seconds)
        upd += u
        secs += s
        steps = st
    value = upd / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": "first %d of %d time steps of %s plus %d gates, per step" % (
                                 steps, wl["steps"], wl["name"], partial)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def fp64_magnetization(wl, capacity):
    """<M_t> of one FP64 evolution on the GPU (the precision form's comparison)."""
    import gc
    import torch
    gc.collect()
    torch.cuda.empty_cache()
    step_dev = make_gpu_runner(wl, capacity, profile=False, fp32=False)[1]
    _, mags, _ = step_dev()
    return mags


def error_entry(mags, ref):
    """|Delta M_t| per step over the steps both runs reached."""
    k = min(len(mags), len(ref))
    per_step = [abs(a - b) for a, b in zip(mags[:k], ref[:k])]
    return {"steps_compared": k, "max_abs": max(per_step) if per_step else None, "per_step": per_step}


def workload_config(wl, precision="fp64", truncation="absolute"):
    return {"workload": wl["name"], "lattice": "heavy-hex 127" if wl["n"] == 127 else "chain %d" % wl["n"],
            "n_qubits": wl["n"], "theta_x": wl["theta_x"], "theta_zz": W.THETA_ZZ,
            "observable": "Z_62" if wl["n"] == 127 else "Z_6", "time_steps": wl["steps"],
            "delta": wl["delta"],
            "truncation": ("absolute |c| < delta after every X gate" if truncation == "absolute" else
                           "relative |c| <= delta * max|c| after every X gate, one gate per pass"),
            "coefficients": precision, "l2": "flushed between timed steps"}


# ---------------------------------------------------------------------------
# Batched theta x observable sweep (one captured program for all problems)
# ---------------------------------------------------------------------------

def sweep_from_name(name: str):
    """sweep[_n=<angles>][_t=<steps>][_delta=<d>]: angles uniform in
    [0, pi/2] x Z-strings of weight 1, 3, 17 around qubit 62."""
    n_theta, steps, delta = 32, 10, 1e-4
    for part in name.split("_")[1:]:
        k, v = part.split("=")
        if k == "n":
            n_theta = int(v)
        elif k == "t":
            steps = int(v)
        elif k == "delta":
            delta = float(v)
    wl = W.sweep_workload(n_theta, steps, delta)
    wl["name"] = name
    return wl


def shard_sweep(wl, rank, world):
    """The problems of one rank when N ranks share a sweep: problem p goes to
    rank p mod N.  The problems are independent, so the ranks exchange no
    data; round-robin gives every rank a similar mix of angles and
    observable weights.  One rank: the sweep itself."""
    if world <= 1:
        return wl
    idx = list(range(rank, len(wl["problems"]), world))
    out = dict(wl)
    out["problems"] = [wl["problems"][p] for p in idx]
    out["theta"] = [wl["theta"][p] for p in idx]
    out["problem_index"] = idx
    return out


def sweep_inputs(wl):
    import numpy as np
    from paper_2506_13241_gb300 import orqa as B
    labels, coefs, pids = [], [], []
    for p, terms in enumerate(wl["problems"]):
        for lab, c in terms:
            labels.append(lab)
            coefs.append(c)
            pids.append(p)
    x, z = B.strings_from_labels(labels, wl["n"])
    return x, z, np.array(coefs, dtype=np.float64), np.array(pids, dtype=np.int32)


def run_plain_sweep(wl, capacity):
    """The plain FP64 path on the same problems, one after another (the
    single-operator calls a user of the plain API makes)."""
    import numpy as np
    import torch
    from paper_2506_13241_gb300 import orqa as B
    n, steps, delta = wl["n"], wl["steps"], wl["delta"]
    ctx = B.Context(n, capacity)
    mags = np.zeros((steps, len(wl["problems"])))
    updates = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, terms in enumerate(wl["problems"]):
        layers = [B.gate_array(layer) for layer in W.kicked_ising_layers(n, wl["edges"], wl["theta"][p])]
        ctx.set_labels(terms)
        for t in range(steps):
            for layer in layers:
                B.orqa_apply_layer(ctx.ctx, layer, delta)
                updates += B.orqa_counters(ctx.ctx)["string_gate_updates"]
            mags[t, p] = B.orqa_expect(ctx.ctx)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    del ctx
    return {"seconds": secs, "updates": updates, "value": updates / secs, "unit": UNIT}, mags


def sweep_launches(ctx_stats, wl, n_zz_launches):
    """Kernel launches of one sweep step: the batched set_operator (merge: 4
    kernels + commit) and the graph (per Trotter step: the ZZ launches and
    their end kernel; the X layer's begin, split, pass-advance and end
    kernels; 6 kernels per chunk pass; 2 expectation kernels)."""
    steps = wl["steps"]
    return 5 + steps * (n_zz_launches + 1 + 4 + 2) + 6 * int(ctx_stats["chunk_passes"])


def run_sweep(args, wl, rank, world):
    import numpy as np
    import torch
    from paper_2506_13241_gb300 import orqa as B
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n, P, steps, delta = wl["n"], len(wl["problems"]), wl["steps"], wl["delta"]
    zz, xx = wl["layers"]
    theta = np.array([[wl["theta"][p]] * len(xx) for p in range(P)])
    fp32 = args.precision == "fp32"
    capacity = int(args.capacity) if args.capacity else int(4e8)
    ctx = B.Context(n, capacity, fp32=fp32, problems=P)
    prog = ctx.program([(zz, False, None), (xx, True, theta)])
    x, z, c, pid = sweep_inputs(wl)
    stream = ctx.stream

    def step():
        B.orqa_set_operator_batch(ctx.ctx, x, z, c, pid)
        return ctx.run_program(prog, steps, delta)

    tuned = None
    if args.autotune:
        B.orqa_set_operator_batch(ctx.ctx, x, z, c, pid)
        best, best_ms = ctx.autotune(prog, steps, delta, trials=1)
        tuned = {"tuning": best, "graph_ms": best_ms}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, updates, mags = 0.0, 0, None
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mags = step()
            e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        updates += B.orqa_counters(ctx.ctx)["string_gate_updates"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = ctx.stats()
    e2e_s = 0.0
    for _ in range(max(1, min(args.steps, 2))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        e2e_s += time.perf_counter() - t0
    e2e_steps = max(1, min(args.steps, 2))
    sizes = ctx.problem_sizes()
    # kernel table of the same evolution, host-driven with per-launch events
    pctx = B.Context(n, capacity, fp32=fp32, problems=P, profile=True)
    B.orqa_set_operator_batch(pctx.ctx, x, z, c, pid)
    zza, xxa = B.gate_array(zz), B.gate_array(xx)
    for _ in range(steps):
        B.orqa_apply_layer(pctx.ctx, zza, delta)
        B.orqa_apply_layer_batch(pctx.ctx, xxa, theta, delta)
        pctx.expect_batch()
    prof = pctx.profile()
    del pctx
    n_zz = 1  # the kicked-Ising ZZ layer is one Clifford set: one closed-form launch
    res = dict(total_ms=total_ms, updates=updates, mags=mags, clocks=clk, prof=prof, e2e_s=e2e_s,
               e2e_updates=updates / args.steps * e2e_steps, stats=st, sizes=sizes, tuned=tuned,
               launches=sweep_launches(st, wl, n_zz) * args.steps,
               h2d=x.nbytes + z.nbytes + c.nbytes + pid.nbytes, d2h=steps * P * 8 + 64)
    del ctx
    return res


def main_sweep(args, world, rank):
    """The batched sweep.  On N ranks its problems are sharded (problem p on
    rank p mod N, no data exchanged): the total work is fixed, so the
    scaling is strong; the time is the slowest rank's and the updates are
    summed over the ranks."""
    import numpy as np
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    wl_all = sweep_from_name(args.workload)
    wl = shard_sweep(wl_all, rank, world)
    from paper_2506_13241_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    res = run_sweep(args, wl, rank, world)
    times, sums = reduce_over_ranks([res["total_ms"], res["e2e_s"]], [res["updates"], res["e2e_updates"]], "cuda")
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    total_ms, e2e_s = times
    updates, e2e_updates = sums
    secs = total_ms * 1e-3
    value = updates / secs
    P = len(wl_all["problems"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wl_all["name"], "lattice": "heavy-hex 127", "problems": P,
                       "theta_x": "%d values uniform in [0, pi/2]" % (P // len(wl["weights"])),
                       "observables": "Z-strings of weight %s around qubit 62" % wl["weights"],
                       "time_steps": wl["steps"], "delta": wl["delta"],
                       "truncation": "absolute |c| < delta after every X gate",
                       "coefficients": args.precision, "execution": "one captured CUDA graph per step",
                       "l2": "flushed between timed steps"},
            "roofline": roofline_entry(res["prof"], 1),
            "e2e": {"value": e2e_updates / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "peak_strings": res["stats"]["last_layer_peak"], "chunk_passes_per_step": res["stats"]["chunk_passes"],
            "final_sizes": {"total": int(res["sizes"].sum()), "max": int(res["sizes"].max())}}
    if world > 1:
        line["config"]["sharding"] = "problem p on rank p mod %d; no data exchanged" % world
    if res["tuned"]:
        line["autotune"] = res["tuned"]
    if args.compare_plain and world == 1:
        plain, pm = run_plain_sweep(wl, int(6e7))
        line["plain_fp64_sequential"] = plain
        line["speedup_vs_plain_fp64"] = value / plain["value"]
        diff = np.abs(np.asarray(res["mags"]) - pm)
        line["magnetization_error_vs_plain_fp64"] = {"max_abs": float(diff.max()),
                                                     "per_step_max": [float(v) for v in diff.max(axis=1)]}
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SWEEP_BOUND = 1e-6  # |Delta M_t| the precision form should stay within


def sweep_comparison(steps_timed=2):
    """The batched theta x observable sweep (32 angles in [0, pi/2] x Z-strings
    of weight 1, 3, 17 around qubit 62, 10 Trotter steps, delta = 1e-4) in
    the FP32-compensated batched form (one captured graph per sweep) against
    the plain FP64 path (one problem after another, per-layer calls): the
    speed-up and max over the problems of |Delta M_t| per Trotter step."""
    import gc

    import numpy as np
    import torch
    from paper_2506_13241_gb300 import orqa as B
    gc.collect()
    torch.cuda.empty_cache()
    wl = sweep_from_name("sweep")
    n, P, steps, delta = wl["n"], len(wl["problems"]), wl["steps"], wl["delta"]
    zz, xx = wl["layers"]
    theta = np.array([[wl["theta"][p]] * len(xx) for p in range(P)])
    ctx = B.Context(n, int(4e8), fp32=True, problems=P)
    ctx.set_tuning(bucket_density=32, grid_per_sm=8)  # the autotuner's choice for this sweep
    prog = ctx.program([(zz, False, None), (xx, True, theta)])
    x, z, c, pid = sweep_inputs(wl)
    stream = ctx.stream

    def step():
        B.orqa_set_operator_batch(ctx.ctx, x, z, c, pid)
        return ctx.run_program(prog, steps, delta)

    mags = step()  # captures the graph
    ms, updates = 0.0, 0
    for _ in range(steps_timed):
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mags = step()
            e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        updates += B.orqa_counters(ctx.ctx)["string_gate_updates"]
    del ctx
    gc.collect()
    torch.cuda.empty_cache()
    plain, pm = run_plain_sweep(wl, int(6e7))
    per_step = np.abs(np.asarray(mags) - pm).max(axis=1)
    within = 0
    for v in per_step:
        if v > SWEEP_BOUND:
            break
        within += 1
    batched = updates / (ms * 1e-3)
    return {"workload": "sweep: %d angles x 3 observables, %d steps, delta %g" % (P // 3, steps, delta),
            "batched_fp32": {"value": batched, "unit": UNIT, "ms_per_sweep": ms / steps_timed},
            "plain_fp64_sequential": plain, "speedup": batched / plain["value"],
            "max_abs_dM_per_step": [float(v) for v in per_step], "bound": SWEEP_BOUND,
            "steps_within_bound": within, "bound_met": within == steps,
            "reference": "the plain FP64 path (its operators equal the CPU oracle's bit for bit in the tests)"}


def main(argv=None):
    args = parse_args(argv)
    if args.workload.startswith("sweep") and args.impl != "reference":
        return main_sweep(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
    wl = W.workload(args.workload)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_2506_13241_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    res = run_gpu(args, wl, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    total_updates = res["updates"]  # summed over the ranks' replicas
    secs = res["total_ms"] * 1e-3
    value = total_updates / secs
    e2e_value = res["e2e_updates"] / res["e2e_s"] if res["e2e_s"] > 0 else None
    launches = kernel_launches(res["prof"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["total_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic", "config": workload_config(wl, args.precision, args.truncation),
            "roofline": roofline_entry(res["prof"], args.steps, wl["name"], args.precision, wl["n"]),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                    "d2h_bytes_per_step": res["d2h"]},
            "gpu_launches": launches, "clocks": res["clocks"],
            "magnetization": res["mags"], "peak_strings": res["peak"], "capacity": res["capacity"]}
    line["fp64"] = fp64_entry(res["prof"], res["fp64_ops"], res["clocks"].get("sm_mhz"))
    if res["invariants"] is not None:
        line["invariants"] = res["invariants"]
    if res["delta_sequence"] is not None:
        line["delta_sequence"] = res["delta_sequence"]
    # secondary metric: anticommuting (string, gate) pairs per second (rank 0's replica)
    line["branch_events_per_s"] = res["branch_events"] / (res["total_ms"] * 1e-3) * world
    line["branch_events"] = res["branch_events"]  # of the timed evolutions on this rank
    if args.precision == "fp32":
        # The precision form's error per step against the GPU FP64 path on
        # the same workload (one untimed evolution after the timed run).
        line["magnetization_error_vs_gpu_fp64"] = error_entry(res["mags"], fp64_magnetization(wl, res["capacity"]))
    if not args.no_extras and world == 1 and wl["n"] == 127 and args.precision == "fp64" and \
            args.truncation == "absolute":
        res["prof"] = None
        line["sweep"] = sweep_comparison()
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is an N = 1 figure
        cb = cpu_baseline(wl, args.cpu_seconds, args.truncation == "relative")
        om = cb.pop("magnetization")
        line["magnetization_error_vs_oracle"] = error_entry(res["mags"], om)
        line["cpu_baseline"] = cb
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
