"""Benchmark: evaluation throughput of lattice splines on one B300 (Gpoints/s).

Workload (one "step"): the BCC configuration -- coefficients on 2 cosets of
128^3 (bounding box 0..255) as the smooth field sin(0.05x)cos(0.07y)+0.1N(0,1),
evaluated with the linear 4-direction and the doubled 8-direction ("quintic")
box splines at 2^24 uniform points and at 2^24 points along 4096 parallel rays
(ray-march order): four launches, 2^26 point evaluations per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Multi-GPU runs (torchrun) shard nothing: every rank
evaluates its own full per-GPU workload (weak scaling), no collective on the
data path; timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "Gpoints/s per spline+lattice and % of gather roofline; fwd+bwd vs plain FP32"
EXT = (128, 128, 128)
N_UNIFORM = 1 << 24
N_RAYS, RAY_STEPS = 4096, 4096
CASES = [("bcc_linear", "uniform"), ("bcc_linear", "rays"), ("bcc_quintic", "uniform"), ("bcc_quintic", "rays")]
WORKLOAD = ("bcc 2x128^3 smooth field; linear + quintic box splines; 2^24 uniform + 2^24 ray points "
            "(4096 rays x 4096 steps)")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(seed_offset: int = 0):
    coef = workloads.coef_smooth("bcc", EXT, seed=0)
    lo, hi = workloads.inner_box("bcc_quintic", EXT)
    uni = workloads.points_uniform(N_UNIFORM, lo, hi, seed=1 + seed_offset)
    rays = workloads.points_rays(N_RAYS, RAY_STEPS, lo, hi, seed=3 + seed_offset)
    return coef, {"uniform": uni, "rays": rays}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------

ORACLE_SAMPLE = {"bcc_linear": 1 << 15, "bcc_quintic": 1 << 11}


def oracle_leg(coef, pts_sets, repeats: int = 1):
    import oracle
    from oracle import specs as ospecs
    cores = len(os.sched_getaffinity(0))
    spec = {"bcc_linear": ospecs.bcc_linear().with_extent(EXT),
            "bcc_quintic": ospecs.bcc_quintic().with_extent(EXT)}
    c64 = coef.astype(np.float64).ravel()
    rng = np.random.default_rng(99)
    samples = {}
    for sp, ps in CASES:
        idx = rng.choice(len(pts_sets[ps]), ORACLE_SAMPLE[sp], replace=False)
        samples[(sp, ps)] = pts_sets[ps][idx].astype(np.float64)
    # time per point for each case, then the step-weighted rate (equal points per case)
    per_pt = {}
    for _ in range(repeats):
        for key, p in samples.items():
            t0 = time.perf_counter()
            oracle.eval_sum(spec[key[0]], c64, p, nthreads=cores)
            dt = time.perf_counter() - t0
            per_pt[key] = min(per_pt.get(key, 1e30), dt / len(p))
    n_per_case = {("bcc_linear", "uniform"): N_UNIFORM, ("bcc_linear", "rays"): N_RAYS * RAY_STEPS,
                  ("bcc_quintic", "uniform"): N_UNIFORM, ("bcc_quintic", "rays"): N_RAYS * RAY_STEPS}
    step_time = sum(per_pt[k] * n_per_case[k] for k in per_pt)
    value = sum(n_per_case.values()) / step_time / 1e9
    sample = "; ".join(f"{k[0]}/{k[1]}: {ORACLE_SAMPLE[k[0]]} pts" for k in samples)
    return value, cores, sample, step_time


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2102_08518_b300.api import Spline, Volume

    coef_np, pts_np = make_inputs(seed_offset=rank)
    dev = torch.device("cuda", local)
    coef = torch.from_numpy(coef_np).to(dev)
    splines = {n: Spline(n, "f32") for n in ("bcc_linear", "bcc_quintic")}
    vols = {n: Volume(s, EXT, coef) for n, s in splines.items()}
    pts = {k: torch.from_numpy(v).to(dev) for k, v in pts_np.items()}
    outs = {k: torch.empty(v.shape[0], device=dev) for k, v in pts.items()}
    stream = torch.cuda.current_stream()

    def step(case_events=None):
        for ci, (sp, ps) in enumerate(CASES):
            if case_events is not None:
                case_events[ci][0].record(stream)
            vols[sp].eval(pts[ps], outs[ps])
            if case_events is not None:
                case_events[ci][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    case_events = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                    for _ in CASES] for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(case_events[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_total = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    ms_step = ms_total / args.steps
    pts_per_step = N_UNIFORM * 2 + N_RAYS * RAY_STEPS * 2
    value = pts_per_step * world / (ms_step * 1e-3) / 1e9
    case_ms = [statistics.mean(case_events[k][ci][0].elapsed_time(case_events[k][ci][1]) for k in range(args.steps))
               for ci in range(len(CASES))]
    per_case = {}
    for (sp, ps), ms in zip(CASES, case_ms):
        n = N_UNIFORM if ps == "uniform" else N_RAYS * RAY_STEPS
        per_case[f"{sp}/{ps}"] = {"gpoints_s": round(n / (ms * 1e-3) / 1e9, 3), "ms": round(ms, 4)}

    # roofline of the dominant kernel: the quintic on uniform points (FP32 FMA bound)
    info = splines["bcc_quintic"].info()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or 2032.0
    peak_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    dom_ms = per_case["bcc_quintic/uniform"]["ms"]
    achieved = 2.0 * info["fma_value"] * N_UNIFORM / (dom_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": "ls_eval__bcc_quintic_f32", "achieved": round(achieved, 3),
                "peak": round(peak_tflops, 2), "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                "traffic": None, "peak_source": f"FP32 FMA: {sms} SMs x 128 lanes x 2 flop x {max_mhz:.0f} MHz",
                "flops_per_point": 2 * info["fma_value"], "regs": info["regs_eval"]}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    host_pts = {k: torch.from_numpy(v).pin_memory() for k, v in pts_np.items()}
    host_out = {k: torch.empty(v.shape[0], dtype=torch.float32).pin_memory() for k, v in pts_np.items()}

    def e2e_step():
        for sp, ps in CASES:
            vols[sp].eval_host(host_pts[ps], host_out[ps])

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = sum(host_pts[ps].numel() * 4 for _, ps in CASES)
    d2h = sum(host_out[ps].numel() * 4 for _, ps in CASES)
    e2e = {"value": round(pts_per_step * world / e2e_s / 1e9, 4), "unit": "Gpoints/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    result = {"metric": METRIC, "value": round(value, 4), "unit": "Gpoints/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic",
              "config": {"workload": WORKLOAD, "points_per_step": pts_per_step, "coef_bytes": coef_np.nbytes,
                         "l2": "points 201 MB per set > 126 MB L2 (inputs larger than L2); coefficient volume "
                               "16 MiB L2-resident by design", "parallelism": f"replicas x{world}"},
              "per_case": per_case, "roofline": roofline, "e2e": e2e, "clocks": clocks,
              "gpu_launches": len(CASES) * args.steps}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = oracle_leg(coef_np, pts_np)
        result["cpu_baseline"] = {"value": round(v, 6), "unit": "Gpoints/s", "cores": cores, "kind": "oracle",
                                  "sample": sample}
    if world > 1:
        dist.destroy_process_group()
    return result if rank == 0 else None


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    coef_np, pts_np = make_inputs()
    for _ in range(args.warmup):
        pass
    vals = []
    t_all = 0.0
    v = cores = sample = None
    for _ in range(args.steps):
        v, cores, sample, st = oracle_leg(coef_np, pts_np)
        vals.append(v)
        t_all += st
    value = statistics.median(vals)
    ms = 1e3 * (N_UNIFORM * 2 + N_RAYS * RAY_STEPS * 2) / (value * 1e9)
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gpoints/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gpoints/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "Gpoints/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
