#!/usr/bin/env python
"""Throughput benchmark of the particle-inference hot path on GB300.

One step = one pass of the whole path on the line-fitting workload (Fig. 1,
§5.1 "linefitting"; synthetic data): 2^24 particles each run one trace over
256 data points (likelihood weighting, §3.6.2), the log-weights are normalised
(log-sum-exp, ESS), the weighted posterior is reduced (degree masses, per-degree
moments, mode), the population is resampled systematically with 64-bit
fixed-point weights, and the particle records are gathered.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  For N > 1 it is launched by torchrun; each rank
runs its own independent instance (Philox counter field `instance` = rank) with
no collective on the data path (weak scaling).  `--impl reference` times the
FP64 CPU oracle on the host cores instead, on a bounded sample of the same
workload per step.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PARTICLES = 1 << 24
N_POINTS = 256
DATA_SEED = 1
INFER_SEED = 1
METRIC = "particle-traces/sec"
UNIT = "traces/s"
WORKLOAD = ("linefitting likelihood weighting, 2^24 particles x 256 points, degree "
            "uniform{2..5}, coefficients N(0,10^2), sigma 0.5; + log-sum-exp/ESS + posterior "
            "reduce + systematic resampling (64-bit fixed point) + gather of 32-byte records")
KERNELS_PER_STEP = 5  # trace (posterior fused), max/LSE pass, scan, ancestors, gather


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--particles", type=int, default=N_PARTICLES,
                    help="particles per step (smaller cases for profiling only)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_index_for_smi(torch, local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        if uuid:
            return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    if vis:
        return vis.split(",")[local_rank]
    return str(local_rank)


# --------------------------------------------------------------------------
def cpu_baseline(n_sample=1 << 22):
    """The oracle (FP64 C) on a bounded sample of the same step, on all host cores."""
    import numpy as np

    import oracle
    import synth
    x, y = synth.poly_dataset(N_POINTS, DATA_SEED)
    m = oracle.poly_model()
    threads = oracle.get_threads()
    t0 = time.perf_counter()
    lw, n, c = oracle.is_poly(m, x, y, n_sample, INFER_SEED)
    oracle.posterior_poly(m, lw, n, c)
    st, anc = oracle.resample_from_lw(lw.astype(np.float32), n_sample, INFER_SEED)
    rec = np.zeros((n_sample, 8), dtype=np.float32)
    oracle.gather(rec, anc)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n_sample} particles x {N_POINTS} points, full step (traces, posterior, "
                      f"resample, gather), FP64 C with OpenMP over {threads} threads, "
                      f"{dt:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synth
    x, y = synth.poly_dataset(N_POINTS, DATA_SEED)
    m = oracle.poly_model()
    threads = oracle.get_threads()

    def step(n):
        lw, nn, c = oracle.is_poly(m, x, y, n, INFER_SEED)
        oracle.posterior_poly(m, lw, nn, c)
        _, anc = oracle.resample_from_lw(lw.astype(np.float32), n, INFER_SEED)
        oracle.gather(np.zeros((n, 8), dtype=np.float32), anc)

    t0 = time.perf_counter()
    step(1 << 16)
    per = (time.perf_counter() - t0) / (1 << 16)
    budget = 90.0  # seconds for the whole run
    n = int(max(1 << 12, min(1 << 22, budget / max(1, args.steps + args.warmup) / per)))
    for _ in range(args.warmup):
        step(n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(n)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = (f"{n} of the 2^24 particles per step, {N_POINTS} points, full step, FP64 C "
              f"oracle with OpenMP over {threads} threads")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "particles_per_step": n, "data_points": N_POINTS},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_2010_08454_gb300 as ppl
    import synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    ppl.lib()

    model = ppl.poly_model()
    x, y = synth.poly_dataset(N_POINTS, DATA_SEED)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.from_numpy(y).to(dev)
    N = args.particles
    instance = rank
    lw = torch.empty(N, dtype=torch.float32, device=dev)
    parts = ppl.poly_particles(N, dev)
    parts_out = ppl.poly_particles(N, dev)
    anc = torch.empty(N, dtype=torch.int32, device=dev)
    res = ppl.result_tensor(dev)
    ws = ppl.workspace(model, N, N_POINTS, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        ppl.ppl_infer_is_instance(model, xd, yd, N, INFER_SEED, instance, out=res, lw_out=lw,
                                  particles_out=parts, ws=ws)
        if ev:
            ev[1].record(stream)
            ev[2].record(stream)
        ppl.ppl_resample(N, INFER_SEED, instance, 0, lw=lw, ancestors=anc, ws=ws)
        if ev:
            ev[3].record(stream)
        ppl.ppl_gather(parts, anc, state_out=parts_out)
        if ev:
            ev[4].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    status = ppl.ppl_workspace_status(ws)
    summary = ppl.read_result(res)
    if status != 0 or summary["status"] != 0:
        raise RuntimeError(f"device status {status}/{summary['status']}")
    # algorithmic FP32 work of the factor, from this population's sampled degrees:
    # per particle and point, Horner (ncoef - 1 FMA) + residual (1 add) + square-accumulate (1 FMA)
    _, deg, _ = ppl.decode_particles(parts)
    counts = torch.bincount(deg.to(torch.int64) - 2, minlength=4).cpu().numpy()
    ncoef = np.arange(2, 6) + 1
    flops_per_launch = float(N_POINTS * np.sum(counts * (2 * (ncoef - 1) + 1 + 2)))

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_index_for_smi(torch, local))
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the previous step's lines from L2 (outside the events)
        step(events[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()

    stage = np.array([[ev[i].elapsed_time(ev[i + 1]) for i in range(4)] for ev in events])
    step_ms = stage.sum(axis=1)
    total_ms = float(step_ms.sum())
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * N * args.steps / (total_ms / 1e3)

    # end to end through the public API with host buffers: pinned H2D of the data,
    # the whole step, D2H of the posterior summary
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    res_h = torch.empty(ppl.RESULT_BYTES, dtype=torch.uint8).pin_memory()
    n_e2e = 0 if args.no_e2e else max(5, min(50, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        xd.copy_(xh, non_blocking=True)
        yd.copy_(yh, non_blocking=True)
        ppl.ppl_infer_is_instance(model, xd, yd, N, INFER_SEED, instance, out=res, lw_out=lw,
                                  particles_out=parts, ws=ws)
        ppl.ppl_resample(N, INFER_SEED, instance, 0, lw=lw, ancestors=anc, ws=ws)
        ppl.ppl_gather(parts, anc, state_out=parts_out)
        res_h.copy_(res, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * N * n_e2e / e2e_s if n_e2e else None  # every rank runs the same loop

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0

    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (peaks or {}).get("sm_max_mhz", 2070.0)
    # FP32 FMA peak: SMs x 128 lanes x 2 FLOP x max SM clock
    peak_tflops = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12
    trace_ms = float(stage[:, 0].mean())
    achieved = flops_per_launch / (trace_ms / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if N == N_PARTICLES else WORKLOAD.replace(
                       "2^24 particles", f"{N} particles"), "particles": N, "data_points": N_POINTS,
                   "data_seed": DATA_SEED, "seed": INFER_SEED, "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (256 MiB write outside the events)"},
        "roofline": {"kernel": "poly_trace_kernel", "bound": "alu", "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": None,
                     "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {max_mhz} MHz",
                     "work": "FP32 flops of the factor: L x (2 ncoef + 1) per trace"},
        "stages_ms": {"trace": trace_ms, "posterior": float(stage[:, 1].mean()),
                      "resample": float(stage[:, 2].mean()), "gather": float(stage[:, 3].mean())},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * N_POINTS * 4,
                "d2h_bytes_per_step": ppl.RESULT_BYTES, "steps": n_e2e},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
        "result": {"log_z": summary["log_z"], "ess": summary["ess"], "map_deg": summary["map_deg"]},
        "wall_s": t_wall,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
