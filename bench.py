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
KERNELS_PER_STEP = 2  # trace (normalisation and posterior fused), resampling (gather fused)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each of the step's kernels on the default workload, from an ncu capture of
# that kernel, with the SHA-256 prefix of the source files it was built from
# (its .cu and the headers it includes).  bench.py reports a figure only while
# the sources still have that digest, so a changed kernel reads null until it
# is captured again.
MEASURED_TRAFFIC = {
    "poly_trace_tc_kernel": {"bytes": 142293 + 538847232,
                             "sources": ["trace_tc.cu", "trace.cuh", "suffstat.cuh", "posterior.cuh",
                                         "dfloat.cuh", "poly.cuh", "rng.cuh", "kernels.h",
                                         "common.cuh"],
                             "sha256": "b4edf735f915de97"},
    "resample_coop_kernel": {"bytes": 68255829 + 545833685,
                             "sources": ["resample_coop.cu", "gridsync.cuh", "fixedpoint.cuh",
                                         "rng.cuh", "kernels.h", "common.cuh"],
                             "sha256": "ca89214dc1a464f8"},
}


def source_digest(sources):
    """First 16 hex digits of the SHA-256 of the kernel's source files (its .cu
    and every header it includes), in the listed order."""
    import hashlib
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2010_08454_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """The captured DRAM bytes of `kernel`, or None when any of its sources
    changed since the capture."""
    ent = MEASURED_TRAFFIC.get(kernel)
    if not ent or ent["bytes"] is None or ent["sha256"] is None:
        return None
    try:
        digest = source_digest(ent["sources"])
    except OSError:
        return None
    return ent["bytes"] if digest == ent["sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the state-space, batched and learned-proposal workloads")
    ap.add_argument("--particles", type=int, default=N_PARTICLES,
                    help="particles per step (smaller cases for profiling only)")
    ap.add_argument("--config", choices=["smc", "batched", "learned", "suffstat", "small",
                                         "normalise", "linefitting_small", "resample_normal"],
                    help="run only this secondary workload and print its line (profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(values, world, device=None):
    """The maximum over ranks of each value; every rank gets the result (one
    all-reduce of a few doubles, host timing only -- no data-path exchange)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def weak_scaling_value(world, units_per_rank, steps, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms / 1e3)


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
def cpu_baseline(n_sample=1 << 22, min_seconds=1.0, max_reps=8):
    """The oracle (FP64 C) on a bounded sample of the same step, on all host
    cores: the sample is repeated until it has run min_seconds (at least 10
    core-seconds on a many-core host), at most max_reps times."""
    import numpy as np

    import oracle
    import synth
    x, y = synth.poly_dataset(N_POINTS, DATA_SEED)
    m = oracle.poly_model()
    threads = oracle.get_threads()
    reps, dt = 0, 0.0
    while reps < max_reps and (reps == 0 or dt < min_seconds):
        t0 = time.perf_counter()
        lw, n, c = oracle.is_poly(m, x, y, n_sample, INFER_SEED)
        oracle.posterior_poly(m, lw, n, c)
        st, anc = oracle.resample_from_lw(lw.astype(np.float32), n_sample, INFER_SEED)
        rec = np.zeros((n_sample, 8), dtype=np.float32)
        oracle.gather(rec, anc)
        dt += time.perf_counter() - t0
        reps += 1
    return {"value": reps * n_sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{reps} x {n_sample} particles x {N_POINTS} points, full step (traces, "
                      f"posterior, resample, gather), FP64 C with OpenMP over {threads} "
                      f"threads, {dt:.2f} s in all"}


# --------------------------------------------------------------------------
# The other workloads of the path, measured in the same run (rank 0).
# --------------------------------------------------------------------------
def _event_ms(torch, fn, reps):
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _device_ms(torch, fn, reps, flush=None):
    """Median device time of one call of fn: all calls are enqueued behind a
    device-side sleep, so the host's launch path never leaves the GPU idle
    between a call's two events; the L2 is flushed before every call, outside
    its events."""
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    torch.cuda.synchronize()
    torch.cuda._sleep(int(2e6 + reps * 4e5))  # ~1 ms + 0.2 ms per call at 2 GHz
    for k in range(reps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        ev[k][0].record(s)
        fn()
        ev[k][1].record(s)
    torch.cuda.synchronize()
    return float(statistics.median(a.elapsed_time(b) for a, b in ev))


def bench_smc(torch, ppl, reps=5):
    """Bootstrap filter on the linear-Gaussian model, T = 200, 2^20 particles: one persistent
    kernel, with the step-by-step path (one CUDA graph of 200 steps) timed beside it."""
    import numpy as np

    import synth
    N, T = 1 << 20, 200
    y = synth.lgssm_dataset(T, 2)
    model = ppl.lgssm_model()
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    lw = torch.zeros_like(x)
    acc = torch.zeros(1, dtype=torch.float64, device="cuda")
    flags = torch.zeros(T, dtype=torch.int32, device="cuda")
    est = torch.zeros((T, 2), dtype=torch.float64, device="cuda")
    ws = ppl.workspace(model, N, T)

    def run_steps():
        for t in range(1, T + 1):
            ppl.ppl_smc_step(model, float(y[t - 1]), t, 2, x, lw, acc, flags[t - 1:t], est[t - 1],
                             ws)

    def reset():
        x.zero_()
        lw.zero_()
        acc.zero_()

    reset()
    run_steps()  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cs):
        run_steps()
    times = []
    for _ in range(reps):
        reset()
        torch.cuda.synchronize()
        times.append(_event_ms(torch, g.replay, 1))
    ms_steps = float(np.median(times))
    logz_steps = float(est[-1, 0])
    # the same filter as one persistent cooperative kernel
    y_dev = torch.from_numpy(y).cuda()
    out = ppl.ppl_smc_run(model, y_dev, N, 2, ws=ws)
    torch.cuda.synchronize()
    times = [_event_ms(torch, lambda: ppl.ppl_smc_run(model, y_dev, N, 2, ws=ws, out=out), 1)
             for _ in range(reps)]
    assert ppl.ppl_workspace_status(ws) == 0
    ms = float(np.median(times))
    logz = float(out["log_z"].item())
    n_res = int(out["resampled"].sum().item())
    # the step separators alone: the filter's grid barriers (one per step, two
    # more per resampling step) at its launch shape, with no work between them
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per_thread = next(r for r in range(1, 9) if -(-N // (1024 * r)) <= sms)
    blocks = -(-N // (1024 * per_thread))
    n_bar = T + 2 * n_res
    bws = ppl.ppl_grid_barrier_probe(blocks, n_bar)
    bar_ms = float(np.median([_event_ms(torch, lambda: ppl.ppl_grid_barrier_probe(blocks, n_bar,
                                                                                  ws=bws), 1)
                              for _ in range(reps)]))
    assert ppl.ppl_workspace_status(bws) == 0
    import oracle
    kal = oracle.kalman_logz(oracle.lgssm_model(), y)
    return {"workload": "bootstrap filter, linear-Gaussian SSM, T=200, 2^20 particles, FP32 "
                        "state, resample when ESS < N/2; all 200 steps in one persistent "
                        "cooperative kernel",
            "metric": "particle-steps/sec", "value": N * T / (ms / 1e3), "unit": "particle-steps/s",
            "ms_per_filter": ms, "resampling_steps": n_res,
            "grid_barriers": {"count": n_bar, "blocks": blocks, "ms_alone": bar_ms,
                              "us_per_barrier": 1e3 * bar_ms / n_bar,
                              "frac_of_filter": bar_ms / ms},
            "log_z": logz, "kalman_log_z": kal, "abs_err_vs_kalman": abs(logz - kal),
            "gpu_launches_per_filter": 1,
            "stepwise_graph": {"ms_per_filter": ms_steps, "log_z": logz_steps,
                               # per step: propagate, resampling with the
                               # state gather fused, commit
                               "gpu_launches_per_filter": 3 * T,
                               "same_particles": bool(torch.equal(out["x"], x))}}


def bench_linefitting_small(torch, ppl, replays=100):
    """The paper's line-fitting example at its own size (Fig. 1, §1.1): 32
    points from seed 0, 10^5 particles, inference seed 0; one call (trace,
    normalisation, posterior) captured in a CUDA graph and replayed."""
    import numpy as np

    import synth
    N, L = 100000, 32
    x, y = synth.poly_dataset(L, 0)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    model = ppl.poly_model()
    ws = ppl.workspace(model, N, L)
    res = ppl.result_tensor()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    parts = ppl.poly_particles(N)

    def call():
        ppl.ppl_infer_is_instance(model, xd, yd, N, 0, 0, out=res, lw_out=lw, particles_out=parts,
                                  ws=ws)
    call()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cs):
        call()
    g.replay()
    torch.cuda.synchronize()
    ms = _event_ms(torch, g.replay, replays)
    r = ppl.read_result(res)
    return {"workload": "linefitting likelihood weighting, 32 points (data seed 0), 10^5 "
                        "particles (seed 0), records and log-weights written; one graph replay "
                        "per call, inputs resident (64 KB of data and 3.6 MB of outputs stay in L2)",
            "metric": "particle-traces/sec", "value": N / (ms / 1e3), "unit": "traces/s",
            "ms_per_call": ms, "replays": replays, "log_z": r["log_z"], "status": r["status"],
            "gpu_launches_per_call": 1}


def bench_resample_normal(torch, ppl, reps=20):
    """The fused resampling + gather on a non-degenerate population: 2^24
    unit-variance normal log-weights (ESS about N/e, so most outputs start a
    new ancestor and the merge path does the work), 32-byte records, against
    the measured HBM bandwidth; L2 flushed before every timed call."""
    import numpy as np

    import synth
    N = 1 << 24
    lw = torch.from_numpy(synth.log_weights(N, 21, "normal", scale=1.0)).cuda()
    rec = torch.from_numpy(np.random.default_rng(5).standard_normal((N, 8)).astype(np.float32)).cuda()
    out = torch.empty_like(rec)
    anc = torch.empty(N, dtype=torch.int32, device="cuda")
    ws = ppl.workspace(ppl.poly_model(), N, 0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def call():
        ppl.ppl_resample_gather(N, 1, lw, rec, state_out=out, ancestors=anc, ws=ws)
    for _ in range(3):
        call()
    ms = _device_ms(torch, call, reps, flush)
    assert ppl.ppl_workspace_status(ws) == 0
    distinct = int(torch.unique(anc).numel())
    algo = N * (4 + 4 + 32) + distinct * 32
    peak = (load_peaks() or {}).get("hbm_gbs")
    gbs = algo / (ms / 1e3) / 1e9
    return {"workload": "systematic resampling (64-bit fixed point) + gather of 32-byte records, "
                        "2^24 particles, lw ~ N(0, 1) (ESS near N/e); the maximum found by the "
                        "statistics pass inside the call",
            "metric": "GB/s (algorithmic)", "value": gbs, "unit": "GB/s", "ms_per_call": ms,
            "bytes_per_call": algo, "distinct_ancestors": distinct, "hbm_peak_gbs": peak,
            "frac": gbs / peak if peak else None,
            "work": "lw 4 B in, ancestor 4 B and record 32 B out per particle; each distinct "
                    "ancestor's record in (the statistics pass re-reads lw: not counted)",
            "gpu_launches_per_call": 2}


def bench_suffstat(torch, ppl, reps=10):
    """The line-fitting workload (2^24 particles x 256 points) with the factor
    from the data's sufficient statistics (a separate variant: the headline
    counts the point-by-point FLOPs)."""
    import numpy as np

    import synth
    N = N_PARTICLES
    x, y = synth.poly_dataset(N_POINTS, DATA_SEED)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    model = ppl.poly_model()
    lw = torch.empty(N, dtype=torch.float32, device="cuda")
    parts = ppl.poly_particles(N)
    ws = ppl.workspace(model, N, N_POINTS)
    res = ppl.result_tensor()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    times = {}
    for name, fn in (("suffstat", ppl.ppl_infer_is_suffstat), ("direct", ppl.ppl_infer_is_instance)):
        def call():
            fn(model, xd, yd, N, INFER_SEED, 0, out=res, lw_out=lw, particles_out=parts, ws=ws)
        for _ in range(3):
            call()
        t = []
        for _ in range(reps):
            flush.fill_(1)
            t.append(_event_ms(torch, call, 1))
        times[name] = float(np.median(t))
    summary = ppl.read_result(res)
    return {"workload": "likelihood weighting, 2^24 particles x 256 points, factor from the "
                        "sufficient statistics (one Cholesky of the 6 x 6 Gram matrix, O(d^2) "
                        "per trace); records and log-weights written as in the headline step",
            "metric": "particle-traces/sec", "value": N / (times["suffstat"] / 1e3),
            "unit": "traces/s", "ms_per_launch": times["suffstat"],
            "direct_ms_per_launch": times["direct"], "log_z": summary["log_z"],
            "gpu_launches_per_call": 2}


def bench_normalise(torch, ppl, reps=20):
    """The normalisation pass on its own (ppl_logsumexp: max, log-sum-exp, ESS
    and argmax of 2^24 FP32 log-weights, one read of lw), against the measured
    HBM bandwidth; L2 flushed before every timed call."""
    import numpy as np

    import synth
    N = N_PARTICLES
    lw = torch.from_numpy(synth.log_weights(N, 12, "normal", scale=20.0)).cuda()
    ws = ppl.workspace(ppl.poly_model(), N, 0)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ppl.ppl_logsumexp(lw, out=out, ws=ws)
    ms = _device_ms(torch, lambda: ppl.ppl_logsumexp(lw, out=out, ws=ws), reps, flush)
    gbs = N * 4 / (ms / 1e3) / 1e9
    peak = (load_peaks() or {}).get("hbm_gbs")
    return {"workload": "log-sum-exp, ESS, max and argmax of 2^24 FP32 log-weights "
                        "(one pass; the headline step fuses it into the trace kernel)",
            "metric": "GB/s of log-weights read", "value": gbs, "unit": "GB/s",
            "ms_per_call": ms, "hbm_peak_gbs": peak, "frac": gbs / peak if peak else None,
            "gpu_launches_per_call": 1}


def bench_small_models(torch, ppl, reps=10):
    """The paper's other importance-sampling benchmarks (Table 1): biasedcoin,
    binomial, a truncated geometric and customdist, 2^24 particles each."""
    import numpy as np
    N = 1 << 24
    rng = np.random.default_rng(12)
    flips = torch.tensor((rng.random(200) < 0.7).astype(np.int32), device="cuda")
    y = torch.tensor(rng.normal(1.0, 1.0, 8).astype(np.float32), device="cuda")
    ws = ppl.workspace(ppl.poly_model(), N, 0)
    cm = ppl.customdist_model()
    runs = {
        "biasedcoin_200_flips": lambda: ppl.ppl_infer_discrete("biasedcoin", N, 1, flips=flips, ws=ws),
        "binomial_10_trials": lambda: ppl.ppl_infer_discrete("binomial", N, 1, limit=10, ws=ws),
        "geometric_depth_12": lambda: ppl.ppl_infer_discrete("geometric", N, 1, limit=12, ws=ws),
        "customdist_8_obs": lambda: ppl.ppl_infer_customdist(cm, y, N, 1, ws=ws),
    }
    out = {}
    for name, fn in runs.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms = float(np.median([_event_ms(torch, fn, 1) for _ in range(reps)]))
        out[name] = {"ms_per_call": ms, "traces_per_s": N / (ms / 1e3)}
    return {"workload": "likelihood weighting, 2^24 particles per model; each call includes its "
                        "result's device-to-host copy (the binding decodes it)",
            "metric": "particle-traces/sec", "unit": "traces/s", "models": out,
            "gpu_launches_per_call": 1}


def bench_batched(torch, ppl, reps=5):
    """4096 uneven line-fitting instances in one persistent launch, autotuned, graph-replayed."""
    import numpy as np

    import synth
    inst = synth.batched_instances(4096, 3)
    model = ppl.poly_model()
    x, y = torch.from_numpy(inst["x"]).cuda(), torch.from_numpy(inst["y"]).cuda()
    doff = torch.from_numpy(inst["data_off"]).cuda()
    poff = torch.from_numpy(inst["part_off"]).cuda()
    ws = ppl.batched_workspace(inst["data_off"], inst["part_off"])
    out = ppl.batch_results_tensor(4096)
    cache = os.path.join(ROOT, "paper_2010_08454_gb300", "_build", "batched_tune.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    plan = ppl.ppl_batched_autotune(model, x, y, doff, poff, inst["data_off"], inst["part_off"],
                                    3, out, ws, cache)
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    ppl.ppl_infer_is_batched(model, x, y, doff, poff, 3, plan, out, ws)
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=cs):
        ppl.ppl_infer_is_batched(model, x, y, doff, poff, 3, plan, out, ws)
    g.replay()
    torch.cuda.synchronize()
    ms = _event_ms(torch, g.replay, reps)
    res = ppl.read_batch_results(out, 4096)
    status = max(r["status"] for r in res)
    n_traces = int(inst["part_off"][-1])
    # expected FP32 flops of the factor under the degree prior: (2 ncoef + 1), mean ncoef 4.5
    flops = float(plan.work) * 10.0
    peaks = load_peaks()
    fp32_peak = (torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 *
                 (peaks or {}).get("sm_max_mhz", 2070.0) * 1e6 / 1e12)
    return {"workload": "4096 line-fitting instances, data lengths log-uniform [16, 4096], "
                        "particles log-uniform [2^10, 2^16], one persistent launch in a CUDA graph",
            "metric": "particle-traces/sec", "value": n_traces / (ms / 1e3), "unit": "traces/s",
            "ms_per_launch": ms, "traces": n_traces, "trace_points": float(plan.work),
            "fp32_tflops": flops / (ms / 1e3) / 1e12,
            # against the FP32 FMA peak: SMs x 128 lanes x 2 FLOP x max SM clock
            "fp32_peak_tflops": fp32_peak,
            "frac": flops / (ms / 1e3) / 1e12 / fp32_peak,
            "autotuned": {"ppt": plan.ppt, "blocks_per_sm": plan.blocks_per_sm},
            "items": int(plan.n_items), "status": status}


def bench_learned(torch, ppl, epochs=4, n_sets=1024, N=1 << 20, reps=3, n_pairs=1 << 22):
    """Learned vs prior proposal: ESS/sec at |delta log Z| < 0.05 on held-out data sets."""
    import numpy as np

    import oracle
    import synth
    model = ppl.poly_model()
    params = ppl.pack_params(synth.mlp_weights(1))
    am, av = torch.zeros_like(params), torch.zeros_like(params)
    batch = 1024
    steps = epochs * (n_pairs // batch)
    block = 64  # training steps per CUDA graph replay
    pws = ppl.proposal_workspace(batch)
    # first-call set-up outside the capture, on scratch copies
    sp, sm, sv = params.clone(), am.clone(), av.clone()
    ppl.ppl_proposal_train_init(sp, batch, pws)
    ppl.ppl_proposal_train_steps(model, sp, sm, sv, n_pairs, batch, 1, 99, 1e-3, None, pws)
    ppl.ppl_proposal_train_init(params, batch, pws)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ppl.ppl_proposal_train_steps(model, params, am, av, n_pairs, batch, block, 99, 1e-3,
                                     None, pws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps // block):
        graph.replay()
    ev1.record()
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    train_ms = ev0.elapsed_time(ev1)
    if ppl.ppl_workspace_status(pws) != 0:
        raise RuntimeError("training: device status")
    # FLOPs of a step: forward 64x256 + 256x256 + 256x48 multiply-adds per
    # pair, and twice that backward (weight and input gradients)
    step_flops = 3 * 2 * (64 * 256 + 256 * 256 + 256 * 48) * batch
    bf16 = (load_peaks() or {}).get("bf16_tflops")
    d = synth.prior_datasets(n_sets, 32, 4)
    x, y = torch.from_numpy(d["x"]).cuda(), torch.from_numpy(d["y"]).cuda()
    xf, yf = x.reshape(-1).contiguous(), y.reshape(-1).contiguous()
    doff_h = np.arange(n_sets + 1, dtype=np.int64) * 32
    poff_h = np.arange(n_sets + 1, dtype=np.int64) * N
    doff, poff = torch.from_numpy(doff_h).cuda(), torch.from_numpy(poff_h).cuda()
    ws = ppl.batched_workspace(doff_h, poff_h)
    plan = ppl.ppl_batched_prepare(model, doff_h, poff_h, 8, 2, ws)
    pws = ppl.proposal_workspace(n_sets)
    prop = torch.empty((n_sets, 48), dtype=torch.float32, device="cuda")
    out_l, out_p = ppl.batch_results_tensor(n_sets), ppl.batch_results_tensor(n_sets)

    def learned():
        ppl.ppl_proposal_forward(model, params, x, y, out=prop, ws=pws)
        ppl.ppl_infer_is_learned(model, xf, yf, doff, poff, 5, plan, prop, out_l, ws)

    def prior():
        ppl.ppl_infer_is_batched(model, xf, yf, doff, poff, 5, plan, out_p, ws)

    learned()
    prior()
    ms_l = _event_ms(torch, learned, reps)
    ms_p = _event_ms(torch, prior, reps)
    rl, rp = ppl.read_batch_results(out_l, n_sets), ppl.read_batch_results(out_p, n_sets)
    om = oracle.poly_model()
    exact = np.array([oracle.poly_exact(om, d["x"][b], d["y"][b])["log_z"] for b in range(n_sets)])
    el = np.abs(np.array([r["log_z"] for r in rl]) - exact)
    ep = np.abs(np.array([r["log_z"] for r in rp]) - exact)
    ess_l = np.array([r["ess"] for r in rl])
    ess_p = np.array([r["ess"] for r in rp])
    ok_l, ok_p = el < 0.05, ep < 0.05
    return {"workload": f"{n_sets} held-out data sets from the model (32 points), {N} particles "
                        f"each; proposal network trained on {n_pairs} forward-simulated pairs x "
                        f"{epochs} epochs",
            "metric": "ESS/sec at |delta log Z| < 0.05", "unit": "ESS/s",
            "learned": {"ess_per_sec": float(ess_l.sum() / (ms_l / 1e3)),
                        "ess_per_sec_at_tol": float(ess_l[ok_l].sum() / (ms_l / 1e3)),
                        "frac_within_0.05": float(ok_l.mean()), "median_abs_err": float(np.median(el)),
                        "median_ess": float(np.median(ess_l)), "ms": ms_l},
            "prior": {"ess_per_sec": float(ess_p.sum() / (ms_p / 1e3)),
                      "ess_per_sec_at_tol": float(ess_p[ok_p].sum() / (ms_p / 1e3)),
                      "frac_within_0.05": float(ok_p.mean()), "median_abs_err": float(np.median(ep)),
                      "median_ess": float(np.median(ess_p)), "ms": ms_p},
            "train_seconds": train_s, "train_steps": steps,
            "train": {"ms_per_step": train_ms / steps, "graph_block_steps": block,
                      "tflops": step_flops * steps / (train_ms / 1e3) / 1e12,
                      "bf16_peak_tflops": bf16,
                      "frac": (step_flops * steps / (train_ms / 1e3) / 1e12 / bf16) if bf16 else None,
                      "work": "3 x 2 x (64 x 256 + 256 x 256 + 256 x 48) FLOP per pair, "
                              "1024 pairs per step",
                      "timing": "CUDA events around the graph replays of all steps"}}


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
    max_lw = ppl.result_max_lw(res)
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
        ppl.ppl_resample_gather(N, INFER_SEED, lw, parts, max_lw_dev=max_lw, instance=instance,
                                t=0, state_out=parts_out, ancestors=anc, ws=ws)
        if ev:
            ev[3].record(stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    status = ppl.ppl_workspace_status(ws)
    summary = ppl.read_result(res)
    if status != 0 or summary["status"] != 0:
        raise RuntimeError(f"device status {status}/{summary['status']}")
    # algorithmic work of the factor, from this population's sampled degrees.
    # The trace kernel forms every residual y - f(x) as a product on the
    # tensor cores: per trace and point, ncoef coefficient columns and the y
    # column, each as three TF32 products (hi hi, hi lo, lo hi) for an
    # FP32-accurate result.  The same factor on FP32 cores would take Horner
    # (ncoef - 1 FMA) + residual (1 add) + square-accumulate (1 FMA).
    _, deg, _ = ppl.decode_particles(parts)
    counts = torch.bincount(deg.to(torch.int64) - 2, minlength=4).cpu().numpy()
    ncoef = np.arange(2, 6) + 1
    tc_flops_per_launch = float(3 * 2 * N_POINTS * np.sum(counts * (ncoef + 1)))
    fp32_flops_per_launch = float(N_POINTS * np.sum(counts * (2 * (ncoef - 1) + 1 + 2)))

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
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

    stage = np.array([[ev[i].elapsed_time(ev[i + 1]) for i in range(3)] for ev in events])
    step_ms = stage.sum(axis=1)
    (total_ms,) = reduce_max([float(step_ms.sum())], world, dev)
    value = weak_scaling_value(world, N, args.steps, total_ms)

    # end to end through the public API with host buffers, as a serving loop:
    # every step copies its data set in from pinned host memory and its
    # posterior summary out to its own pinned slot; the host enqueues the next
    # step while the device runs (stream order keeps each step's buffers
    # intact), waits once at the end, and then checks every step's summary
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    n_e2e = 0 if args.no_e2e else max(5, min(50, args.steps))
    res_h = torch.empty((max(n_e2e, 1), ppl.RESULT_BYTES), dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        xd.copy_(xh, non_blocking=True)
        yd.copy_(yh, non_blocking=True)
        ppl.ppl_infer_is_instance(model, xd, yd, N, INFER_SEED, instance, out=res, lw_out=lw,
                                  particles_out=parts, ws=ws)
        ppl.ppl_resample_gather(N, INFER_SEED, lw, parts, max_lw_dev=max_lw, instance=instance,
                                t=0, state_out=parts_out, ancestors=anc, ws=ws)
        res_h[k].copy_(res, non_blocking=True)
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - t0
    for k in range(n_e2e):
        r = ppl.read_result(res_h[k])
        if r["status"] != 0 or r["log_z"] != summary["log_z"]:
            raise RuntimeError(f"end-to-end step {k}: status {r['status']}, log Z {r['log_z']}")
    (e2e_s,) = reduce_max([e2e_wall], world, dev)
    e2e_value = weak_scaling_value(world, N, n_e2e, e2e_s * 1e3) if n_e2e else None

    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return 0

    # the fused resampling + gather stage against HBM: algorithmic bytes = lw
    # read, ancestors and records written, each distinct ancestor's record read
    rec_bytes = parts[0].numel() * parts.element_size()
    distinct = int(torch.unique(anc).numel())
    rg_bytes = N * (4 + 4 + rec_bytes) + distinct * rec_bytes
    rg_ms = float(stage[:, 2].mean())
    peaks = load_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = (peaks or {}).get("sm_max_mhz", 2070.0)
    # FP32 FMA peak: SMs x 128 lanes x 2 FLOP x max SM clock
    peak_tflops = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12
    # TF32 tensor peak: the measured BF16 burst figure x the nominal dense
    # TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)
    bf16 = (peaks or {}).get("bf16_tflops")
    tf32_peak = (bf16 if bf16 else 1900.0) * 1.1 / 2.25
    trace_ms = float(stage[:, 0].mean())
    achieved = tc_flops_per_launch / (trace_ms / 1e3) / 1e12
    achieved_fp32 = fp32_flops_per_launch / (trace_ms / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if N == N_PARTICLES else WORKLOAD.replace(
                       "2^24 particles", f"{N} particles"), "particles": N, "data_points": N_POINTS,
                   "data_seed": DATA_SEED, "seed": INFER_SEED, "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (256 MiB write outside the events)"},
        "roofline": {"kernel": "poly_trace_tc_kernel", "bound": "tensor", "achieved": achieved,
                     "peak": tf32_peak, "unit": "TFLOP/s", "frac": achieved / tf32_peak,
                     "traffic": measured_traffic("poly_trace_tc_kernel")
                     if N == N_PARTICLES else None,
                     "traffic_unit": "bytes per launch",
                     "peak_source": ("TF32 dense: measured BF16 burst x 1.1/2.25 (nominal ratio), "
                                     "of measured") if bf16 else "fallback BF16 x 1.1/2.25",
                     "work": "TF32 flops of the residual products: 3 (split) x 2 x L x (ncoef + 1) "
                             "per trace, from the sampled degrees",
                     "timing": "CUDA events around ppl_infer_is_instance on its stream (two "
                               "512-byte memsets and the trace kernel)"},
        "roofline_fp32_equivalent": {
            "kernel": "poly_trace_tc_kernel", "bound": "alu", "achieved": achieved_fp32,
            "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved_fp32 / peak_tflops,
            "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 x {max_mhz} MHz",
            "work": "the factor as FP32 Horner would count it: L x (2 ncoef + 1) per trace"},
        "stages_ms": {"trace": trace_ms, "posterior": float(stage[:, 1].mean()),
                      "resample_gather": rg_ms},
        "roofline_resample_gather": {
            "kernel": "resample_coop_kernel (gather fused)", "bound": "hbm",
            "achieved": rg_bytes / (rg_ms / 1e3) / 1e9,
            "peak": (peaks or {}).get("hbm_gbs", 6800.0), "unit": "GB/s",
            "frac": rg_bytes / (rg_ms / 1e3) / 1e9 / (peaks or {}).get("hbm_gbs", 6800.0),
            "peak_source": "measured copy bandwidth" if peaks else "fallback",
            "bytes_per_step": rg_bytes, "distinct_ancestors": distinct,
            "traffic": measured_traffic("resample_coop_kernel") if N == N_PARTICLES else None,
            "traffic_unit": "bytes per launch",
            "work": "lw 4 B in, ancestor 4 B and record out per particle; each distinct "
                    "ancestor's record in"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * N_POINTS * 4,
                "d2h_bytes_per_step": ppl.RESULT_BYTES, "steps": n_e2e},
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "clocks": clocks,
        "result": {"log_z": summary["log_z"], "ess": summary["ess"], "map_deg": summary["map_deg"]},
        "wall_s": t_wall,
    }
    if not args.no_configs:
        out["configs"] = {"linefitting_1e5x32": bench_linefitting_small(torch, ppl),
                          "resample_gather_2e24_normal": bench_resample_normal(torch, ppl),
                          "smc_lgssm_T200_2e20": bench_smc(torch, ppl),
                          "suffstat_linefitting_2e24x256": bench_suffstat(torch, ppl),
                          "small_models_2e24": bench_small_models(torch, ppl),
                          "normalise_2e24": bench_normalise(torch, ppl),
                          "batched_4096": bench_batched(torch, ppl),
                          "learned_proposal_1024x2e20": bench_learned(torch, ppl)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    return 0


def run_config(args):
    import torch

    import paper_2010_08454_gb300.binding as ppl
    torch.cuda.set_device(0)
    ppl.lib()
    fn = {"smc": bench_smc, "batched": bench_batched, "learned": bench_learned,
          "suffstat": bench_suffstat, "small": bench_small_models,
          "normalise": bench_normalise, "linefitting_small": bench_linefitting_small,
          "resample_normal": bench_resample_normal}[args.config]
    print(json.dumps({"config": args.config, "result": fn(torch, ppl)}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config:
        return run_config(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
