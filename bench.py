#!/usr/bin/env python
"""Throughput of the MIPWA likelihood hot path on one GB300 (or N replicas).

One step = one NLL + gradient evaluation (kinematics, Breit-Wigner terms,
spline setup and evaluation, Bose-symmetrised |A|^2, log, normalisation sum,
-2 ln L, adjoint gradient) over the whole workload:

  D+ -> pi- pi+ pi+, rho(770) P-wave + f2(1270) D-wave + 40-knot MIPWA S-wave,
  10^8 accept-reject data events + 10^8 uniform normalisation events stored as
  float32 (s12, s13), FP32-mixed arithmetic (FP64 spline solve and accumulators).

The same events are also timed in the plain FP64 form ("fp64_plain"), end to
end from pinned host buffers ("e2e"), and the FP64 oracle on the host cores
("cpu_baseline"). ``--impl reference`` times the oracle alone.

Prints one JSON line (rank 0).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s per NLL+grad eval (FP32-mixed vs FP64 plain, same GB300); % roofline"
WORKLOAD = ("pipipi_n40_1e8_f32: D+->pi-pi+pi+, rho(770) P + f2(1270) D + 40-knot spline "
            "S-wave, 1e8 accept-reject data + 1e8 uniform normalisation events, float32 "
            "(s12,s13)")


def workload_name(n):
    """The workload string for n data + n normalisation events (the default is 1e8)."""
    if n == 100_000_000:
        return WORKLOAD
    return WORKLOAD.replace("1e8", f"{n:.0e}".replace("+0", "").replace("+", ""))

# Algorithmic work per event (flops; add/sub/mul/div/sqrt/sin/cos/log = 1
# each): the FP64 oracle's own formulas instantiated on an operation-counting
# scalar type (oracle_count_flops), counting the operations that depend on the
# event once each, on this model at these parameters, averaged over PDF-drawn
# data and uniform normalisation events in equal numbers (a test recounts
# them). FWD: -2 ln L only; GRAD: with the gradient's per-event part (weighted
# adjoint, coefficient sums, segment bins); CACHED: the Breit-Wigner basis read
# instead of computed; REIM: the Re/Im S-wave form.
FLOPS_PER_EVENT_FWD = 260.0
FLOPS_PER_EVENT_GRAD = 353.0
FLOPS_PER_EVENT_GRAD_CACHED = 179.0
FLOPS_PER_EVENT_GRAD_REIM = 331.0
FLOPS_PER_EVENT_GRAD_REIM_CACHED = 157.0
# Peaks from unit counts and the maximum SM clock (2070 MHz, 152 SMs), for
# context beside the measured ones: FP32 128 lanes x 2 flop x 152 x 2.07 GHz;
# FP64 1.25 TFLOP/s (GB300 nominal).
PEAK_FP32_TFLOPS = 128 * 2 * 152 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


def _measured_hbm_gbs() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0  # fallback figure for a GB300


HBM_GBS = _measured_hbm_gbs()
# DRAM bytes (read + write) of the fused FP32 NLL+gradient kernel per event
# processed, from one ncu capture on 2e7 + 2e7 events (320.26 MB read + 4.68
# MB written per launch); a launch's traffic is this times its events. None
# once the kernel has changed since the capture.
TRAFFIC_PER_EVENT = (320.259584e6 + 4.678144e6) / 4e7
# The same for the cached-basis kernel (960.15 MB read + 5.28 MB written for
# 2e7 + 2e7 events with their cached Breit-Wigner terms).
TRAFFIC_PER_EVENT_CACHED = (960.150272e6 + 5.282816e6) / 4e7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-events", type=int, default=100_000_000,
                    help="data events (= normalisation events)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--nll-steps", type=int, default=50, help="NLL-only (no gradient) steps")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cached-steps", type=int, default=10)
    ap.add_argument("--toys-steps", type=int, default=3)
    ap.add_argument("--reim-steps", type=int, default=10)
    ap.add_argument("--n-toys", type=int, default=256)
    ap.add_argument("--toys-norm", type=int, default=10_000_000)
    ap.add_argument("--toys-config", type=str, default="",
                    help="norm_chunk,data_chunk,block,blocks_per_sm for the batched toys "
                         "instead of the autotuner's choice")
    ap.add_argument("--paper-fit", type=int, default=1,
                    help="run the Sec. 4 workload (K K K, 40 knots, 100K toys) as full fits")
    ap.add_argument("--paper-toys", type=int, default=20,
                    help="toys fitted at each normalisation grid spacing (Fig. 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi every 25 ms in a child process; a reader thread stamps each
    sample on arrival, and stop() keeps the samples that arrived between
    begin() and end() (plus one sampling period), i.e. during the timed loop."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.025

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.rows = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), line))

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(int(self.PERIOD_S * 1000))],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.perf_counter() + 5.0  # wait for the first sample
        while not self.rows and time.perf_counter() < deadline and self.proc.poll() is None:
            time.sleep(0.02)

    def begin(self):
        self.t0 = time.perf_counter()

    def end(self):
        self.t1 = time.perf_counter()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(self.PERIOD_S)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        rows = []
        for t, line in self.rows:
            if self.t0 is not None and not (self.t0 <= t <= self.t1 + self.PERIOD_S):
                continue
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows), "timed_s": round(self.t1 - self.t0, 3)}


# ------------------------------------------------------------- distributed
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def bench_config(n: int, world: int) -> dict:
    """The workload of one step (the same dict for both arms)."""
    return {"workload": workload_name(n), "n_data": n, "n_norm": n,
            "l2": (f"inputs ({16 * n / 1e9:.2g} GB) larger than L2 (129 MB); no flush needed"
                   if 16 * n > 129e6 else "inputs fit in L2 (129 MB): not a valid bench size"),
            "parallelism": f"replicas x{world} (no collective)"}


# ------------------------------------------------------------- ALU peaks
def probe_peaks(local: int) -> dict:
    """The library's throughput probes (mipwa_probe_peak) on this GPU: FP32
    FMA (scalar and packed f32x2), FP64 FMA and the special-function unit,
    each timed with CUDA events for about 200 ms, with the SM clocks sampled
    during the probes."""
    from paper_1703_03284_gb300.api import probe_peak
    clocks = ClockSampler(local)
    clocks.start()
    clocks.begin()
    out = {}
    for kind in ("ffma", "ffma2", "dfma", "mufu"):
        probe_peak(kind, local, 20.0)  # warm-up
        ops, ms = probe_peak(kind, local, 200.0)
        out[kind] = {"ops_per_s": ops, "ms": ms,
                     "unit": "approximations/s" if kind == "mufu" else "flop/s"}
    clocks.end()
    out["clocks"] = clocks.stop()
    out["fp32_tflops"] = max(out["ffma"]["ops_per_s"], out["ffma2"]["ops_per_s"]) / 1e12
    out["fp64_tflops"] = out["dfma"]["ops_per_s"] / 1e12
    out["note"] = ("grid of SMs x 4 blocks x 256 threads, 8 independent chains per thread; "
                   "fma = 2 flops, packed f32x2 fma = 4")
    return out


# ------------------------------------------------------------- CPU oracle
def oracle_sample(spec, n: int, seed: int):
    """Data and normalisation samples drawn with the oracle's own density."""
    import numpy as np
    import torch

    import oracle
    import synth
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    data = synth.accept_reject(spec, n, synth.numpy_density(lambda x: o.density(truth, x)),
                               seed=seed, dtype=torch.float32).numpy().astype(np.float64)
    norm = synth.uniform_in_plot(spec, n, synth.numpy_density(
        lambda x: o.inside(x).astype(np.float64)), seed=seed + 1,
        dtype=torch.float32).numpy().astype(np.float64)
    return o, data, norm


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _time_oracle(o, params, data, norm, threads, target_s):
    t0 = time.perf_counter()
    o.nll_grad(params, data, norm, threads=threads)
    once = time.perf_counter() - t0
    reps = max(1, min(50, int(target_s / max(once, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(reps):
        o.nll_grad(params, data, norm, threads=threads)
    return reps, time.perf_counter() - t0


def cpu_baseline(spec, params, n: int = 200_000, target_s: float = 10.0):
    """The oracle, as it stands, on a bounded sample: repeated NLL+grad
    evaluations of n + n events for about target_s seconds on all host cores,
    then one thread on a tenth of the sample."""
    o, data, norm = oracle_sample(spec, n, seed=101)
    cores = os.cpu_count() or 1
    reps, dt = _time_oracle(o, params, data, norm, cores, target_s)
    n1 = n // 10
    reps1, dt1 = _time_oracle(o, params, data[:n1], norm[:n1], 1, target_s / 2)
    base = {"value": reps * 2 * n / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{n} data + {n} normalisation events of the same model (float32-rounded, "
                      f"drawn with the oracle's density), {reps} NLL+grad evaluation(s), "
                      f"{cores} OpenMP threads",
            "single_thread": {"value": reps1 * 2 * n1 / dt1, "unit": "events/s", "cores": 1,
                              "sample": f"{n1} data + {n1} normalisation events of the same "
                                        f"sample, {reps1} NLL+grad evaluation(s), 1 thread"}}
    return base, accuracy_vs_oracle(spec, params, o, data, norm, cores)


def accuracy_vs_oracle(spec, params, o, data, norm, cores):
    """The error of each compute form of the library against the oracle on the
    oracle's own sample (the events are float32 values, so every form sees the
    same events)."""
    import numpy as np
    import torch

    from paper_1703_03284_gb300 import F32, F64, Likelihood

    vr, gr = o.nll_grad(params, data, norm, threads=cores)
    a2r = {"data": o.amp2(params, data), "uniform": o.amp2(params, norm)}
    out = {"n_data": len(data), "n_norm": len(norm), "oracle_nll": vr,
           "amp2_note": ("per-event |A|^2 error on data events (drawn from the PDF; the 1e-5 "
                         "relative bar) and on uniform normalisation events (near zeros of A "
                         "the relative error grows as 1/|A|; bar: 1e-5 relative + 1e-8 of the "
                         "mean |A|^2, at most 0.1% of events above 1e-5 relative)")}
    for mode, name in ((F64, "fp64"), (F32, "fp32_mixed")):
        dt = torch.float32 if mode == F32 else torch.float64
        d = torch.from_numpy(data).to("cuda", dt)
        nm = torch.from_numpy(norm).to("cuda", dt)
        lik = Likelihood(torch.cuda.current_device(), mode)
        lik.set_spec(spec)
        lik.set_events(d)
        lik.set_norm_sample(nm)
        v, g = lik.nll_grad(params)
        res = {"nll_abs_err": abs(v - vr), "nll_rel_err": abs(v - vr) / abs(vr),
               "grad_rel_err": float(np.linalg.norm(g - gr) / np.linalg.norm(gr))}
        for kind, ev in (("data", d), ("uniform", nm)):
            a2 = lik.amp2(params, ev).cpu().numpy()
            ref = a2r[kind]
            rel = np.abs(a2 / ref - 1.0)
            res[f"amp2_{kind}"] = {
                "rel_err_median": float(np.median(rel)), "rel_err_max": float(rel.max()),
                "frac_above_1e-5": float(np.mean(rel > 1e-5)),
                "max_err_over_bound": float(np.max(np.abs(a2 - ref) /
                                                   (1e-5 * ref + 1e-8 * ref.mean())))}
        out[name] = res
    return out


def run_reference(args, world, rank):
    import synth
    if rank != 0:
        return
    spec = synth.pipipi(40)
    params = synth.perturbed_params(spec, 3)
    n = 100_000
    o, data, norm = oracle_sample(spec, n, seed=101)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        o.nll_grad(params, data, norm, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.nll_grad(params, data, norm, threads=cores)
    dt = time.perf_counter() - t0
    value = args.steps * 2 * n / dt
    sample = (f"each step: {n} data + {n} normalisation events of the workload's model, "
              f"FP64 oracle NLL+grad on {cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.n_events, args.gpus),
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------ batched toys
def toys_leg(args, stream, rank):
    """256 toys of the 30-knot pi pi pi model, sizes Poisson around log-uniform
    means in [1e4, 1e6], a shared 1e7-event normalisation sample; one batched
    NLL+gradient evaluation (CUDA graph) per step, FP32-mixed with the cached
    basis, against a loop of single-toy FP64 evaluations."""
    import numpy as np
    import torch

    import synth
    from paper_1703_03284_gb300 import F32, F64, Likelihood

    spec = synth.pipipi(30)
    truth = synth.true_params(spec)
    sizes = synth.toy_sizes(args.n_toys, seed=7 + rank)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    gen = Likelihood(torch.cuda.current_device(), F32)
    gen.set_spec(spec)
    pool = synth.accept_reject(spec, int(offsets[-1]), lambda x: gen.amp2(truth, x),
                               seed=11 + 1000 * rank, device="cuda", dtype=torch.float32,
                               chunk=1 << 24)
    norm = synth.uniform_in_plot(spec, args.toys_norm, lambda x: gen.inside(x).to(torch.float64),
                                 seed=12 + 1000 * rank, device="cuda", dtype=torch.float32,
                                 chunk=1 << 24)
    params = np.stack([synth.perturbed_params(spec, 500 + t, 0.02) for t in range(args.n_toys)])
    lik = Likelihood(torch.cuda.current_device(), F32)
    lik.set_spec(spec)
    lik.set_norm_sample(norm)
    lik.set_toys(pool, offsets)
    lik.enable_basis_cache(True)
    t_tune = time.perf_counter()
    if args.toys_config:
        nc, dc, bs, bps = (int(x) for x in args.toys_config.split(","))
        lik.set_toys_config(norm_chunk=nc, data_chunk=dc, block=bs, blocks_per_sm=bps)
        best = dict(lik.toys_config(), n_timed=0, given=True)
    else:
        best = lik.toys_autotune(params)
    t_tune = time.perf_counter() - t_tune
    lik.nll_grad_toys(params)
    launches0 = lik.launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.toys_steps):
        lik.nll_grad_toys(params)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1) / args.toys_steps
    launches_it = (lik.launch_count() - launches0) / args.toys_steps
    pairs = int(offsets[-1]) + args.n_toys * args.toys_norm
    # the same evaluation without the gradient (mipwa_nll_toys)
    lik.nll_toys(params)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.toys_steps):
        lik.nll_toys(params)
    e1.record(stream)
    torch.cuda.synchronize()
    t_nll_ms = e0.elapsed_time(e1) / args.toys_steps
    # looping single-toy evaluations (a few toys timed, scaled to all toys by events)
    loop = {}
    for mode, name in ((F64, "fp64"), (F32, "fp32")):
        single = Likelihood(torch.cuda.current_device(), mode)
        single.set_spec(spec)
        single.set_norm_sample(norm)
        ev_done, t_done = 0, 0.0
        for t in range(4):
            single.set_events(pool[offsets[t]:offsets[t + 1]])
            single.nll_grad(params[t])
            torch.cuda.synchronize()
            l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0.record(stream)
            single.nll_grad(params[t])
            l1.record(stream)
            torch.cuda.synchronize()
            t_done += l0.elapsed_time(l1)
            ev_done += int(sizes[t]) + args.toys_norm
        loop[name] = {"toys_per_s": 1e3 * 4 / t_done, "event_pairs_per_s": ev_done / (t_done / 1e3),
                      "note": "4 toys timed one by one, same events"}
    # the same toys' forward normalisation integrals with the spline values
    # from the tensor cores, checked on 16 toys against the library's FP64
    # |A|^2 over the same stored events
    tc = toys_tc_leg(args, lik, spec, params, sizes, stream)
    # the same toys with the Re/Im form and the moment normalisation
    lik.set_swave_form("reim")
    lik.enable_norm_gram(True)
    qr = np.stack([to_reim(spec, p) for p in params])
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    lik.build_norm_gram()
    b1.record(stream)
    lik.nll_grad_toys(qr)
    torch.cuda.synchronize()
    build_ms = b0.elapsed_time(b1)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(args.toys_steps):
        lik.nll_grad_toys(qr)
    r1.record(stream)
    torch.cuda.synchronize()
    tr_ms = r0.elapsed_time(r1) / args.toys_steps
    reim = {"ms_per_iteration": tr_ms, "toys_per_s": 1e3 * args.n_toys / tr_ms,
            "event_pairs_per_s": pairs / (tr_ms / 1e3), "moments_build_ms": build_ms,
            "dtype": "f32 (cached basis, CUDA graph); normalisation from FP64 cell moments"}
    return {"n_toys": args.n_toys, "events_in_toys": int(offsets[-1]),
            "norm_events": args.toys_norm, "ms_per_iteration": t_ms,
            "toys_per_s": 1e3 * args.n_toys / t_ms,
            "event_pairs_per_s": pairs / (t_ms / 1e3),
            "nll_only": {"ms_per_iteration": t_nll_ms, "toys_per_s": 1e3 * args.n_toys / t_nll_ms,
                         "note": "mipwa_nll_toys, same launch configuration, no gradient"},
            "autotuned": dict(best, seconds=t_tune),
            "gpu_launches_per_iteration": launches_it,
            "loop_single_toy": loop,
            "speedup_vs_fp64_loop": (1e3 * args.n_toys / t_ms) / loop["fp64"]["toys_per_s"],
            "dtype": "f32 (cached basis, CUDA graph)",
            "tensor_core_norm_integrals": tc,
            "reim_moments": reim}


def toys_tc_leg(args, lik, spec, params, sizes, stream):
    """mipwa_toys_norm_tc on the batched toys: the kernel's time per
    iteration (forward integrals of all toys), the error of the integrals
    against FP64, and the -2 ln L shift that error would cause in each toy
    (2 N_t dI/I)."""
    import numpy as np
    import torch

    from paper_1703_03284_gb300 import F64, Likelihood

    n_toys = len(params)
    lik.toys_norm_tc(params)  # builds the cached basis tiles
    torch.cuda.synchronize()
    ms_call = []
    for _ in range(max(3, args.toys_steps)):
        I_tc, ms = lik.toys_norm_tc(params)
        ms_call.append(ms)
    stored = lik.stored_sample("norm")
    ref = Likelihood(torch.cuda.current_device(), F64)
    ref.set_spec(spec)
    rel, dnll = [], []
    for t in range(0, n_toys, max(1, n_toys // 16)):
        I64 = float(ref.amp2(params[t], stored).double().mean())
        r = (I_tc[t] - I64) / I64
        rel.append(r)
        dnll.append(2.0 * float(sizes[t]) * r)
    del ref
    kms = statistics.median(ms_call)
    pairs = n_toys * int(stored.shape[0])
    return {"kernel_ms": kms, "event_toy_pairs_per_s": pairs / (kms / 1e3),
            "I_rel_err_max": float(np.max(np.abs(rel))), "I_rel_err_mean": float(np.mean(rel)),
            "nll_shift_max": float(np.max(np.abs(dnll))), "toys_checked": len(rel),
            "note": ("forward integrals only (no gradient): spline values a(s), phi(s) of both "
                     "channels from tcgen05.mma (bf16 operands in three parts, FP32 accumulation "
                     "in tensor memory), the rest of |A|^2 on the CUDA cores"),
            "cached_basis_bytes": -(-int(stored.shape[0]) // 64) * 24576}


def to_reim(spec, p):
    """Magnitude/phase parameters -> the same knot values as (Re, Im)."""
    import numpy as np

    R, N = spec.n_res, spec.n_knots
    a, phi = p[2 * R:2 * R + N], p[2 * R + N:]
    return np.concatenate([p[:2 * R], a * np.cos(phi), a * np.sin(phi)])


def reim_leg(args, lik, spec, params, events, stream, world):
    """The same events and knot values with the S-wave spline in the complex
    plane taken as Re/Im (A linear in all parameters): FP32-mixed with the
    normalisation summed event by event, then with the per-cell moments
    (built once, FP64), FP32 and FP64. events/s counts data + normalisation
    events per evaluation, as the headline does."""
    import torch

    from paper_1703_03284_gb300 import F32, F64

    q = to_reim(spec, params)

    def timed(steps):
        lik.nll_grad(q)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            lik.nll_grad(q)
        b.record(stream)
        torch.cuda.synchronize()
        t = max_over_ranks(a.elapsed_time(b), world) / steps
        return {"ms_per_step": t, "value": world * events / (t / 1e3), "unit": "events/s"}

    lik.set_swave_form("reim")
    out = {"fp32_direct": timed(args.reim_steps)}
    lik.enable_norm_gram(True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("reim_moments_build")
    a.record(stream)
    lik.build_norm_gram()
    b.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    out["moments_build_ms"] = a.elapsed_time(b)
    out["moments_doubles"] = (spec.n_knots - 1) ** 2 * (22 + 14 * spec.n_res + spec.n_res ** 2)
    torch.cuda.nvtx.range_push("reim_moments")
    out["fp32_moments"] = timed(args.reim_steps)
    torch.cuda.nvtx.range_pop()
    lik.set_compute_mode(F64)
    out["fp64_moments"] = timed(max(1, args.fp64_steps))
    lik.set_compute_mode(F32)
    lik.enable_norm_gram(False)
    lik.set_swave_form("magphase")
    out["note"] = ("per-step time of the moment form: the moment rows (O(cells)) plus the "
                   "event kernel over the data events only")
    return out


# ------------------------------------------------------- the paper's own fit
PAPER_FIT_SECONDS = {"Tesla K40c": 76, "GeForce GTX 980": 67, "GeForce GT 650M": 179,
                     "2x Xeon E5-2680 v3, 24 threads": 50, "same, 1 thread": 791}


def paper_fit_leg(rank, n_toys: int = 20):
    """The workload of Sec. 4: D+ -> K- K+ K+ with the phi(1020) P-wave and a
    40-knot K+K- S-wave, toys of 100K events drawn from the model, each fitted
    with the normalisation on evenly spaced grids of 0.01, 0.004 and 0.001
    GeV^2 (Fig. 2: fitted minus input values at each boundary point for the
    three spacings). Reports per spacing the wall time of the full fits (BFGS
    + Newton steps + Hessian errors, FP64, as the paper's Table 1 reports fit
    times) and, over the toys, the mean and spread of (fit - input) and of the
    pulls (fit - input)/sigma at every knot, for the magnitudes a_k and the
    phases phi_k; the overall mean pull with its error, and the chi^2 of the
    per-knot mean pulls against zero."""
    import numpy as np
    import scipy.optimize  # noqa: F401  (imported here, outside the timed fits)
    import torch

    import synth
    from paper_1703_03284_gb300 import F64, Likelihood
    from paper_1703_03284_gb300.fit import fit

    spec = synth.kkk(40)
    truth = synth.true_params(spec)
    R, N = spec.n_res, spec.n_knots
    dev = torch.cuda.current_device()
    lik = Likelihood(dev, F64)
    lik.set_spec(spec)
    toys = [synth.accept_reject(spec, 100_000, lambda x: lik.amp2(truth, x),
                                seed=42 + 1000 * rank + t, device="cuda") for t in range(n_toys)]
    starts = []
    for t in range(n_toys):
        st = synth.perturbed_params(spec, 43 + t, 0.02)
        st[:2 * R] = truth[:2 * R]
        starts.append(st)
    knots = slice(2 * R, 2 * R + 2 * N)
    out = []
    for spacing in (0.01, 0.004, 0.001):
        grid = synth.spacing_grid_in_plot(spec, spacing, lambda x: lik.inside(x).to(torch.float64),
                                          device="cuda")
        lik.set_norm_sample(grid)
        diffs, pulls, secs, calls, conv = [], [], [], [], 0
        for t in range(n_toys):
            lik.set_events(toys[t])
            if t == 0:
                for _ in range(3):
                    lik.nll_grad(starts[t])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fit(lik, starts[t], fixed=tuple(range(2 * R)))
            secs.append(time.perf_counter() - t0)
            calls.append(res.n_calls)
            conv += int(res.converged)
            d = res.params[knots] - truth[knots]
            diffs.append(d)
            pulls.append(d / res.errors[knots])
        diffs, pulls = np.array(diffs), np.array(pulls)
        pm, ps = pulls.mean(0), pulls.std(0, ddof=1)
        chi2 = float(np.sum((pm / (ps / np.sqrt(n_toys))) ** 2))

        def per_knot(x):
            return {"a": [round(float(v), 4) for v in x[:N]],
                    "phi": [round(float(v), 4) for v in x[N:]]}
        out.append({"grid_spacing_gev2": spacing, "norm_points": int(grid.shape[0]),
                    "n_toys": n_toys, "converged": conv,
                    "fit_seconds_mean": float(np.mean(secs)),
                    "fit_seconds_max": float(np.max(secs)),
                    "nll_grad_calls_mean": float(np.mean(calls)),
                    "mean_pull": float(pulls.mean()),
                    "mean_pull_error": float(pulls.std(ddof=1) / np.sqrt(pulls.size)),
                    "pull_rms": float(np.sqrt(np.mean(pulls ** 2))),
                    "chi2_knot_mean_pulls": chi2, "ndf": 2 * N,
                    "diff_mean_by_knot": per_knot(diffs.mean(0)),
                    "pull_mean_by_knot": per_knot(pm), "pull_std_by_knot": per_knot(ps)})
    return {"workload": (f"D+ -> K- K+ K+, phi(1020) P-wave + 40-knot S-wave, {n_toys} toys of "
                         "100K events each, FP64 fits started 0.02 from the truth, c_phi fixed"),
            "fits": out, "paper_fit_seconds": PAPER_FIT_SECONDS}


# ------------------------------------------------------------------- ours
def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch

    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        run(args, world, rank, local, stream)


def run(args, world, rank, local, stream):
    import torch

    import synth
    from paper_1703_03284_gb300 import F32, F64, Likelihood

    spec = synth.pipipi(40)
    truth = synth.true_params(spec)
    params = synth.perturbed_params(spec, 3)
    n = args.n_events

    lik = Likelihood(local, F32)  # follows torch's current stream (`stream`)
    lik.set_spec(spec)
    # toy data from the model's own |A|^2 (accept-reject), uniform normalisation
    data = synth.accept_reject(spec, n, lambda x: lik.amp2(truth, x), seed=1 + 1000 * rank,
                               device="cuda", dtype=torch.float32, chunk=1 << 24)
    norm = synth.uniform_in_plot(spec, n, lambda x: lik.inside(x).to(torch.float64),
                                 seed=2 + 1000 * rank, device="cuda", dtype=torch.float32,
                                 chunk=1 << 24)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    events = 2 * n

    # ---- FP32-mixed, inputs resident in HBM
    for _ in range(args.warmup):
        lik.nll_grad(params)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = lik.launch_count()
    lik.set_timing(True)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    clocks.begin()
    e0.record(stream)
    for _ in range(args.steps):
        lik.nll_grad(params)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks.end()
    barrier(world)
    clk = clocks.stop()
    t_ms = max_over_ranks(e0.elapsed_time(e1), world)
    launches = lik.launch_count() - launches0
    kms, kn = lik.kernel_time()
    lik.set_timing(False)
    value = world * events * args.steps / (t_ms / 1e3)
    k_s = kms / kn / 1e3
    achieved = FLOPS_PER_EVENT_GRAD * events / k_s / 1e12
    # ---- the pipes' own peaks on this GPU (after the timed loop)
    peaks = probe_peaks(local)
    peak32, peak64 = peaks["fp32_tflops"], peaks["fp64_tflops"]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak32,
                "unit": "TFLOP/s", "frac": achieved / peak32,
                "traffic": None if TRAFFIC_PER_EVENT is None else TRAFFIC_PER_EVENT * events,
                "kernel": "eval_kernel<float,float2,grad>",
                "kernel_ms": kms / kn, "flops_per_event": FLOPS_PER_EVENT_GRAD,
                "events_per_launch": events,
                "peak_note": ("of measured: FP32 FMA throughput of this GPU in this run "
                              "(mipwa_probe_peak, the larger of fma.rn.f32 and fma.rn.f32x2)"),
                "peak_nominal": PEAK_FP32_TFLOPS, "frac_of_nominal": achieved / PEAK_FP32_TFLOPS}

    # ---- NLL alone (no gradient), FP32-mixed, same events
    nll_only = None
    if args.nll_steps > 0:
        lik.nll(params)
        torch.cuda.synchronize()
        n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0.record(stream)
        for _ in range(args.nll_steps):
            lik.nll(params)
        n1.record(stream)
        torch.cuda.synchronize()
        tn = max_over_ranks(n0.elapsed_time(n1), world) / args.nll_steps
        nll_only = {"fp32": {"ms_per_step": tn, "value": world * events / (tn / 1e3),
                             "unit": "events/s"}}

    # ---- plain FP64 on the same events
    fp64 = None
    if args.fp64_steps > 0:
        lik.set_compute_mode(F64)
        lik.nll_grad(params)
        lik.set_timing(True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            lik.nll_grad(params)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = max_over_ranks(f0.elapsed_time(f1), world)
        kms64, kn64 = lik.kernel_time()
        lik.set_timing(False)
        # the same FP64 evaluation with d/d(m_r, Gamma_r) of both resonances
        lik.nll_grad_bw(params)
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(args.fp64_steps):
            lik.nll_grad_bw(params)
        f1.record(stream)
        torch.cuda.synchronize()
        tbw = max_over_ranks(f0.elapsed_time(f1), world) / args.fp64_steps
        if nll_only is not None:
            f0.record(stream)
            for _ in range(args.fp64_steps):
                lik.nll(params)
            f1.record(stream)
            torch.cuda.synchronize()
            tn64 = max_over_ranks(f0.elapsed_time(f1), world) / args.fp64_steps
            nll_only["fp64"] = {"ms_per_step": tn64, "value": world * events / (tn64 / 1e3),
                                "unit": "events/s"}
        lik.set_compute_mode(F32)
        ach64 = FLOPS_PER_EVENT_GRAD * events / (kms64 / kn64 / 1e3) / 1e12
        fp64 = {"value": world * events * args.fp64_steps / (t64 / 1e3), "unit": "events/s",
                "ms_per_step": t64 / args.fp64_steps, "steps": args.fp64_steps,
                "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64,
                             "unit": "TFLOP/s", "frac": ach64 / peak64,
                             "traffic": None, "kernel": "eval_kernel<double,float2,grad>",
                             "peak_note": "of measured: fma.rn.f64 throughput (mipwa_probe_peak)",
                             "peak_nominal": PEAK_FP64_TFLOPS,
                             "frac_of_nominal": ach64 / PEAK_FP64_TFLOPS},
                "with_bw_mass_width_derivatives": {
                    "ms_per_step": tbw, "value": world * events / (tbw / 1e3), "unit": "events/s",
                    "note": "NLL + gradient + d/d(m_r, Gamma_r) of both resonances, FP64"}}

    # ---- FP32-mixed with the cached Breit-Wigner basis (8 + 8R bytes per event)
    cached = None
    if args.cached_steps > 0:
        lik.enable_basis_cache(True)
        lik.nll_grad(params)  # builds the cache
        lik.nll_grad(params)
        lik.set_timing(True)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.cached_steps):
            lik.nll_grad(params)
        c1.record(stream)
        torch.cuda.synchronize()
        tc = max_over_ranks(c0.elapsed_time(c1), world)
        kmsc, knc = lik.kernel_time()
        lik.set_timing(False)
        lik.enable_basis_cache(False)
        k_sc = kmsc / knc / 1e3
        bytes_ev = 8 + 8 * spec.n_res
        achc = FLOPS_PER_EVENT_GRAD_CACHED * events / k_sc / 1e12
        hbm = bytes_ev * events / k_sc / 1e9
        cached = {"value": world * events * args.cached_steps / (tc / 1e3), "unit": "events/s",
                  "ms_per_step": tc / args.cached_steps, "steps": args.cached_steps,
                  "bytes_per_event": bytes_ev,
                  "roofline": {"bound": "alu", "achieved": achc, "peak": peak32,
                               "unit": "TFLOP/s", "frac": achc / peak32,
                               "hbm_gbs": hbm, "hbm_frac_of_measured": hbm / HBM_GBS,
                               "traffic": None if TRAFFIC_PER_EVENT_CACHED is None
                               else TRAFFIC_PER_EVENT_CACHED * events,
                               "kernel": "eval_kernel<float,float2,grad,cached>"}}

    # ---- Re/Im S-wave form: direct, and with the per-cell moment normalisation
    reim = reim_leg(args, lik, spec, params, events, stream, world) if args.reim_steps > 0 else None

    # ---- end to end from pinned host buffers through the C ABI: one pipelined
    # call per step (mipwa_nll_grad_streamed: copies in pieces, each piece
    # checked, grouped and evaluated as it lands), and for comparison the
    # three-call path (set_events, set_norm_sample, nll_grad)
    e2e = None
    if args.e2e_steps > 0:
        data_h = data.cpu().pin_memory()
        norm_h = norm.cpu().pin_memory()
        for _ in range(args.warmup):
            lik.nll_grad_streamed(params, data_h, norm_h)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("e2e")
        g0.record(stream)
        step_ms = []
        # per-step CUDA events on the library's stream: a slow step with a
        # normal device span was held up on the host, a slow device span on
        # the GPU or the host link
        sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.e2e_steps)]
        for k in range(args.e2e_steps):
            t_a = time.perf_counter()
            sev[k][0].record(stream)
            lik.nll_grad_streamed(params, data_h, norm_h)
            sev[k][1].record(stream)
            step_ms.append(1e3 * (time.perf_counter() - t_a))
        g1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        te = max_over_ranks(g0.elapsed_time(g1), world)
        dev_ms = [a.elapsed_time(b) for a, b in sev]
        med = statistics.median(step_ms)
        slow = [(round(h, 2), round(dv, 2)) for h, dv in zip(step_ms, dev_ms) if h > 1.5 * med]
        # the three-call path on the same buffers
        n3 = max(3, args.e2e_steps // 5)
        for _ in range(2):
            lik.set_events(data_h)
            lik.set_norm_sample(norm_h)
            lik.nll_grad(params)
        torch.cuda.synchronize()
        g0.record(stream)
        step3 = []
        for _ in range(n3):
            t_a = time.perf_counter()
            lik.set_events(data_h)
            lik.set_norm_sample(norm_h)
            lik.nll_grad(params)
            step3.append(1e3 * (time.perf_counter() - t_a))
        g1.record(stream)
        torch.cuda.synchronize()
        t3 = g0.elapsed_time(g1) / n3
        # the host link on its own: plain copies of the same pinned buffers
        scratch = torch.empty_like(data)
        h2d_gbs = []
        for buf in (data_h, norm_h):
            scratch.copy_(buf, non_blocking=True)
            g0.record(stream)
            for _ in range(3):
                scratch.copy_(buf, non_blocking=True)
            g1.record(stream)
            torch.cuda.synchronize()
            h2d_gbs.append(3 * buf.numel() * 4 / (g0.elapsed_time(g1) / 1e3) / 1e9)
        del scratch
        P = spec.n_params
        h2d = int(data_h.numel() * 4 + norm_h.numel() * 4 + 8 * P)
        floor_ms = 1e3 * (data_h.numel() * 4 / (h2d_gbs[0] * 1e9) +
                          norm_h.numel() * 4 / (h2d_gbs[1] * 1e9))
        e2e = {"value": world * events * args.e2e_steps / (te / 1e3), "unit": "events/s",
               "ms_per_step": te / args.e2e_steps, "call": "mipwa_nll_grad_streamed",
               "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(8 * (1 + P) + 4 + 2 * 8),
               "host_link_gbs": {"data": h2d_gbs[0], "norm": h2d_gbs[1]},
               "copy_floor_ms": floor_ms,
               "median_over_floor": statistics.median(step_ms) / floor_ms,
               # now and then a single step takes 2-5x longer (its host-to-device
               # copies stall); the mean above includes such steps
               "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms),
                           "max": max(step_ms)},
               "device_step_ms": {"median": statistics.median(dev_ms), "max": max(dev_ms)},
               "slow_steps_host_device_ms": slow,
               "three_call_path": {"ms_per_step": t3, "steps": n3,
                                   "step_ms_median": statistics.median(step3),
                                   "calls": "set_events + set_norm_sample + nll_grad"}}

    toys = None
    if args.toys_steps > 0:
        del lik
        torch.cuda.empty_cache()
        toys = toys_leg(args, stream, rank)

    paper = paper_fit_leg(rank, args.paper_toys) if args.paper_fit else None

    cpu, accuracy = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, accuracy = cpu_baseline(spec, params)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": bench_config(n, world),
            "roofline": roofline, "alu_peaks": peaks, "nll_only": nll_only, "fp64_plain": fp64,
            "fp32_cached_basis": cached,
            "batched_toys": toys, "reim_moment_normalisation": reim,
            "paper_workload_fit": paper, "e2e": e2e,
            "cpu_baseline": cpu, "accuracy_vs_oracle": accuracy,
            "gpu_launches": launches, "clocks": clk,
        }), flush=True)


if __name__ == "__main__":
    main()
