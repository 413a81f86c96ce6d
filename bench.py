#!/usr/bin/env python3
"""Live-WDD benchmark on GB300.

One step = one full live acquisition of the workload: every frame of the 128 x 128 scan
(128 x 128 float32 detector, Poisson 1e4 e-/frame, Hermite-Gauss K = 64) is pushed in 64-frame
batches (projection + phase accumulation), then a snapshot runs the deconvolution and the inverse
DFT.  `value` = frames reconstructed per second over all ranks, timed with CUDA events on the
launch stream with the frames already resident in HBM (1.07 GB of frames per step, larger than
L2).  The optimised path replays the step as one captured CUDA graph; the plain FP32 path
(`baseline_fp32_plain`) runs the same steps eagerly with every push accumulated at once.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent acquisition (replicas, weak scaling, no
collective on the data path); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "c2"
METRIC = "live WDD frames/s and p99 frame latency vs plain FP32 path; % tensor peak"
UNIT = "frames/s"
LATENCY_SNAPSHOT_EVERY = 1024
ACCUM_DEPTH = 4096     # frames staged per tensor-core accumulation on the optimised path
COALESCE = 4096        # pushes gathered into projection launches of up to 4096 frames
TIMING_REPLAYS = 3     # replays of the step captured with stage-timing events
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
EXEC_FACTOR = 3        # tensor-core products per algorithmic product on the split path


def exec_factor(info) -> float:
    """Tensor-core products per algorithmic product of a split plan: three (hi*hi, hi*lo,
    lo*hi) over the scan columns the accumulation computes (S_x / 2 + 1 of S_x; the rest of H
    follows from its Hermitian symmetry)."""
    return EXEC_FACTOR * info["spectrum_cols"] / max(1, info["spectrum_cols_total"])


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch of a kernel on a workload from the committed ncu record, or None
    when no capture ran on that workload or the kernel's source has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(f"{kernel}@{workload}")
        if not rec:
            return None
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != rec["sha256"]:
                return None
        return rec
    except (OSError, ValueError, KeyError):
        return None


def dist_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return _env_int("WORLD_SIZE", 1), _env_int("RANK", 0), _env_int("LOCAL_RANK", 0)


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest value over all ranks: with per-rank step times, the slowest rank's."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job rate: every rank processes its own units (replicas, weak scaling), so the job
    completes world x units per step in the slowest rank's step time."""
    return units_per_rank * world / (ms_per_step * 1e-3)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"],
                    bf16_sust=d.get("bf16_tflops_sustained", d["bf16_tflops"]), src="measured")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sust=1700.0, src="fallback")


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def keep_busy(self, fn, until_samples: int, max_s: float):
        """Runs fn (untimed) in bursts until `until_samples` samples have been read."""
        import torch
        if self.proc is None:
            return
        t_end = time.time() + max_s
        while len(self.lines) < until_samples and time.time() < t_end:
            for _ in range(10):
                fn()
            torch.cuda.synchronize()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "nvidia-smi every 200 ms from just before to just after the timed "
                          "region, the GPU kept busy by untimed replays of the same step"}


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------------------------

def oracle_sample(acq, rc, frames, idx, n_sample: int):
    """Times the oracle's live path (coefficients, accumulation over every scan frequency,
    deconvolution, inverse DFT) on the first n_sample frames.  Returns (seconds, cores)."""
    import oracle.wdd_oracle as W
    p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                  epsilon=rc["epsilon"])
    plan = W.build_plan(p)
    t0 = time.perf_counter()
    o = W.live_wdd(frames[:n_sample], idx[:n_sample], plan)
    W.finalize(o, p)
    return time.perf_counter() - t0, os.cpu_count()


_SINGLE_THREAD_ORACLE = r"""
import sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle.wdd_oracle as W
import synth
acq, rc = synth.config(sys.argv[2])
n = int(sys.argv[3])
frames = np.concatenate([f for _, f in synth.frames(acq, 0, n, chunk=n)])
idx = synth.raster_indices(acq)[:n]
p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"], epsilon=rc["epsilon"])
By, Bx, m_idx, comp, m_neg = W._bases(p)
plan = W.OraclePlan(params=p, By=By, Bx=Bx, m_idx=m_idx, comp=comp, m_neg=m_neg,
                    chi=np.zeros((1, 1)), W=np.zeros((1, rc["rank_k"])), mask=np.ones(1, bool),
                    eps_eff=0.0)
t0 = time.perf_counter()
W.accumulate(W.coefficients(frames, plan), idx, p)
print(time.perf_counter() - t0)
"""


def oracle_single_thread(n_sample: int):
    """The oracle's per-frame work (projection, accumulation over every scan frequency) on one
    host core: a subprocess with the BLAS and OpenMP pools pinned to one thread.  Returns
    seconds or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    root = os.path.dirname(os.path.abspath(__file__))
    try:
        r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD_ORACLE, root, WORKLOAD,
                            str(n_sample)], env=env, capture_output=True, text=True, timeout=300)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def run_reference(args):
    import synth
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    acq, rc = synth.config(WORKLOAD)
    n_sample = 1024
    idx = synth.raster_indices(acq)
    frames = np.concatenate([f for _, f in synth.frames(acq, 0, n_sample, chunk=1024)])
    times = []
    cores = os.cpu_count()
    for it in range(args.warmup + args.steps):
        dt, cores = oracle_sample(acq, rc, frames, idx, n_sample)
        if it >= args.warmup:
            times.append(dt)
    sec = float(np.mean(times))
    fps = n_sample / sec
    sample = (f"{n_sample} of {acq.n_frames} frames of the workload per step (coefficients, "
              "accumulation over all scan frequencies, deconvolution, inverse DFT); plan build "
              "excluded")
    out = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "128x128 scan, 128x128 f32 detector, HG K=64, B=64",
                      "name": WORKLOAD},
           "cpu_baseline": {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# serving mode: six concurrent sessions, seeded Poisson arrivals at 20k frames/s
# ---------------------------------------------------------------------------------------------

def run_serving(args) -> int:
    import torch

    import synth
    from paper_2212_01309_gb300 import serving, wdd
    from synth.torch_gen import TorchFrames

    torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
    mix = synth.serving_mix()
    sessions, plain = [], []
    for sid, (acq, rc) in enumerate(mix):
        frames = TorchFrames(acq).all()
        p = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                        epsilon=rc["epsilon"], precision="split", max_batch=512,
                                        accum_depth=2048, coalesce_frames=1024,
                                        overlap_pushes=True)
        sessions.append(serving.Session(sid=sid, params=p, frames=frames, n_frames=acq.n_frames))
        # the plain path for the same session: FP32 SIMT kernels, every push accumulated at once
        q = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                        epsilon=rc["epsilon"], precision="fp32", max_batch=512,
                                        accum_depth=0)
        plain.append(serving.Session(sid=sid, params=q, frames=frames, n_frames=acq.n_frames))
    torch.cuda.synchronize()
    arrivals = synth.serving_arrivals([s.n_frames for s in sessions])
    free, total = torch.cuda.mem_get_info()
    budget = int(min(free * 0.5, 64 << 30))
    deadline = 0.02
    out = {"mode": "serving", "metric": METRIC, "unit": UNIT, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "6 sessions: scan/detector 64^2/64^2, 128^2/64^2, 128^2/128^2, "
                                  "256^2/128^2, 192x256/96^2, 256^2/256^2; uint16 Poisson frames; "
                                  "batches of 16-512 frames; snapshot every 1024 frames per session",
                      "arrival_rate_fps": 20000, "frames": sum(s.n_frames for s in sessions),
                      "schedule_s": arrivals[-1][0], "hbm_budget_bytes": budget,
                      "precision": "split", "cuda_graph_snapshots": True,
                      "deadline_run_snapshot_max_delay_ms": deadline * 1e3}}
    results = {}
    runs = [("open_loop", sessions, True, None, False),
            ("open_loop_deadline", sessions, True, deadline, False),
            ("open_loop_deadline_grouped", sessions, True, deadline, True),
            ("closed_loop", sessions, False, None, False),
            ("closed_loop_grouped", sessions, False, None, True),
            ("closed_loop_fp32_plain", plain, False, None, False)]
    for mode, specs, open_loop, delay, grouped in runs:
        srv = serving.Server(hbm_budget_bytes=budget, snapshot_every=1024, use_graphs=True,
                             snapshot_max_delay_s=delay, grouped=grouped)
        for s in specs:
            srv.add_session(s)
        setup = srv.admit_now()          # plans (Algorithm 1) built when the sessions are set up
        torch.cuda.synchronize()
        st = srv.run(arrivals, open_loop=open_loop, timeout_s=1800)
        st["session_setup_s"] = setup
        out[mode] = st
        results[mode] = srv.results

    def rel(a, b):   # relative L2 of mean-subtracted phases
        a = a.astype(np.float64) - a.mean()
        b = b.astype(np.float64) - b.mean()
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    out["closed_loop"]["phase_rel_l2_vs_fp32_plain"] = [
        rel(results["closed_loop"][sid], results["closed_loop_fp32_plain"][sid])
        for sid in sorted(results["closed_loop"])]
    out["closed_loop"]["phase_std_per_session"] = [
        float(results["closed_loop"][sid].std()) for sid in sorted(results["closed_loop"])]
    for mode in ("closed_loop", "closed_loop_grouped"):
        out[mode]["speedup_vs_fp32_plain"] = (out[mode]["frames_per_s"] /
                                              out["closed_loop_fp32_plain"]["frames_per_s"])
    out["value"] = out["closed_loop"]["frames_per_s"]
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# extras on the default line: the accumulation at the serving ranks, and a slice of the serving mix
# ---------------------------------------------------------------------------------------------

RANKS = ((64, "hg_tensor"), (128, "hg_energy"), (256, "hg_tensor"))


def accumulate_by_rank(acq, d_frames, idx, stream, peaks, n_frames=4096, reps=5) -> dict:
    """The tensor-core accumulation of one flush of n_frames staged frames on this scan at ranks
    K = 64, 128 and 256 (the serving mix's ranks): device time of the flush (split pre-pass and
    accumulation launch, CUDA events around them on the launch stream), algorithmic 4 S K flops
    per frame and the tensor-core products the split path executes (exec_factor), against the
    measured bf16 dense peak.  Median of `reps` flushes."""
    from paper_2212_01309_gb300 import wdd
    S = acq.scan_y * acq.scan_x
    out = {}
    for K, basis in RANKS:
        p = wdd.params_from_acquisition(acq, basis=basis, rank_k=K, epsilon=1e-3,
                                        precision="split", max_batch=1024,
                                        accum_depth=n_frames, coalesce_frames=1024,
                                        overlap_pushes=True)
        ms = []
        with wdd.Plan(p) as g:
            info = dict(g.info(), spectrum_cols_total=acq.scan_x)
            kern = wdd.ACCUM_KERNEL[info["accum_kernel"]]
            xf = exec_factor(info)
            for r in range(reps + 1):
                g.reset(stream=stream)
                for a in range(0, n_frames, 1024):
                    g.push(d_frames[a:a + 1024], idx[a:a + 1024], stream=stream)
                g.set_stage_timing(True)
                g.flush(stream=stream)
                g.set_stage_timing(False)
                st = g.stage_times()
                if r > 0:
                    ms.append(st["accumulate"][0])
            g.check_device()
        flush_ms = float(np.median(ms))
        alg = 4.0 * S * K * n_frames / (flush_ms * 1e-3) / 1e12
        out[f"K{K}"] = {"basis": basis, "kernel": kern, "flush_frames": n_frames,
                        "flush_ms": flush_ms,
                        "achieved_algorithmic": alg, "achieved_executed": xf * alg,
                        "peak": peaks["bf16"], "unit": "TFLOP/s",
                        "frac_algorithmic": alg / peaks["bf16"],
                        "frac_executed": xf * alg / peaks["bf16"]}
    return out


def serving_slice(seconds=2.0, deadline_s=0.02) -> dict:
    """The serving mix (six sessions) over the first `seconds` of its seeded 20k frames/s
    arrival schedule: open loop at the schedule with a snapshot deadline, closed loop (every
    batch available at once) on the split path, and closed loop on the plain FP32 path; each
    session ends (final snapshot) with the slice's last frame."""
    import torch

    import synth
    from paper_2212_01309_gb300 import serving, wdd
    from synth.generator import NOISE_BLOCK
    from synth.torch_gen import TorchFrames
    mix = synth.serving_mix()
    arrivals = synth.serving_arrivals([a.n_frames for a, _ in mix])
    arrivals = [a for a in arrivals if a[0] <= seconds]
    need = [0] * len(mix)
    for _, sid, start, count in arrivals:
        need[sid] = max(need[sid], start + count)
    specs = {"split": [], "fp32": []}
    for sid, (acq, rc) in enumerate(mix):
        if need[sid] == 0:
            continue
        gen = TorchFrames(acq)
        nblk = (need[sid] + NOISE_BLOCK - 1) // NOISE_BLOCK
        frames = torch.cat([gen.block(b) for b in range(nblk)])[:need[sid]].contiguous()
        for prec in ("split", "fp32"):
            kw = dict(precision="split", accum_depth=2048, coalesce_frames=1024,
                      overlap_pushes=True) if prec == "split" else dict(precision="fp32",
                                                                         accum_depth=0)
            p = wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                            epsilon=rc["epsilon"], max_batch=512, **kw)
            specs[prec].append(serving.Session(sid=sid, params=p, frames=frames,
                                               n_frames=need[sid]))
    torch.cuda.synchronize()
    out = {"schedule_s": seconds, "frames": int(sum(need)), "arrival_rate_fps": 20000,
           "snapshot_every": 1024, "deadline_ms": deadline_s * 1e3,
           "sessions": sum(1 for n in need if n)}
    runs = [("open_loop_deadline", "split", True, deadline_s, False),
            ("open_loop_deadline_grouped", "split", True, deadline_s, True),
            ("closed_loop", "split", False, None, False),
            ("closed_loop_grouped", "split", False, None, True),
            ("closed_loop_fp32_plain", "fp32", False, None, False)]
    for mode, prec, open_loop, delay, grouped in runs:
        srv = serving.Server(snapshot_every=1024, use_graphs=True, snapshot_max_delay_s=delay,
                             grouped=grouped)
        for sp in specs[prec]:
            srv.add_session(sp)
        srv.admit_now()
        torch.cuda.synchronize()
        st = srv.run(arrivals, open_loop=open_loop, timeout_s=600)
        out[mode] = {"frames_per_s": st["frames_per_s"], "p50_ms": st["latency_p50_ms"],
                     "p99_ms": st["latency_p99_ms"], "wall_s": st["wall_s"]}
    out["speedup_vs_fp32_plain"] = (out["closed_loop"]["frames_per_s"] /
                                    out["closed_loop_fp32_plain"]["frames_per_s"])
    out["grouped_speedup_vs_fp32_plain"] = (out["closed_loop_grouped"]["frames_per_s"] /
                                            out["closed_loop_fp32_plain"]["frames_per_s"])
    return out


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------

# Workloads the benchmark can time.  `step` = frames per timed step (None: the whole scan);
# `desc` names the workload in the JSON line.
WORKLOADS = {
    "c2": dict(step=None, desc="128x128 scan, 128x128 f32 detector (Poisson 1e4 e-/frame), "
                                "Hermite-Gauss K=64, 64-frame pushes, snapshot per step"),
    "paper": dict(step=None, desc="128x128 scan, 128x128 uint16 detector (Poisson 1e4 e-/frame), "
                                   "Hermite-Gauss K=256 (L=16), 256-frame pushes, snapshot per step"),
    "c3": dict(step=None, desc="256x256 scan, 128x128 uint16 detector (Poisson 1e3 e-/frame), "
                                "Hermite-Gauss energy basis K=128, 256-frame pushes, snapshot per step"),
    "c5": dict(step=16384, desc="512x512 scan, 256x256 uint16 detector (Poisson 1e3 e-/frame), "
                                 "Hermite-Gauss K=256 (L=16), 512-frame pushes: the first 16384 "
                                 "frames (32 scan rows) of the acquisition per step, then a "
                                 "snapshot at full size"),
}
PLAIN_SAMPLE = 4096    # frames the plain FP32 path is timed on for workloads other than c2


def oracle_per_frame(acq, rc, frames, idx, n_sample: int):
    """The oracle's per-frame work (coefficients, accumulation over every scan frequency) on
    n_sample frames; the Wiener filter (Algorithm 1) is not built.  Returns (seconds, cores)."""
    import oracle.wdd_oracle as W
    p = W.Params.from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                  epsilon=rc["epsilon"])
    By, Bx, m_idx, comp, m_neg = W._bases(p)
    plan = W.OraclePlan(params=p, By=By, Bx=Bx, m_idx=m_idx, comp=comp, m_neg=m_neg,
                        chi=np.zeros((1, 1)), W=np.zeros((1, rc["rank_k"])),
                        mask=np.ones(1, bool), eps_eff=0.0)
    t0 = time.perf_counter()
    W.accumulate(W.coefficients(frames[:n_sample], plan), idx[:n_sample], p)
    return time.perf_counter() - t0, os.cpu_count()


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", choices=["auto", "fp32", "split"], default="auto")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-rank accumulation and serving-slice extras of the c2 line")
    ap.add_argument("--serving", action="store_true",
                    help="run the multi-session serving workload instead (separate JSON line)")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)

    import torch
    import torch.distributed as dist

    import synth
    from paper_2212_01309_gb300 import wdd
    from synth.generator import NOISE_BLOCK
    from synth.torch_gen import TorchFrames

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    name = args.workload
    wl = WORKLOADS[name]
    default_line = name == WORKLOAD
    acq, rc = synth.config(name)
    B = rc["batch"]
    idx_all = synth.raster_indices(acq)
    S = wl["step"] or acq.n_frames          # frames per step
    idx = idx_all[:S]
    if default_line:
        frames = synth.all_frames(acq)       # numpy: the CPU baseline times the same frames
        d_frames = torch.from_numpy(frames).cuda()
    else:
        frames = None
        gen = TorchFrames(acq)
        nblk = (S + NOISE_BLOCK - 1) // NOISE_BLOCK
        d_frames = torch.cat([gen.block(b) for b in range(nblk)])[:S].contiguous()
        del gen
    h_frames = d_frames.cpu().pin_memory()
    stream = torch.cuda.Stream()
    obj = torch.empty((acq.scan_y, acq.scan_x), dtype=torch.complex64, device="cuda")
    phase = torch.empty((acq.scan_y, acq.scan_x), dtype=torch.float32, device="cuda")
    h_phase = torch.empty_like(phase, device="cpu").pin_memory()
    frames_bytes = acq.det * acq.det * np.dtype(acq.np_dtype).itemsize

    split_ok = True
    path = args.path
    if path in ("auto", "split"):
        try:
            wdd.Plan(wdd.params_from_acquisition(acq, basis=rc["basis"], rank_k=rc["rank_k"],
                                                 precision="split", max_batch=B,
                                                 accum_depth=ACCUM_DEPTH)).close()
        except wdd.WddError:
            split_ok = False
            if path == "split":
                raise
        path = "split" if split_ok else "fp32"

    def mk(precision, depth, overlap, mode="direct", coalesce=0):
        return wdd.Plan(wdd.params_from_acquisition(
            acq, basis=rc["basis"], rank_k=rc["rank_k"], epsilon=rc["epsilon"],
            precision=precision, max_batch=B, accum_depth=depth, overlap_pushes=overlap,
            accum_mode=mode, coalesce_frames=coalesce))

    # the plain path: FP32 SIMT, every push accumulated at once, eager launches
    plain = mk("fp32", 0, False)
    # the optimised path: tensor-core split accumulation over ACCUM_DEPTH staged frames,
    # consecutive pushes overlapped and gathered into 4096-frame projection launches (the
    # frames are resident for the whole step)
    opt = mk(path, ACCUM_DEPTH, True, coalesce=COALESCE)

    def step(plan, src, n=S):
        plan.reset(stream=stream)
        for a in range(0, n, B):
            plan.push(src[a:min(a + B, n)], idx[a:min(a + B, n)], stream=stream)
        plan.snapshot(obj, phase, stream=stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, k):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / k
        barrier()
        return max_over_ranks(ms, world, device="cuda")

    extras = {}
    with torch.cuda.stream(stream):
        # ---- plain FP32 path (eager, every push accumulated at once); on workloads other than
        # the default it is timed on the first PLAIN_SAMPLE frames (its cost per frame is
        # constant) -----------------------------------------------------------------------------
        n_plain = S if default_line else min(S, PLAIN_SAMPLE)
        for _ in range(min(args.warmup, 3 if default_line else 1)):
            step(plain, d_frames, n_plain)
        ms_plain_n = timed(lambda: step(plain, d_frames, n_plain),
                           args.steps if default_line else 2)
        ph_plain = phase.clone() if default_line else None
        ms_plain = ms_plain_n * S / n_plain   # per step of S frames

        # ---- optimised path: staged accumulation, one CUDA graph per acquisition -------------
        for _ in range(args.warmup):
            step(opt, d_frames)
        torch.cuda.synchronize()
        launches0 = opt.info()["kernel_launches"]
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step(opt, d_frames)
        launches_per_step = opt.info()["kernel_launches"] - launches0
        for _ in range(args.warmup):
            graph.replay()
        # nvidia-smi samples every 200 ms: keep the GPU loaded with untimed replays until its
        # first sample arrives, time exactly `steps` replays, then keep it loaded until one more
        # sample lands, so the recorded clocks bracket the timed region under the same load
        clocks = ClockSampler(local)
        clocks.start()
        clocks.keep_busy(graph.replay, until_samples=1, max_s=5.0)
        ms_opt = timed(graph.replay, args.steps)
        clocks.keep_busy(graph.replay, until_samples=len(clocks.lines) + 1, max_s=1.0)
        clk = clocks.stop()
        ph_opt = phase.clone()

        # ---- stage times of the optimised path: the step captured with an event pair around
        # every launch (event-record graph nodes on the launch stream, so no host gaps) -------
        opt.set_stage_timing(True)
        tgraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(tgraph, stream=stream):
            step(opt, d_frames)
        opt.set_stage_timing(False)
        for _ in range(TIMING_REPLAYS):
            tgraph.replay()
        torch.cuda.synchronize()
        st = opt.stage_times()
        del tgraph

        if default_line:
            # ---- variant: scan-row factorised accumulation (not the paper's form) -----------
            sep = mk(path, ACCUM_DEPTH, True, mode="separable", coalesce=COALESCE)
            for _ in range(args.warmup):
                step(sep, d_frames)
            sgraph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(sgraph, stream=stream):
                step(sep, d_frames)
            for _ in range(args.warmup):
                sgraph.replay()
            ms_sep = timed(sgraph.replay, args.steps)
            ph_sep = phase.clone()
            sep.close()
            del sgraph

            # ---- comparison method: classical WDD on the whole dataset (Eq. 2-3) -------------
            off = wdd.OfflinePlan(wdd.params_from_acquisition(acq, basis=rc["basis"],
                                                              rank_k=rc["rank_k"],
                                                              epsilon=rc["epsilon"]))

            def off_step():
                off.reconstruct(d_frames, obj, phase, stream=stream)
            for _ in range(args.warmup):
                off_step()
            ms_off = timed(off_step, args.steps)
            ph_off = phase.clone()
            off_info = off.info()
            off.close()

            # ---- probe reconstruction (row f4, Sect. 10): the swapped classical deconvolution
            # from an object estimate (the classical result above), then a live plan's Wiener
            # filter rebuilt from the recovered probe (Algorithm 1 again)
            est = obj.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pplan = wdd.OfflinePlan(wdd.params_from_acquisition(acq, basis=rc["basis"],
                                                                rank_k=rc["rank_k"],
                                                                epsilon=rc["epsilon"]), obj=est)
            torch.cuda.synchronize()
            probe_plan_s = time.perf_counter() - t0
            probe = torch.empty_like(obj)

            def probe_step():
                pplan.reconstruct(d_frames, probe, phase, stream=stream)
            for _ in range(args.warmup):
                probe_step()
            ms_probe = timed(probe_step, args.steps)
            probe_bytes = int(pplan.info()["device_bytes"])
            pplan.close()
            upd = mk(path, ACCUM_DEPTH, True, coalesce=COALESCE)
            upd.set_probe(probe)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                upd.set_probe(probe)
            torch.cuda.synchronize()
            set_probe_ms = (time.perf_counter() - t0) / 3 * 1e3
            upd.close()

        # ---- end to end through the public API from pinned host memory ---------------------
        def e2e_step():
            step(opt, h_frames)
            h_phase.copy_(phase, non_blocking=True)
        for _ in range(2):
            e2e_step()
        ms_e2e = timed(e2e_step, max(2, args.steps // 2))

        # the host link these frames cross: a plain pinned-to-device copy of the same bytes
        d_copy = torch.empty_like(d_frames)
        d_copy.copy_(h_frames, non_blocking=True)
        ms_link = timed(lambda: d_copy.copy_(h_frames, non_blocking=True), 2)
        del d_copy

        lat = []
        if default_line:
            # ---- frame-to-snapshot latency (snapshot every 1024 frames) --------------------
            opt.reset(stream=stream)
            torch.cuda.synchronize()
            pending = []
            for a in range(0, S, B):
                t_arr = time.perf_counter()
                opt.push(d_frames[a:a + B], idx[a:a + B], stream=stream)
                pending.append((t_arr, min(B, S - a)))
                if (a + B) % LATENCY_SNAPSHOT_EVERY == 0 or a + B >= S:
                    opt.snapshot(obj, phase, stream=stream)
                    stream.synchronize()
                    t_done = time.perf_counter()
                    for t0, n in pending:
                        lat.extend([t_done - t0] * n)
                    pending = []
    torch.cuda.synchronize()

    def phase_diff(a, b):
        return float(np.linalg.norm((a - a.mean()).cpu().numpy() - (b - b.mean()).cpu().numpy()) /
                     np.linalg.norm((b - b.mean()).cpu().numpy()))

    # ---- roofline of the dominant kernel --------------------------------------------------
    peaks = _peaks()
    proj_kernel = {1: "project_tc_kernel", 3: "project_rows_kernel"}.get(
        opt.info()["proj_engine"], "project_kernel")
    K = rc["rank_k"]
    Sf = acq.scan_y * acq.scan_x               # scan frequencies
    stage_ms = {k: v[0] for k, v in st.items()}
    dom = max(stage_ms, key=stage_ms.get)
    # launches per flush of the optimised path: the split pre-pass, then one accumulation launch
    # (all TMEM segments of the flush)
    per_flush = 2 if path == "split" else 1
    flush_frames = min(ACCUM_DEPTH, S)
    acc_info = dict(opt.info(), spectrum_cols_total=acq.scan_x)
    acc_kernel = wdd.ACCUM_KERNEL[acc_info["accum_kernel"]]
    xf = exec_factor(acc_info) if path == "split" else 1.0
    ms_launch = st[dom][0] / max(1, st[dom][1])
    if dom == "accumulate":
        ms_launch *= per_flush           # one flush of ACCUM_DEPTH frames
        flops = 4.0 * Sf * K * flush_frames
        ach = flops / (ms_launch * 1e-3) / 1e12
        if path == "split":
            tr_a = _traffic(acc_kernel, name)
            roof = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16"], "unit": "TFLOP/s",
                    "frac": ach / peaks["bf16"],
                    "traffic": (tr_a["bytes_per_launch"] * flush_frames / tr_a["frames_per_launch"])
                               if tr_a else None,
                    "achieved_executed": xf * ach,
                    "frac_executed": xf * ach / peaks["bf16"],
                    "note": f"one flush of {flush_frames} frames (split pre-pass + one "
                            f"accumulation launch); algorithmic 4*S*K flops per frame over all S "
                            f"scan frequencies; the split path executes {xf:.3f}x that (hi*hi, "
                            f"hi*lo, lo*hi of phase factors and coefficients on the "
                            f"{acc_info['spectrum_cols']} of {acq.scan_x} scan columns it "
                            f"computes; the rest of H by Hermitian symmetry); peak = "
                            f"{peaks['src']} bf16 dense (fp16 same rate)"}
        else:
            roof = {"bound": "alu", "achieved": ach, "peak": FP32_SIMT_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP32_SIMT_PEAK_TFLOPS, "traffic": None,
                    "note": "FP32 FMA peak = 152 SMs x 128 lanes x 2 x 2.07 GHz"}
    elif dom == "project":
        # the event pairs captured in the graph hold the last replay: ms and launches per step
        frames_per_launch = S / max(1, st["project"][1])
        bpl = frames_per_launch * frames_bytes
        ach = bpl / (ms_launch * 1e-3) / 1e9
        tr = _traffic(proj_kernel, name)
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm"], "unit": "GB/s",
                "frac": ach / peaks["hbm"],
                "traffic": (tr["bytes_per_launch"] * frames_per_launch / tr["frames_per_launch"])
                           if tr else None,
                "algorithmic_bytes": bpl,
                "note": f"algorithmic bytes = {frames_per_launch:.0f} frames per launch ({B}-frame "
                        f"pushes gathered) x {frames_bytes} B; duration from events around each "
                        f"launch (serialised; launches overlap in the timed step); peak = "
                        f"{peaks['src']} copy bandwidth"}
    else:
        bpl = 16.0 * Sf * K
        ach = bpl / (ms_launch * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm"], "unit": "GB/s",
                "frac": ach / peaks["hbm"], "traffic": None}
    roof["kernel"] = proj_kernel if dom == "project" else (acc_kernel if dom == "accumulate" else dom)
    roof["launch_ms"] = ms_launch
    # the accumulation, whatever the dominant kernel
    acc_ms = st["accumulate"][0] / max(1, st["accumulate"][1]) * per_flush   # per flush
    acc_alg = 4.0 * Sf * K * flush_frames / (acc_ms * 1e-3) / 1e12
    acc_peak = peaks["bf16"] if path == "split" else FP32_SIMT_PEAK_TFLOPS
    acc_x = xf
    tr_acc = _traffic(acc_kernel, name) if path == "split" else None
    roof_acc = {"bound": "tensor" if path == "split" else "alu",
                "kernel": f"split_coeff + {acc_kernel} (one flush of {flush_frames} frames)"
                if path == "split" else acc_kernel, "flush_ms": acc_ms,
                "traffic": (tr_acc["bytes_per_launch"] * flush_frames / tr_acc["frames_per_launch"])
                           if tr_acc else None,
                "achieved_algorithmic": acc_alg, "achieved_executed": acc_alg * acc_x,
                "peak": acc_peak, "unit": "TFLOP/s",
                "frac_algorithmic": acc_alg / acc_peak, "frac_executed": acc_alg * acc_x / acc_peak,
                "note": f"algorithmic 4 S K flops per frame over all S scan frequencies; the "
                        f"split path executes {xf:.3f}x that (hi*hi, hi*lo and lo*hi products, "
                        f"Re and Im, on the {acc_info['spectrum_cols']} of {acq.scan_x} scan "
                        f"columns it computes); peak = measured bf16 dense (FP16 same rate)"}
    # the projection, whatever the dominant kernel: bytes of the frames one launch reads
    pj_launches = max(1, st["project"][1])
    pj_fpl = S / pj_launches
    pj_ms = st["project"][0] / pj_launches
    pj_tr = _traffic(proj_kernel, name) if path == "split" else None
    roof_proj = {"bound": "hbm", "kernel": proj_kernel, "launch_ms": pj_ms,
                 "frames_per_launch": pj_fpl,
                 "achieved": pj_fpl * frames_bytes / (pj_ms * 1e-3) / 1e9, "peak": peaks["hbm"],
                 "unit": "GB/s",
                 "frac": pj_fpl * frames_bytes / (pj_ms * 1e-3) / 1e9 / peaks["hbm"],
                 "traffic": (pj_tr["bytes_per_launch"] * pj_fpl / pj_tr["frames_per_launch"])
                            if pj_tr else None,
                 "note": "algorithmic bytes = the frames one launch reads; duration from CUDA "
                         "events around each launch"}

    # ---- extras of the default line: the accumulation at the serving ranks, a serving slice --
    if default_line and not args.no_extras and rank == 0 and world == 1 and path == "split":
        with torch.cuda.stream(stream):
            extras["accumulate_by_rank"] = accumulate_by_rank(acq, d_frames, idx, stream, peaks)
            # the same flushes on a 256x256 scan (the same detector and frames): four times the
            # scan frequencies, so the accumulation CTAs fill several waves of the SMs
            acq256 = dataclasses.replace(acq, scan_y=256, scan_x=256, obj_y=512, obj_x=512)
            extras["accumulate_by_rank_scan256"] = accumulate_by_rank(
                acq256, d_frames, synth.raster_indices(acq256), stream, peaks)
        extras["serving"] = serving_slice()

    # ---- CPU baseline (rank 0, N = 1) -------------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if default_line:
            n_sample = 1024
            dt, cores = oracle_sample(acq, rc, frames, idx, n_sample)
            cpu = {"value": n_sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{n_sample} frames of the workload (coefficients, accumulation over "
                             f"all {Sf} scan frequencies, deconvolution, inverse DFT); plan build "
                             f"excluded"}
            n1 = 256
            dt1 = oracle_single_thread(n1)
            if dt1:
                cpu["single_thread"] = {
                    "value": n1 / dt1, "unit": UNIT, "cores": 1,
                    "sample": f"{n1} frames: coefficients and accumulation over all {Sf} scan "
                              "frequencies (the per-frame work), BLAS pinned to one thread"}
        else:
            n_sample = 128 if Sf * K > 1e7 else 512
            fr = np.concatenate([f for _, f in synth.frames(acq, 0, n_sample, chunk=n_sample)])
            dt, cores = oracle_per_frame(acq, rc, fr, idx_all, n_sample)
            cpu = {"value": n_sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{n_sample} frames of the workload: coefficients and accumulation "
                             f"over all {Sf} scan frequencies (the per-frame work; the Wiener "
                             f"filter and the snapshot excluded)"}

    if rank == 0:
        config = {"workload": wl["desc"], "name": name, "path": path,
                  "accum_depth": ACCUM_DEPTH, "overlap_pushes": True, "coalesce_frames": COALESCE,
                  "cuda_graph": True, "frames_per_step": S,
                  "l2": f"inputs larger than L2 ({S * frames_bytes / 1e9:.2f} GB of frames per step)"}
        out = {
            "metric": METRIC, "value": job_throughput(S, world, ms_opt), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_opt, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if path == "fp32" else "f16-split/f32",
            "data": "synthetic",
            "config": config,
            "baseline_fp32_plain": {"value": job_throughput(S, world, ms_plain), "unit": UNIT,
                                    "ms_per_step": ms_plain, "speedup": ms_plain / ms_opt,
                                    "timed_frames": n_plain},
        }
        if default_line:
            out["baseline_fp32_plain"]["phase_rel_l2_vs_plain"] = phase_diff(ph_opt, ph_plain)
            off_bytes = float(S) * frames_bytes + 40.0 * S * acq.det * acq.det
            out["variant_separable"] = {
                "value": job_throughput(S, world, ms_sep), "unit": UNIT, "ms_per_step": ms_sep,
                "phase_rel_l2_vs_plain": phase_diff(ph_sep, ph_plain),
                "note": "same step with the scan DFT factorised by rows (accum_mode separable, "
                        "FP32 SIMT): not the paper's form, the same H up to rounding"}
            out["variant_classical"] = {
                "value": job_throughput(S, world, ms_off), "unit": UNIT, "ms_per_step": ms_off,
                "device_bytes": off_info["device_bytes"],
                "live_plan_device_bytes": int(opt.info()["device_bytes"]),
                "roofline": {"bound": "hbm", "achieved": off_bytes / (ms_off * 1e-3) / 1e9,
                             "peak": peaks["hbm"], "unit": "GB/s",
                             "frac": off_bytes / (ms_off * 1e-3) / 1e9 / peaks["hbm"],
                             "algorithmic_bytes": off_bytes},
                "phase_rel_l2_vs_live": phase_diff(ph_off, ph_opt),
                "note": "classical WDD (Eq. 2-3) on the same resident frames: FFT over both "
                        "scan axes, inverse detector FFT fused with the Wiener product and the "
                        "sum over r, inverse DFT; algorithmic bytes = frames + 40 B per "
                        "(frequency, pixel): write and re-read the scan spectrum per scan axis "
                        "and read it with the Wiener kernel once; a different estimator than "
                        "the Hermite-Gauss live path, so the phase difference is not a parity "
                        "figure"}
            out["variant_probe"] = {
                "swap_plan_s": probe_plan_s, "swap_ms_per_reconstruction": ms_probe,
                "swap_device_bytes": probe_bytes, "set_probe_ms": set_probe_ms,
                "note": "row f4: the swapped (classical-form) deconvolution with the Wiener "
                        "kernel built from an object estimate (plan build, host clock) and run "
                        "on the step's resident frames (CUDA events); then a live plan's chi and "
                        "Wiener weights rebuilt from the recovered probe (host clock, device "
                        "synchronised)"}
            lat_ms = np.array(lat) * 1e3
            out["latency_ms"] = {"p50": float(np.percentile(lat_ms, 50)),
                                 "p99": float(np.percentile(lat_ms, 99)),
                                 "snapshot_every": LATENCY_SNAPSHOT_EVERY,
                                 "note": "single session, host-synchronised snapshot every "
                                         "1024 frames; the serving mix's open-loop "
                                         "frame-to-snapshot latency is under 'serving'"}
        out.update({
            "stage_ms_per_step": stage_ms,
            "roofline": roof,
            "roofline_accumulate": roof_acc,
            "roofline_project": roof_proj,
            "cpu_baseline": cpu,
            "e2e": {"value": job_throughput(S, world, ms_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": int(S * frames_bytes + 4 * S),
                    "d2h_bytes_per_step": int(4 * acq.scan_y * acq.scan_x),
                    "roofline": {"bound": "host link",
                                 "achieved": S * frames_bytes / (ms_e2e * 1e-3) / 1e9,
                                 "peak": S * frames_bytes / (ms_link * 1e-3) / 1e9,
                                 "unit": "GB/s",
                                 "frac": ms_link / ms_e2e,
                                 "note": "peak = a plain copy of the step's frames from pinned "
                                         "host memory to the device, measured in this run"},
                    "note": "frames read by the kernels from pinned host memory; phase copied back"},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clk,
        })
        out.update(extras)
        print(json.dumps(out), flush=True)
    plain.close()
    opt.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
