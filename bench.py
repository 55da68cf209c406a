"""Throughput of the DiffCloud loss + vertex gradient on GB300.

One step (the default workload, batched_uneven) = the loss and every vertex gradient of 64
cloth trajectories of uneven sizes (grids 15x15 to 80x80, 20 to 100 frames, 2 000 to 30 000
target points per frame): area CDFs, sampling, one persistent nearest-neighbour launch over
all frames, neighbour recovery, losses and the adjoint scatter, planned once at the
autotuned shape and replayed from a CUDA graph. The metric is point pairs per second (one
pair = one (sim point, target point) distance of Eq. 1). `--workload trajectory_50x50`
times one dc_loss_traj call over the 40-frame 50x50 trajectory instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]

N > 1 runs under torchrun, one independent copy of the workload per GPU (weak scaling, no
collective on the data path). `--impl reference` times the FP64 CPU oracle on bounded
samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

FLOP_PER_PAIR = 8        # 3 sub + 3 mul/fma products + 2 adds per distance, shared by both directions
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM
# mma.sync m16n8k16 f16 -> f32 throughput of the GB300, measured with independent MMA chains
# on every SM (TFLOP/s): the ceiling of the legacy warp-level tensor path
MMA_SYNC_TFLOPS = 600.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the nearest-neighbour kernel,
# keyed by (workload, kernel, mode), from one-pass ncu captures of one launch:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k 'regex:k_tcpass$' -c 1 python bench.py --steps 2 --warmup 3 --kernels-only --shape tensor:0
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k 'regex:k_tcpass$' -s 3 -c 1 python bench.py --workload trajectory_50x50 --steps 3 \
#       --warmup 3 --no-cpu-baseline [--mode eq2]  (and --workload trajectory_100x100;
#       -k regex:k_chamfer for --workload single_frame)
CHAMFER_TRAFFIC_BYTES = {("batched_uneven", "k_tcpass", "eq1"): 7.72e9 + 5.41e9,
                         ("trajectory_50x50", "k_tcpass", "eq1"): 53.58e6 + 8.11e6,
                         ("trajectory_50x50", "k_tcpass", "eq2"): 26.11e6 + 0.04e6,
                         ("trajectory_100x100", "k_tcpass", "eq1"): 431.75e6 + 281.22e6,
                         # the direct engine (--shape direct:2), -k regex:k_chamfer; the
                         # single frame runs on it by default
                         ("single_frame", "k_chamfer<true>", "eq1"): 182.53e3,
                         ("trajectory_50x50", "k_chamfer<true>", "eq1"): 22.79e6,
                         ("trajectory_50x50", "k_chamfer<false>", "eq2"): 19.57e6}


def measured_peaks():
    """The generated peak measurements of this machine's GPUs, if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="batched_uneven",
                   choices=["trajectory_50x50", "trajectory_100x100", "single_frame",
                            "batched_uneven", "serving"])
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="batched_uneven: skip the 40-frame trajectory line kept beside it")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--mode", default="eq1", choices=["eq1", "eq2"],
                   help="eq1: Eq. 1 bidirectional mean (default); eq2: Eq. 2 unidirectional sum")
    p.add_argument("--item-pairs", type=float, default=16e9,
                   help="serving: time slice of a long request, in point pairs")
    p.add_argument("--batch-pairs", type=float, default=16e9,
                   help="serving: batch size while the queue is short, in point pairs")
    p.add_argument("--batch-trajectories", type=int, default=None,
                   help="batched_uneven: only its first K trajectories (a small case for ncu)")
    p.add_argument("--frames", type=int, default=None,
                   help="use only the first FRAMES frames of the trajectory (profiling runs)")
    p.add_argument("--shape", default=None,
                   help="ENGINE:WARPS (tensor:0, tcgen05:0, direct:2): the nearest-neighbour "
                        "engine; batched_uneven plans with it instead of timing every shape")
    p.add_argument("--kernels-only", action="store_true",
                   help="batched_uneven: only the planned launch sequence (no plain per-frame "
                        "comparison, end-to-end leg, side line or CPU baseline; profiling runs)")
    return p.parse_args()


def make_workload(name, frames=None, rank=0):
    """The named workload; under torchrun every rank gets its own copy (its own seed)."""
    from paper_2204_03139_gb300.ranks import rank_seed

    sb = workloads.SEED_BASE
    if name == "trajectory_50x50":
        return workloads.trajectory_50x50(seed=rank_seed(sb + 2, rank), T=frames or 40)
    if name == "trajectory_100x100":
        return workloads.trajectory_100x100(seed=rank_seed(sb + 4, rank), T=frames or 100)
    if name == "single_frame":
        return workloads.single_frame(seed=rank_seed(sb + 1, rank))
    if name == "batched_uneven":
        return workloads.batched_uneven(seed=rank_seed(sb + 3, rank))
    raise SystemExit(f"unknown workload {name}")


def arm_config(tr, args, world):
    """The workload's config, the same for the GB300 arm and the reference arm."""
    return config_of(tr, {"parallelism": f"{world} independent trajectories"
                          if world > 1 else "1 GPU",
                          "mode": "Eq. 2 unidirectional sum, fwd + vertex grad"
                          if args.mode == "eq2" else
                          "Eq. 1 bidirectional mean, fwd + vertex grad"})


def config_of(tr, extra=None):
    c = {"workload": tr.name, "frames": tr.T, "grid": f"{int(round(tr.V ** 0.5))}x"
         f"{int(round(tr.V ** 0.5))}", "V": tr.V, "F": tr.F, "N": tr.n(0), "M": tr.m(0),
         "pairs_per_step": tr.pairs(), "mode": "Eq. 1 bidirectional mean, fwd + vertex grad",
         "seed": tr.meta.get("seed"),
         "l2": "flushed between timed steps (256 MiB write outside the step events)"}
    c.update(extra or {})
    return c


# ---------------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), float(f[2]), f[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in busy for i, s in enumerate(r[3]) if s == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(busy), "power_w_max": max(r[2] for r in rows)}


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------------------------
def oracle_sample_step(tr, k, n_s, mode=0):
    """One bounded sample: frame k % T with its first n_s draws and first n_s targets."""
    import oracle

    t = k % tr.T
    oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t)[:n_s], tr.frame_targets(t)[:n_s],
                 mode=mode, details=False)
    return n_s * n_s


def calibrate_oracle(tr, seconds, mode=0):
    """Largest sample size (up to a full frame) whose oracle step takes about `seconds`."""
    n_full = min(tr.n(0), tr.m(0))
    n_s = 1000
    while True:
        t0 = time.perf_counter()
        oracle_sample_step(tr, 0, n_s, mode)
        el = time.perf_counter() - t0
        if el >= seconds or n_s >= n_full:
            return n_s, el
        n_s = min(n_full, int(n_s * max(1.3, min(4.0, (seconds / max(el, 1e-4)) ** 0.5))))


def cpu_model() -> str:
    """The host CPU's model name (Arm hosts may only give the implementer and part numbers)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model", "Hardware"):
        for line in info:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    parts = {ln.split(":", 1)[0].strip(): ln.split(":", 1)[1].strip() for ln in info if ":" in ln}
    if "CPU implementer" in parts:
        # Arm's part numbers for its Neoverse cores
        names = {"0xd0c": "Neoverse N1", "0xd40": "Neoverse V1", "0xd49": "Neoverse N2",
                 "0xd4f": "Neoverse V2", "0xd84": "Neoverse V3", "0xd8e": "Neoverse N3"}
        part = parts.get("CPU part", "?")
        name = names.get(part) if parts["CPU implementer"] == "0x41" else None
        return name or f"implementer {parts['CPU implementer']} part {part}"
    return "unknown"


def cpu_baseline(tr, seconds, mode=0):
    import oracle

    n_s, _ = calibrate_oracle(tr, min(seconds, 5.0), mode)
    t0 = time.perf_counter()
    pairs, k = 0, 0
    while time.perf_counter() - t0 < seconds or k == 0:
        pairs += oracle_sample_step(tr, k, n_s, mode)
        k += 1
    el = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same on one core, on a shorter sample (about a tenth of the time)
    oracle.set_num_threads(1)
    try:
        n1, _ = calibrate_oracle(tr, max(0.5, seconds / 20), mode)
        t1, p1, k1 = time.perf_counter(), 0, 0
        while time.perf_counter() - t1 < seconds / 10 or k1 == 0:
            p1 += oracle_sample_step(tr, k1, n1, mode)
            k1 += 1
        one = {"value": p1 / (time.perf_counter() - t1), "sample": f"{k1} frame evaluations, "
               f"first {n1} draws and targets each"}
    finally:
        oracle.set_num_threads(cores)
    return {"value": pairs / el, "unit": "pairs/s", "cores": cores,
            "cpu_model": cpu_model(), "one_core": one,
            "kind": "oracle",
            "sample": f"{k} frame evaluations of {tr.name} (frame k mod {tr.T}), each with its "
                      f"first {n_s} draws and first {n_s} targets"
                      f"{' (the whole frame)' if n_s >= min(tr.n(0), tr.m(0)) else ''}: loss + "
                      f"vertex gradient, FP64 with float32 neighbour decisions, {el:.1f} s"}


def batched_config(trajs, args, world):
    """The batched workload's config, the same for the GB300 arm and the reference arm."""
    return {"workload": f"batched_uneven_{len(trajs)}traj", "trajectories": len(trajs),
            "frames": sum(t.T for t in trajs), "pairs_per_step": sum(t.pairs() for t in trajs),
            "mode": "Eq. 2 unidirectional sum, fwd + vertex grad"
            if args.mode == "eq2" else "Eq. 1 bidirectional mean, fwd + vertex grad",
            "parallelism": f"{world} independent batches" if world > 1 else "1 GPU",
            "seed": workloads.SEED_BASE + 3}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle

    oracle.build()
    mode = oracle.UNIDIR_SUM if args.mode == "eq2" else oracle.BIDIR_MEAN
    if args.workload == "batched_uneven":
        trajs = make_workload("batched_uneven")
        # the frames of the fixed 8-trajectory subset, in order, one per step
        frames = [(tr, t) for tr in batch_cpu_subset(trajs) for t in range(tr.T)]
        tr0 = frames[0][0]
        config = batched_config(trajs, args, world)
    else:
        tr0 = make_workload(args.workload, args.frames)
        frames = [(tr0, t) for t in range(tr0.T)]
        config = arm_config(tr0, args, world)
    # size each step so that warmup + steps take about two minutes
    per_step = max(0.02, min(1.0, 120.0 / max(1, args.steps + args.warmup)))
    n_s, _ = calibrate_oracle(tr0, per_step, mode)

    def step(k):
        tr, t = frames[k % len(frames)]
        n = min(n_s, tr.n(t), tr.m(t))
        oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t)[:n], tr.frame_targets(t)[:n],
                     mode=mode, details=False)
        return n * n

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    pairs = 0
    for k in range(args.steps):
        pairs += step(args.warmup + k)
    el = time.perf_counter() - t0
    value = pairs / el
    cores = oracle.num_threads()
    sample = (f"each step: one frame of the workload (in order"
              f"{', over the trajectories 0, 8, ..., 56 of the batch' if args.workload == 'batched_uneven' else ''}"
              f") cut to its first {n_s} draws and {n_s} targets (fewer if the frame has fewer)")
    line = {"metric": "chamfer_fwd_bwd_point_pairs_per_s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "note": "the FP64 oracle on the host cores; each step is a bounded sample of the "
                    "workload (see cpu_baseline.sample), timed on the host clock",
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------------------------
def run_gpu(args, rank, world, dist):
    import torch

    from paper_2204_03139_gb300 import _lib

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tr = make_workload(args.workload, args.frames, rank)
    pairs = tr.pairs()
    T, V, F, N, M = tr.T, tr.V, tr.F, tr.n(0), tr.m(0)

    # inputs resident in HBM
    v = torch.from_numpy(tr.verts).to(dev)
    f = torch.from_numpy(tr.faces).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).to(dev)
    y = torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).to(dev)
    out = {"loss_total": torch.empty(1, device=dev), "loss_frames": torch.empty(T, device=dev),
           "grad_verts": torch.empty((T, V, 3), device=dev),
           "nn_ab": torch.empty((T, N), dtype=torch.int32, device=dev),
           "nn_ba": torch.empty((T, M), dtype=torch.int32, device=dev),
           "ws": torch.empty(_lib.dc_workspace_size(T, V, F, N, M), dtype=torch.uint8,
                             device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    mode = _lib.UNIDIR_SUM if args.mode == "eq2" else _lib.BIDIR_MEAN

    def step():
        _lib.dc_loss_traj(v, f, d, y, mode=mode, out=out)

    clocks = ClockSampler(local)
    r = _lib.dc_loss_traj(v, f, d, y, mode=mode, out=out, check=True)  # validates the inputs
    t_w = time.perf_counter()
    k = 0
    while k < args.warmup or time.perf_counter() - t_w < 1.0:
        step()
        k += 1
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = _lib.launch_count()
    _lib.prof_start(args.steps)
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    chamfer_ms, chamfer_n = _lib.prof_stop()
    launches = _lib.launch_count() - launches0
    clk = clocks.stop()
    per = [a.elapsed_time(b) for a, b in ev]
    from paper_2204_03139_gb300.ranks import max_over_ranks

    total_ms = max_over_ranks(sum(per), dist)  # the job takes as long as its slowest rank
    ms_per_step = total_ms / args.steps
    value = world * pairs / (ms_per_step / 1e3)

    # end to end: host (pinned) inputs -> device, the call, gradient + loss back to the host
    hv = torch.from_numpy(tr.verts).pin_memory()
    hf = torch.from_numpy(tr.faces).pin_memory()
    hd = torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).pin_memory()
    hy = torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).pin_memory()
    hg = torch.empty((T, V, 3), dtype=torch.float32).pin_memory()
    hl = torch.empty(1, dtype=torch.float32).pin_memory()
    dv, df, dd, dy = (torch.empty_like(hv, device=dev), torch.empty_like(hf, device=dev),
                      torch.empty_like(hd, device=dev), torch.empty_like(hy, device=dev))
    h2d = sum(t.numel() * t.element_size() for t in (hv, hf, hd, hy))
    d2h = hg.numel() * 4 + 4

    def e2e_step():
        dv.copy_(hv, non_blocking=True)
        df.copy_(hf, non_blocking=True)
        dd.copy_(hd, non_blocking=True)
        dy.copy_(hy, non_blocking=True)
        rr = _lib.dc_loss_traj(dv, df, dd, dy, mode=mode, out=out)
        hg.copy_(rr["grad_verts"], non_blocking=True)
        hl.copy_(rr["loss_total"], non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()

    for _ in range(3):
        e2e_step()
    # wall time of each end-to-end step (the L2 flush before it is excluded)
    e2e_times = []
    for _ in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e2e_step()
        e2e_times.append(time.perf_counter() - t1)
    e2e_sync_value = world * pairs / statistics.mean(e2e_times)

    # end to end, pipelined (the public LossPipeline): every step copies its inputs from pinned
    # host memory and its gradient and loss back; while one step computes, the next one's
    # inputs and the previous one's results are in flight. The caller reads each step's loss
    # from host memory before that step's host buffers are reused.
    from paper_2204_03139_gb300.pipeline import LossPipeline

    pipe = LossPipeline(T, V, tr.F, tr.n(0), tr.m(0), device=dev, mode=mode, depth=2)
    houts = [(LossPipeline.pinned((T, V, 3)), LossPipeline.pinned(1)) for _ in range(2)]
    hin = (hv, hf, hd, hy)

    def run_pipe(k_steps):
        pend = []
        for k in range(k_steps):
            if len(pend) == 2:  # the host buffers of step k - 2 are reused now: read its loss
                ev, o = pend.pop(0)
                ev.synchronize()
                float(o[1][0])
            o = houts[k % 2]
            pend.append((pipe.submit(*hin, grad_out=o[0], loss_out=o[1]), o))
        for ev, o in pend:
            ev.synchronize()
            float(o[1][0])

    run_pipe(3)
    n_pipe = max(args.e2e_steps, 4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    run_pipe(n_pipe)
    pipe_s = time.perf_counter() - t1
    if pipe.status() != _lib.DC_OK:
        raise RuntimeError("device-side error in the pipelined end-to-end run")
    e2e_value = world * pairs * n_pipe / pipe_s
    piped = {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
             "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * pipe_s / n_pipe, "steps": n_pipe,
             "api": "pipeline.LossPipeline: pinned host inputs -> device, dc_loss_traj with "
                    "the vertex gradient, gradient + loss -> pinned host, consecutive steps "
                    "overlapped on three streams (L2 not flushed: every step's inputs arrive "
                    "from host memory)"}
    synced = {"value": e2e_sync_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
              "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * statistics.mean(e2e_times),
              "steps": args.e2e_steps,
              "api": "one synchronous step: copies in, dc_loss_traj, copies out, stream "
                     "synchronise (L2 flushed before each step)"}
    # both are public paths; a user picks the faster one for the problem size (the pipeline
    # pays a few tens of microseconds of stream and event overhead per step)
    e2e_best, e2e_other = (piped, synced) if e2e_value >= e2e_sync_value else (synced, piped)

    if rank != 0:
        return
    # measured FP32 FMA throughput (scalar and packed f32x2), the cross-check of the peak
    fma_clk = ClockSampler(local)
    fma = {"scalar": max(_lib.fp32_fma_rate(False, device=dev) for _ in range(2)),
           "packed": max(_lib.fp32_fma_rate(True, device=dev) for _ in range(2))}
    fma_mhz = fma_clk.stop().get("sm_mhz")
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = clk.get("sm_mhz") or 0.0
    sm_max = clk.get("sm_max_mhz") or 0.0
    peak_tflops = 2 * FP32_LANES_PER_SM * sms * sm_mhz * 1e6 / 1e12 if sm_mhz else None
    chamfer_avg_s = chamfer_ms / max(1, chamfer_n) / 1e3
    achieved = FLOP_PER_PAIR * pairs / chamfer_avg_s / 1e12 if chamfer_n else None
    # the engine the library ran (the workspace header's engine word, offset 52)
    engine = int(out["ws"][52:56].cpu().view(torch.int32)[0])
    if engine in (_lib.ENGINE_TENSOR, _lib.ENGINE_TCGEN05):
        kernel = "k_tcpass5" if engine == _lib.ENGINE_TCGEN05 else "k_tcpass"
    else:
        kernel = "k_chamfer<true>" if mode == _lib.BIDIR_MEAN else "k_chamfer<false>"
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": (achieved / peak_tflops) if (achieved and peak_tflops) else None,
            "traffic": (CHAMFER_TRAFFIC_BYTES.get((args.workload, kernel, args.mode))
                        if args.frames is None else None),
            "kernel": kernel,
            "peak_basis": f"FP32 FMA peak 2 x {FP32_LANES_PER_SM} lanes x {sms} SMs x median "
                          f"SM clock under load ({sm_mhz:.0f} MHz); at the {sm_max:.0f} MHz "
                          f"maximum it is "
                          f"{2 * FP32_LANES_PER_SM * sms * sm_max * 1e6 / 1e12:.1f} TFLOP/s",
            "kernel_ms": chamfer_avg_s * 1e3,
            "pairs_per_s_kernel": pairs / chamfer_avg_s if chamfer_n else None}
    best_fma = max(fma.values()) / 1e12
    roof["peak_measured"] = {
        "scalar_fma_tflops": fma["scalar"] / 1e12, "packed_fma_tflops": fma["packed"] / 1e12,
        "sm_mhz": fma_mhz, "tflops": best_fma,
        "frac_of_measured": (achieved / best_fma) if achieved else None,
        "how": "dc_fp32_fma_rate: independent FMA chains on every SM at full occupancy; the "
               "larger of the scalar and packed rates"}
    srt = sorted(per)
    line = {"metric": "chamfer_fwd_bwd_point_pairs_per_s", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": arm_config(tr, args, world),
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1,
                                                                    int(0.99 * len(srt)))]},
            "traj_loss_grad_per_s": world * 1e3 / ms_per_step,
            "roofline": roof,
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": e2e_best,
            "e2e_other": e2e_other,
            "loss_total": float(r["loss_total"][0])}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(tr, args.cpu_seconds,
                                            1 if args.mode == "eq2" else 0)
    print(json.dumps(line), flush=True)


def batch_cpu_subset(trajs):
    """The fixed subset of the batch that the CPU baseline times: every eighth trajectory
    (8 of 64), whole, in order."""
    return trajs[::8]


def batch_cpu_baseline(trajs, seconds_cap=60.0):
    """The FP64 oracle over whole frames of the fixed 8-trajectory subset (stops early, at a
    frame boundary, if it passes seconds_cap)."""
    import oracle

    sub = batch_cpu_subset(trajs)
    t0 = time.perf_counter()
    pairs, frames, done = 0, 0, 0
    for tr in sub:
        for t in range(tr.T):
            oracle.frame(tr.verts[t], tr.faces, tr.frame_draws(t), tr.frame_targets(t),
                         details=False)
            pairs += tr.n(t) * tr.m(t)
            frames += 1
            if time.perf_counter() - t0 > seconds_cap:
                break
        else:
            done += 1
            continue
        break
    el = time.perf_counter() - t0
    return {"value": pairs / el, "unit": "pairs/s", "cores": oracle.num_threads(),
            "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"subset of the batch: trajectories 0, 8, ..., 56 ({len(sub)} of "
                      f"{len(trajs)}); {frames} whole frames ({done} whole trajectories), "
                      f"{pairs:.3e} pairs, loss + vertex gradient, FP64 with float32 neighbour "
                      f"decisions, {el:.1f} s"}


def run_batched(args, rank, world, dist):
    """64 trajectories of uneven sizes (the headline): the batched form (one planned launch
    sequence at the autotuned shape, replayed from a CUDA graph) against the plain per-frame
    form (one dc_loss_traj call per frame)."""
    import torch

    from paper_2204_03139_gb300 import _lib, autotune
    from paper_2204_03139_gb300.batch import BatchedLoss, DeviceTrajectory, per_frame_loss

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    trajs = make_workload("batched_uneven", rank=rank)
    if args.batch_trajectories:
        trajs = trajs[:args.batch_trajectories]
    pairs = sum(t.pairs() for t in trajs)
    frames = sum(t.T for t in trajs)
    dts = [DeviceTrajectory.from_host(t, dev) for t in trajs]
    mode = _lib.UNIDIR_SUM if args.mode == "eq2" else _lib.BIDIR_MEAN
    # the autotuner times every shape on this batch and plans with the fastest
    if args.shape:
        eng, wd = args.shape.split(":")
        tuning = {"best": (eng, int(wd)), "ms": {}}
    else:
        tuning = autotune.tune_batch(dts, mode=mode, grad=True, reps=2, save=False)
    shape = tuning["best"]
    b = BatchedLoss(dts, mode=mode, grad=True, graph=True, shape=shape)
    b.run(check=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    clocks = ClockSampler(local)
    for _ in range(max(3, args.warmup)):
        b.run()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    stream = torch.cuda.current_stream(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        b.run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    _lib.check_ws(b.ws)
    # graph replays launch nothing from the host: count and time the Chamfer kernel on the
    # same launch sequence issued eagerly on the batch's stream
    launches0 = _lib.launch_count()
    _lib.prof_start(3)
    with torch.cuda.stream(b.stream):
        for _ in range(3):
            b._launch()
    torch.cuda.synchronize()
    chamfer_ms, chamfer_n = _lib.prof_stop()
    launches = (_lib.launch_count() - launches0) // 3 * steps
    from paper_2204_03139_gb300.ranks import max_over_ranks

    per = [a.elapsed_time(c) for a, c in ev]
    ms = max_over_ranks(statistics.mean(per), dist)
    if args.kernels_only:
        if rank == 0:
            print(json.dumps({"workload": "batched_uneven", "ms_per_step": ms,
                              "pairs_per_s": world * pairs / (ms / 1e3),
                              "shape": list(shape), "kernel_ms": chamfer_ms / max(1, chamfer_n),
                              "gpu_launches": launches}), flush=True)
        return
    # the plain per-frame form on the same inputs, at the same shape
    with autotune.tuned(shape):
        per_frame_loss(dts, mode=mode)
        torch.cuda.synchronize()
        pf_steps = 2
        t0 = time.perf_counter()
        for _ in range(pf_steps):
            per_frame_loss(dts, mode=mode)
        torch.cuda.synchronize()
    pf_ms = 1e3 * (time.perf_counter() - t0) / pf_steps
    # end to end: the batch's inputs from pinned host memory each step, gradients and the
    # total back, the host reading each step's total. (1) One batch at a time: copies in,
    # the graph, copies out, synchronise.
    host = [(torch.from_numpy(t.verts).pin_memory(), torch.from_numpy(t.faces).pin_memory(),
             torch.from_numpy(t.draws).pin_memory(), torch.from_numpy(t.targets).pin_memory())
            for t in trajs]
    hg = [torch.empty(tuple(d.verts.shape), dtype=torch.float32).pin_memory() for d in dts]
    h2d = sum(v.numel() * 4 + f.numel() * 4 + d.numel() * 4 + y.numel() * 4
              for v, f, d, y in host)
    d2h = sum(g.numel() * 4 for g in hg) + 4
    e2e = []
    for _ in range(3):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for (hv, hf, hd, hy), d in zip(host, dts):
            d.verts.copy_(hv, non_blocking=True)
            d.faces.copy_(hf, non_blocking=True)
            d.draws.copy_(hd, non_blocking=True)
            d.targets.copy_(hy, non_blocking=True)
        tot = b.run()
        for g, gv in zip(hg, b.grad_verts):
            g.copy_(gv, non_blocking=True)
        float(tot[0])
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t1)
    sync_s = statistics.mean(e2e)
    # (2) The public BatchPipeline: while one batch computes, the next one's inputs are copied
    # in and the previous one's results out; the host reads each total before its buffers
    # are reused.
    from paper_2204_03139_gb300.pipeline import BatchPipeline

    del b  # the pipeline plans its own slots
    torch.cuda.empty_cache()
    pipe = BatchPipeline([(t.V, t.F, t.n_off, t.m_off) for t in trajs], device=dev, mode=mode,
                         depth=2, grad=True, shape=shape)
    houts = [([torch.empty(tuple(d.verts.shape), dtype=torch.float32).pin_memory()
               for d in dts], torch.empty(1, dtype=torch.float32).pin_memory())
             for _ in range(2)]

    def run_pipe(k_steps):
        pend = []
        for k in range(k_steps):
            if len(pend) == 2:  # the host buffers of step k - 2 are reused now: read its total
                ev, o = pend.pop(0)
                ev.synchronize()
                float(o[1][0])
            o = houts[k % 2]
            pend.append((pipe.submit(host, grads_out=o[0], total_out=o[1]), o))
        for ev, o in pend:
            ev.synchronize()
            float(o[1][0])

    run_pipe(2)
    n_pipe = 8
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    run_pipe(n_pipe)
    pipe_s = (time.perf_counter() - t1) / n_pipe
    if pipe.status() != _lib.DC_OK:
        raise RuntimeError("device-side error in the pipelined end-to-end run")
    del pipe
    piped = {"value": world * pairs / pipe_s, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
             "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * pipe_s, "steps": n_pipe,
             "api": "pipeline.BatchPipeline: every trajectory's verts, faces, draws and targets "
                    "copied in from pinned host memory, the planned batch replayed from a CUDA "
                    "graph, every gradient and the total copied out and the total read on the "
                    "host, consecutive batches overlapped on three streams"}
    synced = {"value": world * pairs / sync_s, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
              "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * sync_s, "steps": len(e2e),
              "api": "BatchedLoss.run (CUDA graph) with the same copies, one batch at a time: "
                     "copies in, the graph, copies out, synchronise"}
    e2e_best, e2e_other = (piped, synced) if pipe_s <= sync_s else (synced, piped)
    if rank != 0:
        return
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk.get("sm_mhz") or 0.0
    sm_max = clk.get("sm_max_mhz") or 0.0
    peak = (2 * FP32_LANES_PER_SM * props.multi_processor_count * sm_mhz * 1e6 / 1e12
            if sm_mhz else None)
    ck = chamfer_ms / max(1, chamfer_n) / 1e3
    ach = FLOP_PER_PAIR * pairs / ck / 1e12 if chamfer_n else None
    tc = shape[0] in ("tensor", "tcgen05")
    kernel = ({"tensor": "k_tcpass", "tcgen05": "k_tcpass5"}[shape[0]] if tc else
              ("k_chamfer<true>" if mode == _lib.BIDIR_MEAN else "k_chamfer<false>"))
    traffic = CHAMFER_TRAFFIC_BYTES.get(("batched_uneven", kernel, args.mode))
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if (ach and peak) else None,
            "traffic": traffic if not args.batch_trajectories else None,
            "kernel": kernel, "kernel_ms": ck * 1e3,
            "pairs_per_s_kernel": pairs / ck if chamfer_n else None,
            "accounting": "8 flop per unique (sim point, target) pair, the distance shared by "
                          "both directions, against the FP32 CUDA-core FMA peak 2 x "
                          f"{FP32_LANES_PER_SM} lanes x {props.multi_processor_count} SMs x "
                          f"median SM clock under load ({sm_mhz:.0f} MHz; {sm_max:.0f} MHz max)"}
    if tc:
        # the pass evaluates each pair once per direction on the tensor cores: one m16n8k16
        # MMA (4096 flop) per 128 pairs, in both directions for Eq. 1
        dirs = 2 if mode == _lib.BIDIR_MEAN else 1
        mma_tflops = dirs * 32.0 * pairs / ck / 1e12 if chamfer_n else None
        roof["note"] = ("the nearest-neighbour pass runs on the tensor cores (split-fp16 "
                        "expanded form, exact direct-form re-check of the candidates), so the "
                        "8-flop FP32 accounting can exceed the CUDA-core peak; the tensor "
                        "view is below")
        if shape[0] == "tcgen05":
            # tcgen05 f16 runs at the bf16 rate: the measured cuBLAS bf16 burst peak
            tpk = measured_peaks().get("bf16_tflops")
            roof["tensor"] = {"achieved": mma_tflops, "unit": "TFLOP/s (f16 MMA, 32 flop per "
                              "pair per direction)", "peak": tpk,
                              "peak_basis": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
                              "frac": (mma_tflops / tpk) if (mma_tflops and tpk) else None}
        else:
            # against the warp-level MMA rate this kernel can reach, and against the tensor
            # cores' measured peak (f16 at the bf16 rate), which only tcgen05 MMAs approach
            tpk = measured_peaks().get("bf16_tflops")
            roof["tensor"] = {"achieved": mma_tflops, "unit": "TFLOP/s (f16 MMA, 32 flop per "
                              "pair per direction)", "peak_mma_sync_measured": MMA_SYNC_TFLOPS,
                              "frac_of_mma_sync": (mma_tflops / MMA_SYNC_TFLOPS)
                              if mma_tflops else None,
                              "peak_tensor_measured": tpk,
                              "frac_of_tensor_peak": (mma_tflops / tpk)
                              if (mma_tflops and tpk) else None}
    line = {"metric": "chamfer_fwd_bwd_point_pairs_per_s", "value": world * pairs / (ms / 1e3),
            "unit": "pairs/s", "n_gpus": world, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {**batched_config(trajs, args, world),
                       "form": "one planned launch sequence replayed from a CUDA graph",
                       "shape": {"engine": shape[0], "warps_per_cta": shape[1],
                                 "tuned_ms": {f"{k[0]}:{k[1]}": v
                                              for k, v in tuning["ms"].items()}},
                       "l2": "flushed between timed steps (256 MiB write outside the step events)"},
            "comparison": {"plain_per_frame_ms_per_step": pf_ms,
                           "plain_per_frame_pairs_per_s": pairs / (pf_ms / 1e3),
                           "batched_over_plain": pf_ms / ms},
            "traj_loss_grad_per_s": world * len(trajs) * 1e3 / ms,
            "roofline": roof,
            "clocks": clk, "gpu_launches": launches,
            "e2e": e2e_best, "e2e_other": e2e_other}
    if not args.no_extra:
        line["trajectory_50x50"] = quick_trajectory_line(args, dev, mode)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(trajs)
    print(json.dumps(line), flush=True)


def quick_trajectory_line(args, dev, mode):
    """The 40-frame 50x50 trajectory (one dc_loss_traj with the gradient per step), a short
    run kept beside the batched headline."""
    import torch

    from paper_2204_03139_gb300 import _lib

    tr = make_workload("trajectory_50x50")
    T, V, F, N, M = tr.T, tr.V, tr.F, tr.n(0), tr.m(0)
    v = torch.from_numpy(tr.verts).to(dev)
    f = torch.from_numpy(tr.faces).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(tr.draws_tn3())).to(dev)
    y = torch.from_numpy(np.ascontiguousarray(tr.targets_tm3())).to(dev)
    out = {"ws": torch.empty(_lib.dc_workspace_size(T, V, F, N, M), dtype=torch.uint8,
                             device=dev)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(5):
        _lib.dc_loss_traj(v, f, d, y, mode=mode, out=out)
    torch.cuda.synchronize()
    steps = 50
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    _lib.prof_start(steps)
    for i in range(steps):
        flush.zero_()
        ev[i][0].record()
        _lib.dc_loss_traj(v, f, d, y, mode=mode, out=out)
        ev[i][1].record()
    torch.cuda.synchronize()
    kms, kn = _lib.prof_stop()
    _lib.check_ws(out["ws"])
    ms = statistics.mean(a.elapsed_time(c) for a, c in ev)
    return {"workload": tr.name, "ms_per_step": ms, "pairs_per_s": tr.pairs() / (ms / 1e3),
            "chamfer_kernel_ms": kms / max(kn, 1),
            "chamfer_pairs_per_s": tr.pairs() / (kms / max(kn, 1) / 1e3)}


def run_serving(args, rank, world, dist):
    """Poisson stream of loss+gradient requests: 90% at the 50x50 / 10 000-point size, 10% at
    the 100x100 / 32 768-point size, served with continuous batching under a 120 GB budget.
    Each rate runs a fixed arrival window; latencies include queueing."""
    import torch

    from paper_2204_03139_gb300.serve import Server, serve_plain

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    small = [workloads.lift_trajectory(workloads.SEED_BASE + 50 + k, 50, 40, 10_000, 10_000,
                                       name=f"small{k}") for k in range(4)]
    big = [workloads.trajectory_100x100(seed=workloads.SEED_BASE + 60)]
    window = float(os.environ.get("DC_SERVE_WINDOW_S", "1.0"))

    def arrivals(rate, seed):
        rng = workloads.rng_for(seed)
        t, out = 0.0, []
        while True:
            t += rng.exponential(1.0 / rate)
            if t > window:
                return out
            is_big = rng.random() < 0.1
            pool = big if is_big else small
            out.append((t, pool[int(rng.integers(len(pool)))]))

    def run_rate(rate, seed):
        reqs = arrivals(rate, seed)
        srv = Server(dev, hbm_budget=120 << 30, item_pairs=args.item_pairs,
                     max_batch_pairs=args.batch_pairs)
        futs = []
        t0 = time.perf_counter()
        for at, tr in reqs:
            now = time.perf_counter() - t0
            if now < at:
                time.sleep(at - now)
            futs.append(srv.submit(tr))
        res = [f.result(timeout=600) for f in futs]
        t_end = time.perf_counter() - t0
        srv.close()
        st = srv.stats()
        lat = np.array([r.latency_s for r in res])
        pairs = sum(tr.pairs() for _, tr in reqs)
        return {"rate_hz": rate, "requests": len(reqs), "window_s": window,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "throughput_pairs_per_s": pairs / t_end,
                "mean_batch_requests": float(np.mean([r.batch_requests for r in res])),
                "batches": st["batches"],
                "scheduler_host_ms_per_batch": st["host_ms_per_batch"],
                "scheduler_host_ms_per_batch_p99": st["host_ms_per_batch_p99"]}

    # warm-up: build pinned copies, first launches
    w = Server(dev, hbm_budget=120 << 30, item_pairs=args.item_pairs,
               max_batch_pairs=args.batch_pairs)
    for tr in small + big:
        w.submit(tr).result(timeout=600)
    w.close()
    rates = [500, 300, 250, 200, 100]
    results = [run_rate(r, 1000 + r) for r in rates]
    plain = []
    serve_plain(arrivals(100, 7)[:3], dev)  # warm-up
    for plain_rate in (200, 100):
        preqs = arrivals(plain_rate, 1000 + plain_rate)
        t0 = time.perf_counter()
        plat = np.array(serve_plain(preqs, dev))
        t_end = time.perf_counter() - t0
        plain.append({"rate_hz": plain_rate, "requests": len(preqs),
                      "p50_ms": float(np.percentile(plat, 50) * 1e3),
                      "p99_ms": float(np.percentile(plat, 99) * 1e3),
                      "throughput_pairs_per_s": sum(tr.pairs() for _, tr in preqs) / t_end})
    if rank != 0:
        return
    head = results[0]
    line = {"metric": "chamfer_fwd_bwd_point_pairs_per_s",
            "value": head["throughput_pairs_per_s"], "unit": "pairs/s", "n_gpus": world,
            "steps": head["requests"], "warmup": len(small) + len(big),
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_poisson", "item_pairs": args.item_pairs,
                       "batch_pairs": args.batch_pairs, "mix": "90% 50x50 T40 10k x 10k, "
                       "10% 100x100 T100 32768 x 32768", "hbm_budget_gb": 120,
                       "latency": "from arrival to the result on the host, queueing included"},
            "serving": results,
            "plain_per_request": plain}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td

        td.init_process_group("gloo")
        dist = td
    if args.impl == "reference":
        # the oracle pool runs before any GPU work (forking after CUDA init is unsafe)
        run_reference(args, rank, world)
    elif args.workload == "batched_uneven":
        run_batched(args, rank, world, dist)
    elif args.workload == "serving":
        run_serving(args, rank, world, dist)
    elif args.shape:
        from paper_2204_03139_gb300 import autotune

        eng, wd = args.shape.split(":")
        with autotune.tuned((eng, int(wd))):
            run_gpu(args, rank, world, dist)
    else:
        run_gpu(args, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
