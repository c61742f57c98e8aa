#!/usr/bin/env python3
"""Spatial Pooler benchmark: frames/s and column-updates/s at 1024 columns x
256 synapses.

Workload (one "step"): the paper-scale frame SP -- 960x540 blobbed binary
frames (density U[5%,20%], 7x7 box blur), 1024 columns on a 32x32 grid of
receptive-field centres, 256 potential synapses from a 64x64 window, fp32
permanences U[0.1,0.3], threshold 0.2, min_overlap 4, k 40 global
inhibition -- run over a 500-frame sequence with learning on (inc 0.05,
dec 0.02).  Frames are synthetic (seeded) and packed 32 bits per word.  Each
step is the whole hot path (overlap, inhibition, learning) for 500 frames,
one fused kernel per frame, with the frames and SP state resident in HBM.
L2 (129 MB, larger than state + frames) is flushed by a 256 MiB write
between timed steps.

Under torchrun each rank runs its own independent SP instance (the path has
no cross-instance exchange), so `value` is the sum over ranks (weak scaling).

`--impl reference` times the plain CPU oracle (the parity reference) on the
host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FRAMES = 500
WORKLOAD = "paper-scale frame SP: 960x540 blobbed frames, 1024 col x 256 syn (64x64 RF), k=40 global, learn on, 500-frame sequence"
METRIC = "SP frames/s (1024 col x 256 syn, 960x540 input, learning on)"
STEP_KERNEL = "sp_step_kernel"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=N_FRAMES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def build_inputs(rank, n_frames):
    from paper_1608_01966_gb300 import workloads as wl
    seed = wl.BASE_SEED + 2 + 1000 * rank
    case = wl.frame_case(seed=seed)
    frames = wl.blob_frames(n_frames, seed=seed)
    return case, frames, wl.pack(frames)


def algorithmic_bytes_per_frame(case, learn=True):
    """Bytes one frame must move at minimum in the canonical layout: the
    pools and permanences (4 B each per synapse), the packed frame, the
    overlaps written, the winner list and, when learning, the winners'
    permanence rows written back."""
    b = case.C * case.S * 4 * 2 + case.n_words * 4 + case.C * 4 + case.k * 4
    if learn:
        b += case.k * case.S * 4
    return b


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("sp_step.cu", "sp_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1608_01966_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu
    summary, only if the kernel source is unchanged since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "sp_step_traffic.json")) as f:
            d = json.load(f)
        if d.get("source_sha") == kernel_source_sha():
            return d.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def time_oracle(case, frames_u8, seconds):
    """Time the oracle (as it stands, one thread) over whole passes of the
    frame sequence until `seconds` elapse; returns (frames/s, frames done)."""
    import oracle
    p = oracle.params(case.C, case.S, case.n_in, case.thr, case.inc, case.dec,
                      case.min_overlap, case.k, case.inhibition, case.gw, case.gh, case.radius)
    perm = case.perm.copy()
    done = 0
    t0 = time.perf_counter()
    chunk = 25
    while True:
        for i in range(0, frames_u8.shape[0], chunk):
            oracle.run(p, case.idx, perm, case.boost, frames_u8[i:i + chunk], True)
            done += min(chunk, frames_u8.shape[0] - i)
            if time.perf_counter() - t0 >= seconds:
                return done / (time.perf_counter() - t0), done


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    case, frames, _ = build_inputs(0, args.frames)
    import oracle
    p = oracle.params(case.C, case.S, case.n_in, case.thr, case.inc, case.dec,
                      case.min_overlap, case.k)
    sample = 25  # frames per reference step (bounded sample of the 500-frame step)
    perm = case.perm.copy()
    for w in range(args.warmup):
        oracle.run(p, case.idx, perm, case.boost, frames[:sample], True)
    times = []
    for s in range(args.steps):
        i0 = (s * sample) % (args.frames - sample + 1)
        t0 = time.perf_counter()
        oracle.run(p, case.idx, perm, case.boost, frames[i0:i0 + sample], True)
        times.append(time.perf_counter() - t0)
    fps = sample * len(times) / sum(times)
    ms = 1000.0 * sum(times) / len(times) * (args.frames / sample)
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": args.frames},
        "column_updates_per_s": fps * case.C,
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": f"{sample} frames of the 500-frame sequence per step, one thread"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    import paper_1608_01966_gb300 as spg

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    case, frames_u8, packed = build_inputs(rank, args.frames)
    n, nw = packed.shape
    mw = (case.C + 31) // 32
    stream = torch.cuda.Stream(dev)  # a dedicated stream: events and kernels share it
    torch.cuda.set_stream(stream)
    d_frames = torch.from_numpy(packed.view(np.int32)).to(dev)
    d_masks = torch.zeros((n, mw), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)

    def step():
        spg.sp_compute_frames_device(h, d_frames, n, nw, True, d_masks, stream)

    for _ in range(max(3, args.warmup)):
        step()
    spg.sp_sync(h)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = spg.sp_kernel_launch_count()
    for s in range(args.steps):
        flush.fill_(s)  # L2 flush, outside the step's events
        starts[s].record(stream)
        step()
        ends[s].record(stream)
    torch.cuda.synchronize()
    launches = spg.sp_kernel_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms_local = sum(step_ms) / len(step_ms)
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms_local], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    else:
        ms = ms_local
    value = world * n / (ms / 1000.0)

    # end to end through the public API with host buffers (pinned frames in,
    # active masks out), every copy inside the timed region
    h_frames = torch.from_numpy(packed.view(np.int32)).pin_memory()
    h_masks = torch.zeros((n, mw), dtype=torch.int32).pin_memory()
    hf = h_frames.numpy().view(np.uint32)
    hm = h_masks.numpy().view(np.uint32)
    spg.sp_compute_frames(h, hf, True, hm)  # warm the staging buffers
    e2e_steps = max(1, min(args.steps, 5))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        spg.sp_compute_frames(h, hf, True, hm)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * n / e2e_s

    spg.sp_destroy(h)

    peak, peak_kind = read_peaks()
    per_launch = algorithmic_bytes_per_frame(case, learn=True)
    kernel_launches_per_step = n
    avg_launch_s = (ms / 1000.0) / kernel_launches_per_step
    achieved = per_launch / avg_launch_s / 1e9
    traffic = read_traffic()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps_cpu, done = time_oracle(case, frames_u8, args.cpu_seconds)
        cpu = {"value": fps_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} frames of the same 500-frame learning sequence, one thread, ~{args.cpu_seconds:.0f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "columns": case.C, "synapses": case.S,
                       "input": "960x540", "winners_set_size": case.k, "learn": True,
                       "frames_per_step": n, "instances_per_gpu": 1,
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"{world} independent instance(s), one per GPU"},
            "column_updates_per_s": value * case.C,
            "us_per_frame": ms * 1000.0 / n,
            "roofline": {"bound": "hbm", "kernel": STEP_KERNEL, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_launch": per_launch,
                         "avg_launch_us": avg_launch_s * 1e6},
            "e2e": {"value": e2e_value, "unit": "frames/s",
                    "h2d_bytes_per_step": int(n * nw * 4), "d2h_bytes_per_step": int(n * mw * 4)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
