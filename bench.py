#!/usr/bin/env python3
"""Spatial Pooler benchmark: frames/s and column-updates/s at 1024 columns x
256 synapses.

Headline workload (one "step" = one batch frame): the paper-scale frame SP --
960x540 blobbed binary frames (density U[5%,20%], 7x7 box blur), 1024
columns on a 32x32 grid of receptive-field centres, 256 potential synapses
from a 64x64 window, fp32 permanences U[0.1,0.3], threshold 0.2,
min_overlap 4, k 40 global inhibition, learning on (inc 0.05, dec 0.02) --
run as 256 independent SP instances per GPU (own pools, permanences and
frame streams), each computing one frame per step: overlap, inhibition and
learning for all 256 in one launch.  The 565 MB of SP state is far larger
than the 129 MB L2, so every step streams it from HBM (no flush needed).
Frames come from a pool of 64 seeded blobbed frames, instance i taking
frame (7 i + t) mod 64 at step t.

Secondary (`single_sp`): one such SP over a 500-frame learning sequence
(the latency-bound serial case), L2 flushed between steps.  `serve`: 32
simulated video streams (Poisson arrivals, 30 fps each, mixed 320x180 /
640x360 / 960x540) on the library's continuous-batching server -- frames/s
and per-frame latency p50/p99 in ms, open loop and at saturation.

Under torchrun every rank runs its own 256 instances (no cross-instance
exchange), so `value` is the sum over ranks (weak scaling).

`--impl reference` times the plain CPU oracle (the parity reference) on the
host cores on a bounded sample of the same workload.
"""
import argparse
import concurrent.futures as cf
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

INSTANCES = 256
REGIONS = 5  # timed regions of --steps steps each; the median is reported
FRAME_POOL = 64
SEQ_FRAMES = 500
WORKLOAD = ("paper-scale frame SP x 256 independent instances: 960x540 blobbed frames, "
            "1024 col x 256 syn (64x64 RF), k=40 global, learning on, one frame per instance per step")
METRIC = "SP frames/s (1024 col x 256 syn, 960x540 input, learning on)"


ALU_TOPS = 152 * 128 * 2.07e9 / 1e12  # int32 lane operations per second, in T


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--instances", type=int, default=INSTANCES)
    ap.add_argument("--seq-frames", type=int, default=SEQ_FRAMES)
    ap.add_argument("--no-single", action="store_true", help="skip the single-SP sequence")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense tensor-core run")
    ap.add_argument("--no-encoder", action="store_true", help="skip the frame-encoder runs")
    ap.add_argument("--per-frame-calls", action="store_true",
                    help="one API call (one launch) per step instead of one per run of steps")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default CTA split instead of autotuning it")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="serving workload run, open loop at 30 fps per stream (0 = skip)")
    ap.add_argument("--serve-sweep-seconds", type=float, default=3.0,
                    help="seconds of each load point of the serving sweep (0 = skip the sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def reduce_max(x, device=None):
    """Max over ranks of a float (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def instance_seed(rank, i):
    """Seed of SP i on `rank`: every rank steps its own, distinct SPs."""
    from paper_1608_01966_gb300 import workloads as wl
    return wl.BASE_SEED + 2 + 1000003 * rank + 17 * i


def make_cases(n, rank):
    """n frame-SP instances with their own seeds (generated in parallel: the
    generators are C code called without the GIL)."""
    from paper_1608_01966_gb300 import workloads as wl
    seeds = [instance_seed(rank, i) for i in range(n)]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        return list(ex.map(lambda s: wl.frame_case(seed=s), seeds))


def make_frame_pool(rank):
    from paper_1608_01966_gb300 import synth, workloads as wl
    seed = wl.BASE_SEED + 2 + 1000003 * rank
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        fr = list(ex.map(lambda t: synth.frame_blobbed(
            synth.derive_seed(seed, synth.PURPOSE_FRAME, t), 960, 540), range(FRAME_POOL)))
    fr = np.stack(fr)
    return fr, wl.pack(fr)


def algorithmic_bytes_per_frame(case, learn=True):
    """Bytes one SP frame must move at minimum in the canonical layout: the
    pools and permanences (4 B each per synapse), the packed frame, the
    overlaps written, the winner list and, when learning, the winners'
    permanence rows written back."""
    b = case.C * case.S * 4 * 2 + case.n_words * 4 + case.C * 4 + case.k * 4
    if learn:
        b += case.k * case.S * 4
    return b


def compact_form(case):
    """Whether an SP qualifies for the compact form: 16-bit pool offsets from
    a per-column base plus one connected bit per synapse (S up to 256, rows
    padded to a multiple of 32 synapses, every pool spanning at most 65536
    inputs)."""
    if os.environ.get("SP_BATCH_COMPACT", "1").startswith("0"):
        return False
    if case.S > 256:
        return False
    return int((case.idx.max(axis=1) - case.idx.min(axis=1)).max()) <= 0xFFFF


FORM_TEXT = {
    "window": "window: per column a 64x64 bitmap of connected synapses + box origin, counted "
              "against the CTA's frame rows in shared memory; fp32 permanences touched only by "
              "learning columns",
    "compact": "compact: 16-bit pool offsets + connected bits, fp32 permanences touched only by "
               "learning columns",
    "full": "full: 32-bit pools + fp32 permanences",
}


def window_bytes_per_frame(case, learn=True):
    """Bytes one SP frame moves on the window form: per column a 512-byte
    bitmap of connected synapses and a box origin, the frame, the overlaps,
    the winner list and, when learning, the winners' pool indices read,
    permanences read and written, and bitmaps rewritten."""
    b = case.C * 512 + case.C * 4 + case.n_words * 4 + case.C * 4 + case.k * 4
    if learn:
        b += case.k * (case.S * 4 * 3 + 512)
    return b


def form_bytes_per_frame(case, form, learn=True):
    """Algorithmic bytes of one SP frame in the form the batch runs it on
    (a name of FORM_NAMES, as sp_batch_forms reports it)."""
    if form == "window":
        return window_bytes_per_frame(case, learn)
    if form == "compact":
        return compact_bytes_per_frame(case, learn)
    return algorithmic_bytes_per_frame(case, learn)


def compact_bytes_per_frame(case, learn=True):
    """Bytes one SP frame moves on the compact form: offsets (2 B) and
    connected bits (1/8 B) per synapse of rows padded to a multiple of 32, a
    base per column, the frame, the overlaps, the winner list and, when
    learning, the winners' permanence rows read and written plus their
    connected bits rewritten."""
    sp = (case.S + 31) // 32 * 32
    b = (case.C * sp * 2 + case.C * sp // 8 + case.C * 4 + case.n_words * 4
         + case.C * 4 + case.k * 4)
    if learn:
        b += case.k * case.S * 8 + case.k * sp // 8
    return b


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("sp_step.cu", "sp_kernels.cuh", "sp_device.cuh", "sp_abi.cu"):
        with open(os.path.join(ROOT, "paper_1608_01966_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel):
    """DRAM bytes per step (one batch frame) of the batch kernel from the
    committed ncu summary, only while the kernel source is unchanged since
    the capture and the capture is of the same kernel."""
    try:
        with open(os.path.join(ROOT, "profiles", "sp_batch_step_traffic.json")) as f:
            d = json.load(f)
        if d.get("source_sha") == kernel_source_sha() and d.get("kernel") == kernel:
            return d.get("dram_bytes_per_step")
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


def oracle_sample(cases, pool_u8, seconds, start_step=0):
    """The oracle as it stands (one thread), instance by instance in the
    headline workload's order (step t: instance i on frame (7 i + t) mod 64),
    until `seconds` elapse.  Returns (SP frames/s, SP frames done)."""
    import oracle
    states = {}
    done = 0
    t0 = time.perf_counter()
    step = start_step
    while True:
        for i, c in enumerate(cases):
            if i not in states:
                states[i] = (oracle.params(c.C, c.S, c.n_in, c.thr, c.inc, c.dec, c.min_overlap,
                                           c.k), c.perm.copy())
            p, perm = states[i]
            fr = pool_u8[(7 * i + step) % FRAME_POOL]
            oracle.run(p, c.idx, perm, c.boost, fr[None, :], True)
            done += 1
            if time.perf_counter() - t0 >= seconds:
                return done / (time.perf_counter() - t0), done
        step += 1


def oracle_sample_parallel(cases, pool_u8, seconds, threads):
    """The same oracle on `threads` host threads, each stepping its own
    instances in order (the SPs are independent; the oracle's C code runs
    without the GIL).  Returns (SP frames/s over all threads, frames done)."""
    import threading
    import oracle
    stop = time.perf_counter() + seconds
    counts = [0] * threads

    def work(j):
        mine = [(i, c, oracle.params(c.C, c.S, c.n_in, c.thr, c.inc, c.dec, c.min_overlap, c.k),
                 c.perm.copy()) for i, c in enumerate(cases) if i % threads == j]
        step = 0
        while time.perf_counter() < stop:
            for i, c, p, perm in mine:
                oracle.run(p, c.idx, perm, c.boost, pool_u8[(7 * i + step) % FRAME_POOL][None, :],
                           True)
                counts[j] += 1
                if time.perf_counter() >= stop:
                    return
            step += 1

    ts = [threading.Thread(target=work, args=(j,)) for j in range(threads)]
    t0 = time.perf_counter()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    el = time.perf_counter() - t0
    return sum(counts) / el, sum(counts)


def run_uneven_batch(spg, torch, dev, stream, members=64, frames=16, steps=5):
    """64 independent SPs of uneven shapes (columns 128..4096, synapses
    16..256, inputs 256..16384 bits at 2-20 % density, k = 2 % of columns,
    learning on), stepped by persistent launches of 16 frames: once with the
    default schedule and splits, once autotuned (each from fresh handles)."""
    from paper_1608_01966_gb300 import workloads as wl
    cases, dens = wl.uneven_cases(members)
    fr = [wl.pack(f) for f in wl.uneven_frames(cases, dens, frames)]

    def timed(tune):
        hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
        b = spg.sp_batch_create(hs)
        info = spg.sp_batch_get_info(b)
        fo, _ = spg.sp_batch_offsets(b)
        fw = (info["frame_words"] + 3) // 4 * 4
        d = torch.from_numpy(wl.batch_frames(fr, fo, fw).view(np.int32)).to(dev)
        mw = info["mask_words"]
        dm = torch.zeros((frames, mw), dtype=torch.int32, device=dev)
        cpw = spg.sp_batch_autotune(b, d, 4, fw) if tune else 0
        sched = spg.sp_batch_schedule(b, len(hs))
        spg.sp_batch_compute_device(b, d, frames, fw, True, dm, mw, stream)
        spg.sp_batch_sync(b)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(steps):
            spg.sp_batch_compute_device(b, d, frames, fw, True, dm, mw, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / (steps * frames)
        forms_b = spg.sp_batch_forms(b)
        spg.sp_batch_destroy(b)
        for h in hs:
            spg.sp_destroy(h)
        return ms, cpw, sched, forms_b

    ms0, _, _, _ = timed(False)
    ms, cpw, sched, forms_b = timed(True)
    upd = sum(c.C for c in cases)
    peak, kind = read_peaks()
    forms = [spg.FORM_NAMES[int(f)] for f in forms_b]
    moved = sum(form_bytes_per_frame(c, f) for c, f in zip(cases, forms))
    gbs = moved / (ms / 1000.0) / 1e9
    per = sched[2]
    return {"workload": f"{members} uneven SPs (C 128..4096, S 16..256, inputs 256..16384 bits), "
                        f"learning on, {frames} frames per persistent launch, autotuned",
            "schedule": {"ctas_per_sm": sched[0], "cols_in_flight": sched[1],
                         "cols_per_warp": cpw if cpw != spg.SP_MIXED_SPLIT else "per member",
                         "member_cols_per_warp": {str(v): per.count(v) for v in sorted(set(per))}},
            "us_per_batch_frame": ms * 1000.0,
            "default_schedule_us_per_batch_frame": ms0 * 1000.0,
            "tuning_gain": ms0 / ms,
            "frames_per_s": members / (ms / 1000.0),
            "column_updates_per_s": upd / (ms / 1000.0),
            "roofline": {"bound": "hbm", "kernel": "sp_batch_run_kernel", "achieved": gbs,
                         "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": kind,
                         "form_bytes_per_batch_frame": moved,
                         "forms": {f: forms.count(f) for f in sorted(set(forms))}}}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    n_sample = 8  # instances per reference step (bounded sample of the 256-instance step)
    cases = make_cases(n_sample, 0)
    pool_u8, _ = make_frame_pool(0)
    import oracle
    params = [oracle.params(c.C, c.S, c.n_in, c.thr, c.inc, c.dec, c.min_overlap, c.k)
              for c in cases]
    perms = [c.perm.copy() for c in cases]

    def step(t):
        for i, c in enumerate(cases):
            oracle.run(params[i], c.idx, perms[i], c.boost,
                       pool_u8[(7 * i + t) % FRAME_POOL][None, :], True)

    for w in range(args.warmup):
        step(w)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        step(args.warmup + s)
        times.append(time.perf_counter() - t0)
    fps = n_sample * len(times) / sum(times)
    ms = 1000.0 * sum(times) / len(times) * (args.instances / n_sample)
    sample = f"{n_sample} of the {args.instances} instances per step, one frame each, one thread"
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": args.instances},
        "column_updates_per_s": fps * 1024,
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_single_sp(spg, torch, case, pool_packed, n_frames, steps, dev, stream):
    """One SP over an n_frames learning sequence (frames cycled from the
    pool), L2 flushed between steps; returns (frames/s, us per frame)."""
    idx = [t % FRAME_POOL for t in range(n_frames)]
    frames = np.ascontiguousarray(pool_packed[idx])
    d = torch.from_numpy(frames.view(np.int32)).to(dev)
    dm = torch.zeros((n_frames, (case.C + 31) // 32), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    for _ in range(3):
        spg.sp_compute_frames_device(h, d, n_frames, frames.shape[1], True, dm, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for s in range(steps):
        flush.fill_(s)
        ev[s][0].record(stream)
        spg.sp_compute_frames_device(h, d, n_frames, frames.shape[1], True, dm, stream)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    spg.sp_destroy(h)
    del flush
    return n_frames / (ms / 1000.0), ms * 1000.0 / n_frames


def read_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# Nominal dense fp8 / bf16 tensor rate on this part (4.5 / 2.25 PFLOP/s).
FP8_PER_BF16 = 2.0


def run_dense_tc(spg, torch, dev, stream, members=16, frames=256, steps=5):
    """16 SPs with dense pools (1024 inputs x 1024 columns, k = 20) inferring
    256 frames each: the frames' e4m3 image, one tensor-core launch for all
    overlaps (16 x 256 x 1024 x 1024 multiply-adds of {0,1} e4m3 operands)
    and one Alg. 2 launch per run; the connection images are built once (the
    permanences do not change without learning)."""
    from paper_1608_01966_gb300 import workloads as wl
    n_in, C = 1024, 1024
    cases, fr = wl.dense_cases(members, frames, C=C, n_in=n_in)
    packed = [wl.pack(f) for f in fr]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, _ = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    d = torch.from_numpy(wl.batch_frames(packed, fo, fw).view(np.int32)).to(dev)
    mw = info["mask_words"]
    dm = torch.zeros((frames, mw), dtype=torch.int32, device=dev)
    for _ in range(3):
        spg.sp_batch_infer_device(b, d, frames, fw, dm, mw, stream)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(steps):
        spg.sp_batch_infer_device(b, d, frames, fw, dm, mw, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    spg.sp_batch_destroy(b)
    for h in hs:
        spg.sp_destroy(h)
    flops = 2.0 * members * frames * C * n_in
    bf16, kind = read_bf16_peak()
    peak = bf16 * FP8_PER_BF16
    kind += " bf16 x nominal fp8/bf16 ratio 2"
    tf = flops / (ms / 1000.0) / 1e12
    return {"workload": f"{members} dense SPs (1024 inputs x 1024 columns) x {frames} frames, "
                        "inference, tensor cores (tcgen05 kind::f8f6f4, e4m3 {0,1}, fp32 accumulate)",
            "ms_per_run": ms, "frames_per_s": members * frames / (ms / 1000.0),
            "tensor": {"achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                       "peak_kind": kind}}


def run_batched_mixed(spg, torch, dev, stream, frames=256, steps=5):
    """The batched workload as one call: the 64 uneven SPs and the 16 dense SPs
    (1024 x 1024) in one batch, inference over 256 frames per
    sp_batch_infer_device call (tensor cores for the dense members, one
    persistent launch for the others)."""
    from paper_1608_01966_gb300 import workloads as wl
    unv, dens = wl.uneven_cases(64)
    dcases, dfr = wl.dense_cases(16, frames)
    cases = unv + dcases
    fr = wl.uneven_frames(unv, dens, frames) + dfr
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, _ = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    d = torch.from_numpy(wl.batch_frames([wl.pack(f) for f in fr], fo, fw).view(np.int32)).to(dev)
    mw = info["mask_words"]
    dm = torch.zeros((frames, mw), dtype=torch.int32, device=dev)
    for _ in range(3):
        spg.sp_batch_infer_device(b, d, frames, fw, dm, mw, stream)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(steps):
        spg.sp_batch_infer_device(b, d, frames, fw, dm, mw, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / steps
    forms = [spg.FORM_NAMES[int(f)] for f in spg.sp_batch_forms(b)]
    spg.sp_batch_destroy(b)
    for h in hs:
        spg.sp_destroy(h)
    n = len(cases)
    return {"workload": f"64 uneven SPs + 16 dense SPs (1024 x 1024) in one batch, inference, "
                        f"{frames} frames per call (dense members on the tensor cores, the others "
                        "in one persistent launch)",
            "ms_per_call": ms, "frames_per_s": n * frames / (ms / 1000.0),
            "column_updates_per_s": sum(c.C for c in cases) * frames / (ms / 1000.0),
            "forms": {f: forms.count(f) for f in sorted(set(forms))}}


def run_encoder(spg, torch, dev, stream, n_frames=128, steps=5, reduce=1):
    """Frame encoder over n_frames 960x540 colour frames in one call (inputs
    larger than L2), then the encoder feeding one frame-shaped SP (learning
    on) from device frames and from pinned host frames."""
    from paper_1608_01966_gb300 import synth, workloads as wl
    uniq = wl.rgb_frames(16, 960, 540, seed=wl.BASE_SEED + 6)
    frames = np.ascontiguousarray(uniq[np.arange(n_frames) % 16].reshape(n_frames, -1))
    e = spg.sp_encoder_create(spg.sp_encoder_config_init(reduce=reduce))
    info = spg.sp_encoder_get_info(e)
    fb, words = info["src_bytes"], info["out_words"]
    d_src = torch.from_numpy(frames).to(dev)
    d_bits = torch.zeros((n_frames, words), dtype=torch.int32, device=dev)
    for _ in range(3):
        spg.sp_encode_device(e, d_src, n_frames, fb, d_bits, words, stream)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(steps):
        spg.sp_encode_device(e, d_src, n_frames, fb, d_bits, words, stream)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_enc = s0.elapsed_time(s1) / steps
    out = {"workload": f"{n_frames} colour frames 960x540 (RGB, 1.56 MB each) per call, "
                       f"reduce {reduce} -> {info['out_w']}x{info['out_h']}, 11x11 binomial "
                       "window, offset 2",
           "frames_per_s": n_frames / (ms_enc / 1000.0), "us_per_frame": ms_enc * 1000.0 / n_frames}
    peak, kind = read_peaks()
    gbs = n_frames * (fb + words * 4) / (ms_enc / 1000.0) / 1e9
    # integer operations per output pixel: block sums (3 per source pixel),
    # luma (3), two 11-tap binomial passes (22), rounding and compare (3)
    ops_px = 3 * reduce * reduce + 3 + 22 + 3
    tops = n_frames * info["out_bits"] * ops_px / (ms_enc / 1000.0) / 1e12
    t_hbm = (fb + words * 4) / (peak * 1e9)
    t_alu = info["out_bits"] * ops_px / (ALU_TOPS * 1e12)
    if t_alu > t_hbm:
        out["roofline"] = {"bound": "alu", "kernel": "sp_encode_kernel", "achieved": tops,
                           "peak": ALU_TOPS, "unit": "Tops/s", "frac": tops / ALU_TOPS,
                           "peak_kind": "derived: 152 SMs x 128 int32 lanes x 2.07 GHz",
                           "int_ops_per_output_pixel": ops_px, "hbm_gbs": gbs}
    else:
        out["roofline"] = {"bound": "hbm", "kernel": "sp_encode_kernel", "achieved": gbs,
                           "peak": peak, "unit": "GB/s", "frac": gbs / peak, "peak_kind": kind,
                           "algorithmic_bytes_per_frame": int(fb + words * 4)}
    if reduce == 1:
        case = wl.frame_case()
        h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
        mw = spg.sp_get_info(h)["mask_words"]
        d_masks = torch.zeros((n_frames, mw), dtype=torch.int32, device=dev)
        for _ in range(2):
            spg.sp_encode_compute_device(e, h, d_src, n_frames, fb, True, d_masks, stream)
        torch.cuda.synchronize()
        s0.record(stream)
        for _ in range(steps):
            spg.sp_encode_compute_device(e, h, d_src, n_frames, fb, True, d_masks, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / steps
        out["with_sp"] = {"frames_per_s": n_frames / (ms / 1000.0),
                          "us_per_frame": ms * 1000.0 / n_frames,
                          "workload": "encoder + one paper-scale frame SP (1024 x 256, k 40, "
                                      "learning) on device frames"}
        pinned = torch.from_numpy(frames).pin_memory().numpy()
        masks = np.zeros((n_frames, mw), np.uint32)
        spg.sp_encode_compute(e, h, pinned, True, masks)
        t0 = time.perf_counter()
        for _ in range(steps):
            spg.sp_encode_compute(e, h, pinned, True, masks)
        dt = (time.perf_counter() - t0) / steps
        out["with_sp"]["e2e"] = {"frames_per_s": n_frames / dt, "h2d_bytes_per_frame": int(fb),
                                 "d2h_bytes_per_frame": int(mw * 4),
                                 "note": "pinned host colour frames in, active-column masks out"}
        spg.sp_destroy(h)
    spg.sp_encoder_destroy(e)
    del d_src, d_bits
    return out


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
    stream = torch.cuda.Stream(dev)  # a dedicated stream: events and kernels share it
    torch.cuda.set_stream(stream)

    n = args.instances
    cases = make_cases(n, rank)
    pool_u8, pool_packed = make_frame_pool(rank)
    handles = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(handles)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    mw = info["mask_words"]
    # every distinct batch frame a step can see: step t uses pattern t mod 64
    nw = pool_packed.shape[1]
    batch = np.zeros((FRAME_POOL, fw), np.uint32)
    for t in range(FRAME_POOL):
        for i in range(n):
            o = int(fo[i])
            batch[t, o:o + nw] = pool_packed[(7 * i + t) % FRAME_POOL]
    d_batch = torch.from_numpy(batch.view(np.int32)).to(dev)
    d_masks = torch.zeros((FRAME_POOL, mw), dtype=torch.int32, device=dev)
    cols_per_warp = None
    if not args.no_autotune:  # set-up, outside the timed region
        cols_per_warp = spg.sp_batch_autotune(b, d_batch, 8, fw)
        info = spg.sp_batch_get_info(b)
    sched = spg.sp_batch_schedule(b, n)
    forms = [spg.FORM_NAMES[int(f)] for f in spg.sp_batch_forms(b)]

    def step(t):
        r = t % FRAME_POOL
        spg.sp_batch_compute_device(b, d_batch[r], 1, fw, True, d_masks[r], mw, stream)

    def steps(t0, k):
        """k consecutive steps from step t0: one call per run of pool frames
        (a call over several frames is one persistent launch)."""
        if args.per_frame_calls:
            for t in range(t0, t0 + k):
                step(t)
            return
        t = t0
        while t < t0 + k:
            r = t % FRAME_POOL
            m = min(t0 + k - t, FRAME_POOL - r)
            spg.sp_batch_compute_device(b, d_batch[r], m, fw, True, d_masks[r], mw, stream)
            t += m

    warm = max(3, args.warmup)
    steps(0, warm)
    spg.sp_batch_sync(b)
    torch.cuda.synchronize()

    # REGIONS timed regions of exactly K steps each (CUDA events on the
    # launching stream, barrier + synchronize on both sides); the line reports
    # the median region, max over ranks
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    # about a second of the same steps under the clock sampler before the
    # regions, so the samples see the GPU under this load (untimed)
    t_next = warm
    t_end = time.perf_counter() + 1.0
    while time.perf_counter() < t_end:
        steps(t_next, args.steps)
        t_next += args.steps
        torch.cuda.synchronize()
    region_ms, launches = [], 0
    for _ in range(REGIONS):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        launches0 = spg.sp_kernel_launch_count()
        start.record(stream)
        steps(t_next, args.steps)
        end.record(stream)
        torch.cuda.synchronize()
        launches = spg.sp_kernel_launch_count() - launches0
        t_next += args.steps
        region_ms.append(reduce_max(start.elapsed_time(end) / args.steps, dev))
    clk = clocks.stop()
    ms = statistics.median(region_ms)
    if world > 1:
        dist.barrier()
    value = world * n / (ms / 1000.0)

    # end to end through the public API with host buffers: every step's batch
    # frame copied in from pinned memory and its mask record copied back
    # copy-in of the first chunk and compute of the last amortised over the run;
    # the copies (about 200 GB/s from pinned host memory here) bound the rest
    e2e_steps = max(4, min(3 * args.steps, 96))
    h_frames = torch.from_numpy(
        np.ascontiguousarray(batch[np.arange(e2e_steps) % FRAME_POOL]).view(np.int32)).pin_memory()
    h_masks = torch.zeros((e2e_steps, mw), dtype=torch.int32).pin_memory()
    hf = h_frames.numpy().view(np.uint32)
    hm = h_masks.numpy().view(np.uint32)
    spg.sp_batch_compute(b, hf, True, hm)  # warm the staging buffers
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    spg.sp_batch_compute(b, hf, True, hm)
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dev)
    e2e_value = world * n / e2e_s

    spg.sp_batch_destroy(b)
    for h in handles:
        spg.sp_destroy(h)
    del d_batch, d_masks

    single = None
    if not args.no_single:
        fps1, us1 = run_single_sp(spg, torch, cases[0], pool_packed, args.seq_frames, 5, dev,
                                  stream)
        single = {"workload": f"one paper-scale frame SP, {args.seq_frames}-frame learning "
                              "sequence, state in one 16-CTA cluster's shared memory, L2 flushed "
                              "between steps",
                  "frames_per_s": fps1, "us_per_frame": us1}

    dense_tc = None
    if not args.no_dense:
        dense_tc = run_dense_tc(spg, torch, dev, stream)

    uneven = mixed = None
    if not args.no_dense:
        uneven = run_uneven_batch(spg, torch, dev, stream)
        mixed = run_batched_mixed(spg, torch, dev, stream)

    encoder = None
    if not args.no_encoder:
        encoder = [run_encoder(spg, torch, dev, stream, reduce=1),
                   run_encoder(spg, torch, dev, stream, reduce=4)]

    serve = None
    if args.serve_seconds > 0 and rank == 0:
        from paper_1608_01966_gb300 import serve_sim
        serve = serve_sim.simulate(streams=32, fps=30.0, seconds=args.serve_seconds,
                                   saturate_seconds=3.0, sweep_seconds=args.serve_sweep_seconds)

    peak, peak_kind = read_peaks()
    canonical = sum(algorithmic_bytes_per_frame(c) for c in cases)
    moved = sum(form_bytes_per_frame(c, f) for c, f in zip(cases, forms))
    # the algorithmic bytes of the form the kernel runs on, per step, over
    # the average time of a step
    achieved = moved / (ms / 1000.0) / 1e9
    persistent = (not args.per_frame_calls and args.steps > 1
                  and os.environ.get("SP_DISABLE_PERSISTENT", "0") != "1")
    kernel_name = "sp_batch_run_kernel" if persistent else "sp_batch_step_kernel"
    steps_per_launch = (args.steps / max(1, launches)) if persistent else 1
    traffic = read_traffic(kernel_name)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps_cpu, done = oracle_sample(cases[:16], pool_u8, args.cpu_seconds)
        cpu = {"value": fps_cpu, "unit": "frames/s", "cores": 1, "kind": "oracle",
               "sample": f"{done} SP frames of the same workload (first 16 instances in step "
                         f"order), one thread, ~{args.cpu_seconds:.0f} s"}
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (
            os.cpu_count() or 1)
        fps_all, done_all = oracle_sample_parallel(cases[:max(16, threads)], pool_u8,
                                                   args.cpu_seconds / 2, threads)
        cpu["all_cores"] = {"value": fps_all, "unit": "frames/s", "cores": threads,
                            "cores_note": "the cores this process may run on (its affinity "
                                          f"mask); the host reports {os.cpu_count()}",
                            "sample": f"{done_all} SP frames, instances split over {threads} "
                                      f"threads, ~{args.cpu_seconds / 2:.0f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "columns": 1024, "synapses": 256,
                       "input": "960x540", "winners_set_size": 40, "learn": True,
                       "instances_per_gpu": n, "frames_per_step_per_instance": 1,
                       "cols_per_warp": (cols_per_warp if cols_per_warp != spg.SP_MIXED_SPLIT
                                         else "per member"),
                       "autotuned": cols_per_warp is not None,
                       "schedule": {"ctas_per_sm": sched[0], "cols_in_flight": sched[1]},
                       "ctas_per_launch": int(info["ctas"]),
                       "state_bytes_per_gpu": int(sum(c.C * c.S * 8 for c in cases)),
                       "l2": "inputs larger than L2 (SP state streamed every step), no flush",
                       "parallelism": f"{world} GPU(s) x {n} independent instances"},
            "column_updates_per_s": value * 1024,
            "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "algorithmic_bytes_per_step": moved,
                         "form": FORM_TEXT[forms[0]] if len(set(forms)) == 1 else
                                 {f: forms.count(f) for f in sorted(set(forms))},
                         "traffic_over_algorithmic": (traffic / moved) if traffic else None,
                         "canonical_bytes_per_step": canonical,
                         "canonical_equiv_frac": canonical / (ms / 1000.0) / 1e9 / peak,
                         "avg_us_per_step": ms * 1000.0,
                         "region_us_per_step": [r * 1000.0 for r in region_ms],
                         "steps_per_launch": steps_per_launch},
            "e2e": {"value": e2e_value, "unit": "frames/s",
                    "h2d_bytes_per_step": int(info["frame_words"] * 4),
                    "d2h_bytes_per_step": int(mw * 4)},
            "gpu_launches": int(launches),
            "clocks": clk,
            "single_sp": single,
            "dense_tc": dense_tc,
            "uneven_batch": uneven,
            "batched_mixed": mixed,
            "encoder": encoder,
            "serve": serve,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
