"""Simulated video-stream serving on the library's server (sp_server_*).

S streams (default 32) with Poisson frame arrivals (default mean 30 fps
each) at round-robin resolutions 320x180, 640x360 and 960x540 (blobbed binary
frames, cycled from a seeded pool per resolution).  Each stream owns an SP of
1024 columns x 256 synapses from a 64x64 window, learning on, duty cycles
tracked.  The load comes from the library's native load generator
(include/sp_loadgen.h: producer threads submit at the arrival times, a
collector keeps every frame's latency, submit -> result on the host): a
closed-loop run keeps every stream's queue full to find the saturation
throughput, a sweep of open-loop loads at fractions of it gives p50/p99 at
each, and the workload itself runs open loop at its own rate.

    python -m paper_1608_01966_gb300.serve_sim --seconds 60
"""
import argparse
import heapq
import json
import threading
import time

import numpy as np

from . import _binding as spg
from . import synth, workloads as wl

RESOLUTIONS = [(320, 180), (640, 360), (960, 540)]


def _frame_pools(n_per_res, seed):
    pools = {}
    for r, (W, H) in enumerate(RESOLUTIONS):
        fr = [synth.frame_blobbed(synth.derive_seed(seed, synth.PURPOSE_FRAME, 1000 * r + t), W, H)
              for t in range(n_per_res)]
        pools[(W, H)] = wl.pack(np.stack(fr))
    return pools


def open_streams(srv, n, seed, duty_period=1000.0):
    sids, res = [], []
    for i in range(n):
        W, H = RESOLUTIONS[i % 3]
        cfg = spg.sp_config_init(input_w=W, input_h=H, num_columns=1024, col_grid_w=32,
                                 col_grid_h=32, synapses_per_column=256,
                                 pool_mode=spg.SP_POOL_WINDOW, rf_w=64, rf_h=64,
                                 perm_init_lo=0.1, perm_init_hi=0.3, connect_threshold=0.2,
                                 perm_inc=0.05, perm_dec=0.02, min_overlap=4,
                                 winners_set_size=40, duty_period=duty_period,
                                 seed=synth.derive_seed(seed, synth.PURPOSE_INSTANCE, i))
        sids.append(spg.sp_server_open_stream(srv, cfg))
        res.append((W, H))
    return sids, res


class _Collector(threading.Thread):
    def __init__(self, srv, expected):
        super().__init__(daemon=True)
        self.srv, self.expected = srv, expected
        self.lat = []
        self.errors = 0
        self.t_last = None

    def run(self):
        while len(self.lat) + self.errors < self.expected:
            for r, _ in spg.sp_server_poll(self.srv, max_results=512, wait_ms=20):
                if r["status"] != 0:
                    self.errors += 1
                else:
                    self.lat.append(r["latency_us"])
                self.t_last = time.perf_counter()


def _submit(srv, sid, frame, learn=True):
    while True:
        try:
            return spg.sp_server_submit(srv, sid, frame, learn)
        except spg.SpError as e:
            if e.status != 5:  # anything but a full queue
                raise
            time.sleep(0.0002)


def run_open_loop(srv, sids, res, pools, seconds, fps, seed):
    """Poisson arrivals: every stream's inter-arrival times are exponential
    with mean 1/fps; frames are submitted at their arrival times."""
    rng = np.random.default_rng(seed)
    events = []
    for i in range(len(sids)):
        t = rng.exponential(1.0 / fps)
        while t < seconds:
            events.append((t, i))
            t += rng.exponential(1.0 / fps)
    heapq.heapify(events)
    col = _Collector(srv, len(events))
    col.start()
    spg.sp_server_get_stats(srv, reset=True)
    t0 = time.perf_counter()
    count = [0] * len(sids)
    while events:
        t, i = heapq.heappop(events)
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        pool = pools[res[i]]
        _submit(srv, sids[i], pool[count[i] % pool.shape[0]])
        count[i] += 1
    col.join(timeout=seconds + 30)
    elapsed = (col.t_last or time.perf_counter()) - t0
    lat = np.array(col.lat)
    return {"frames": int(lat.size), "errors": col.errors, "seconds": elapsed,
            "frames_per_s": lat.size / elapsed if elapsed > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) / 1000 if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) / 1000 if lat.size else None}


def run_closed_loop(srv, sids, res, pools, seconds):
    """Every stream's queue is kept full (saturation): one producer thread
    offers the next frame of every stream in one sp_server_submit_many call
    per round; streams whose queues are full refuse it and get it again in
    the next round."""
    stop = threading.Event()
    n = len(sids)
    depth = min(p.shape[0] for p in pools.values())
    # host address of frame j of stream i's pool
    ptr = np.array([[pools[res[i]][j].ctypes.data for j in range(depth)] for i in range(n)],
                   dtype=np.uint64)
    ids = np.asarray(sids, dtype=np.uint32)
    learn = np.ones(n, np.int32)
    rows = np.arange(n)

    def producer():
        seq = np.zeros(n, np.int64)
        while not stop.is_set():
            st, _ = spg.sp_server_submit_many_ptrs(srv, ids, ptr[rows, seq % depth], learn)
            ok = st == 0
            if not ((st == 0) | (st == 5)).all():  # anything but a full queue
                raise spg.SpError(int(st[~ok & (st != 5)][0]), "sp_server_submit_many", "")
            seq += ok
            if not ok.any():
                time.sleep(0)

    return _saturate(srv, producer, stop, seconds)


def _saturate(srv, producer, stop, seconds):
    """Run `producer` in a thread for `seconds` while results are drained
    (no per-result Python objects); latency percentiles from the server."""
    th = threading.Thread(target=producer, daemon=True)
    spg.sp_server_get_stats(srv, reset=True)
    taken = bad = 0
    t0 = time.perf_counter()
    th.start()
    while time.perf_counter() - t0 < seconds:
        n, b = spg.sp_server_drain(srv, wait_ms=10)
        taken += n
        bad += b
    elapsed = time.perf_counter() - t0
    st = spg.sp_server_get_stats(srv)
    stop.set()
    th.join()
    while spg.sp_server_drain(srv, wait_ms=100)[0]:
        pass
    return {"frames": taken, "errors": bad, "seconds": elapsed, "frames_per_s": taken / elapsed,
            "p50_ms": st["p50_us"] / 1000, "p99_ms": st["p99_us"] / 1000}


def run_closed_loop_device(srv, sids, res, pools, seconds):
    """Saturation with frames already on the device (as an on-GPU decoder and
    the frame encoder would leave them): one producer offers every stream's
    next frame per sp_server_submit_many_device call."""
    import torch
    stop = threading.Event()
    n = len(sids)
    depth = min(p.shape[0] for p in pools.values())
    d_pools = {k: torch.from_numpy(v[:depth].view(np.int32)).cuda() for k, v in pools.items()}
    ptr = np.array([[d_pools[res[i]][j].data_ptr() for j in range(depth)] for i in range(n)],
                   dtype=np.uint64)
    ids = np.asarray(sids, dtype=np.uint32)
    learn = np.ones(n, np.int32)
    rows = np.arange(n)
    torch.cuda.synchronize()

    def producer():
        seq = np.zeros(n, np.int64)
        while not stop.is_set():
            st, _ = spg.sp_server_submit_many_device(srv, ids, ptr[rows, seq % depth], learn)
            ok = st == 0
            if not ((st == 0) | (st == 5)).all():
                raise spg.SpError(int(st[~ok & (st != 5)][0]), "sp_server_submit_many_device", "")
            seq += ok
            if not ok.any():
                time.sleep(0)

    out = _saturate(srv, producer, stop, seconds)
    out["frames_from"] = "device"
    return out


def _native(srv, sids, res, pools, rate, seconds, producers, seed):
    """One load-generator run (native producer and collector threads)."""
    r = spg.sp_loadgen_run(srv, sids, [pools[res[i]] for i in range(len(sids))], rate, seconds,
                           producers=producers, learn=True, seed=seed)
    return {"offered_per_s": r["offered_per_s"], "frames_per_s": r["frames_per_s"],
            "frames": r["completed"], "refused": r["refused"], "errors": r["errors"],
            "seconds": r["seconds"], "p50_ms": r["p50_us"] / 1000, "p90_ms": r["p90_us"] / 1000,
            "p99_ms": r["p99_us"] / 1000, "p999_ms": r["p999_us"] / 1000,
            "max_ms": r["max_us"] / 1000, "frames_per_launch": r["frames_per_launch"]}


SWEEP = (0.1, 0.25, 0.5, 0.75, 0.9, 1.0)
KNEE_P99_MS = 1.0  # latency objective of the knee


def simulate(streams=32, fps=30.0, seconds=60.0, saturate_seconds=3.0, sweep_seconds=3.0,
             seed=0x5EED0005, budget_bytes=8 << 30, producers=4):
    """The serving workload on the library's server, driven by the native
    load generator (include/sp_loadgen.h): the closed-loop saturation
    throughput; a sweep of open-loop Poisson loads at fractions of it
    (p50/p99 latency at each, and the knee: the highest load whose p99 stays
    within KNEE_P99_MS while at least 99 % of the offered frames are served);
    and the workload itself, every stream at `fps`, for `seconds`."""
    pools = _frame_pools(16, seed)
    words = max(p.shape[1] for p in pools.values())
    srv = spg.sp_server_create(max_streams=streams, queue_depth=4, max_input_words=words,
                               device_budget_bytes=budget_bytes, max_active=64)
    try:
        sids, res = open_streams(srv, streams, seed)
        out = {"streams": streams, "fps_per_stream": fps,
               "resolutions": "round-robin 320x180 / 640x360 / 960x540",
               "producer": f"native load generator, {producers} producer threads + collector"}
        sat = None
        if saturate_seconds > 0:
            sat = _native(srv, sids, res, pools, 0.0, saturate_seconds, producers, seed + 1)
            out["closed_loop"] = sat
        if sat and sweep_seconds > 0:
            pts = []
            for k, frac in enumerate(SWEEP):
                rate = frac * sat["frames_per_s"] / streams
                pt = _native(srv, sids, res, pools, rate, sweep_seconds, producers, seed + 2 + k)
                pt["fraction_of_saturation"] = frac
                pts.append(pt)
            out["sweep"] = pts
            knee = None
            for pt in pts:
                served = pt["frames"] / max(1.0, pt["offered_per_s"] * sweep_seconds)
                if pt["p99_ms"] <= KNEE_P99_MS and served >= 0.99:
                    knee = pt
            out["knee"] = None if knee is None else {
                "fraction_of_saturation": knee["fraction_of_saturation"],
                "frames_per_s": knee["frames_per_s"], "p99_ms": knee["p99_ms"],
                "rule": f"highest load with p99 <= {KNEE_P99_MS} ms and >= 99 % of the offered "
                        "frames served (the rest arrive at a full stream queue)"}
        if seconds > 0:
            out["open_loop"] = _native(srv, sids, res, pools, fps, seconds, producers, seed)
        st = spg.sp_server_get_stats(srv)
        out["launches"] = st["launches"]
        out["frames_per_launch"] = st["frames_in_launches"] / max(1, st["launches"])
        for sid in sids:
            spg.sp_server_close_stream(srv, sid)
    finally:
        spg.sp_server_destroy(srv)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=32)
    ap.add_argument("--fps", type=float, default=30.0)
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--saturate-seconds", type=float, default=3.0)
    ap.add_argument("--sweep-seconds", type=float, default=3.0)
    a = ap.parse_args()
    print(json.dumps(simulate(a.streams, a.fps, a.seconds, a.saturate_seconds, a.sweep_seconds)))


if __name__ == "__main__":
    main()
