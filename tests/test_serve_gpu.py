"""The serving loop: streams submitted concurrently from several threads and
batched by the library's worker must give, frame for frame, the results of
each stream computed alone (and of the CPU oracle) -- bit-exact -- and
streams are admitted against the device-memory budget."""
import random
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import workloads as wl  # noqa: E402
from helpers import oracle_params  # noqa: E402

pytestmark = pytest.mark.gpu

RES = [(320, 180), (640, 360), (960, 540)]


def _streams(n, frames_per_stream, duty=0.0):
    cases, frames = [], []
    for i in range(n):
        W, H = RES[i % 3]
        c = wl.grid_case(f"s{i}", 1024, 256, wl.BASE_SEED + 500 + i, W=W, H=H, k=40)
        cases.append(c)
        frames.append(wl.blob_frames(frames_per_stream, W=W, H=H, seed=wl.BASE_SEED + 500 + i))
    return cases, frames


def _oracle_lists(case, frames, learn, duty_period=0.0):
    perm = case.perm.copy()
    p = oracle_params(case)
    out, duty = [], np.zeros(case.C, np.float32)
    for t in range(frames.shape[0]):
        a = oracle.run(p, case.idx, perm, case.boost, frames[t:t + 1], learn[t])[0]
        if duty_period:
            oracle.duty_update(duty, a, duty_period)
        out.append(np.flatnonzero(a))
    return out, perm, duty


def test_results_same_alone_and_in_the_mix():
    n, F = 6, 10
    cases, frames = _streams(n, F)
    learn = [[(t % 4) != 3 for t in range(F)] for _ in range(n)]
    words = max(wl.pack(f).shape[1] for f in frames)
    srv = spg.sp_server_create(max_streams=8, queue_depth=4, max_input_words=words,
                               device_budget_bytes=1 << 30, max_active=64)
    sids = [spg.sp_server_open_stream(srv, c.config(), state=(c.idx, c.perm, c.boost))
            for c in cases]
    packed = [wl.pack(f) for f in frames]
    got = {i: {} for i in range(n)}
    seqs = {i: [] for i in range(n)}
    errors = []

    def client(members):
        rng = random.Random(members[0])
        try:
            for t in range(F):
                for i in members:
                    while True:
                        try:
                            spg.sp_server_submit(srv, sids[i], packed[i][t], learn[i][t])
                            break
                        except spg.SpError as e:  # queue full: retry
                            if e.status != 5:
                                raise
                            time.sleep(0.0005)
                    time.sleep(rng.random() * 0.002)
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    threads = [threading.Thread(target=client, args=(m,)) for m in ([0, 3], [1, 4], [2, 5])]
    for th in threads:
        th.start()
    done, deadline = 0, time.time() + 60
    while done < n * F and time.time() < deadline:
        for r, act in spg.sp_server_poll(srv, wait_ms=50):
            assert r["status"] == 0
            i = sids.index(r["stream_id"])
            got[i][r["frame_seq"]] = act
            seqs[i].append(r["frame_seq"])
            done += 1
    for th in threads:
        th.join()
    assert not errors, errors
    assert done == n * F
    st = spg.sp_server_get_stats(srv)
    assert st["completed"] == n * F and st["launches"] >= 1
    for i, c in enumerate(cases):
        assert seqs[i] == sorted(seqs[i])  # per-stream order
        ref, perm, _ = _oracle_lists(c, frames[i], learn[i])
        for t in range(F):
            np.testing.assert_array_equal(got[i][t], ref[t], err_msg=f"stream {i} frame {t}")
        np.testing.assert_array_equal(
            spg.sp_server_get_permanences(srv, sids[i], (c.C, c.S)), perm)
        # alone: the same stream through sp_compute
        h = spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost)
        for t in range(F):
            spg.sp_compute(h, packed[i][t], learn[i][t])
            np.testing.assert_array_equal(spg.sp_active_columns(h), got[i][t])
        spg.sp_destroy(h)
    for sid in sids:
        spg.sp_server_close_stream(srv, sid)
    spg.sp_server_destroy(srv)


def test_admission_by_device_memory_budget():
    cases = [wl.grid_case(f"a{i}", 1024, 256, wl.BASE_SEED + 550 + i) for i in range(3)]
    probe = spg.sp_server_create(max_streams=2, queue_depth=2, max_input_words=16200,
                                 device_budget_bytes=1 << 34, max_active=64)
    spg.sp_server_open_stream(probe, cases[0].config(), state=(cases[0].idx, cases[0].perm, None))
    per_stream = spg.sp_server_get_stats(probe)["device_bytes_used"]
    spg.sp_server_destroy(probe)
    srv = spg.sp_server_create(max_streams=8, queue_depth=2, max_input_words=16200,
                               device_budget_bytes=int(2.5 * per_stream), max_active=64)
    a = spg.sp_server_open_stream(srv, cases[0].config(), state=(cases[0].idx, cases[0].perm, None))
    b = spg.sp_server_open_stream(srv, cases[1].config(), state=(cases[1].idx, cases[1].perm, None))
    with pytest.raises(spg.SpError) as e:
        spg.sp_server_open_stream(srv, cases[2].config(),
                                  state=(cases[2].idx, cases[2].perm, None))
    assert e.value.status == 5  # SP_EBUSY: the third stream does not fit the budget
    assert spg.sp_server_get_stats(srv)["device_bytes_used"] == 2 * per_stream
    spg.sp_server_close_stream(srv, a)
    assert spg.sp_server_get_stats(srv)["device_bytes_used"] == per_stream
    c = spg.sp_server_open_stream(srv, cases[2].config(), state=(cases[2].idx, cases[2].perm, None))
    assert spg.sp_server_get_stats(srv)["open_streams"] == 2
    spg.sp_server_close_stream(srv, b)
    spg.sp_server_close_stream(srv, c)
    spg.sp_server_destroy(srv)


def test_duty_cycles_match_the_oracle():
    """Duty cycles tracked on the device (single frames, sequences in the
    cluster kernel, batches) follow d <- d + (a - d) / P of the oracle."""
    case = wl.frame_case(seed=wl.BASE_SEED + 600)
    frames = wl.blob_frames(30, seed=wl.BASE_SEED + 600)
    learn = [True] * 30
    ref, perm, duty = _oracle_lists(case, frames, learn, duty_period=20.0)
    cfg = case.config(duty_period=20.0)
    packed = wl.pack(frames)
    h = spg.sp_create_from_state(cfg, case.idx, case.perm, case.boost)
    for t in range(3):  # single frames
        spg.sp_compute(h, packed[t], True)
    d = torch.from_numpy(packed[3:].view(np.int32)).cuda()
    spg.sp_compute_frames_device(h, d, 27, packed.shape[1], True, None,
                                 torch.cuda.current_stream())  # one cluster launch
    np.testing.assert_array_equal(spg.sp_active_columns(h), ref[-1])
    np.testing.assert_array_equal(spg.sp_get_duty_cycles(h), duty)
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


@pytest.mark.parametrize("device", [False, True])
def test_submit_many_matches_the_oracle(device):
    """Frames offered for every stream at once (sp_server_submit_many, or
    sp_server_submit_many_device with the frames already on the GPU), full
    queues refusing and the frame offered again next round: every stream's
    results and permanences equal the oracle's, in order."""
    n, F = 5, 12
    cases, frames = _streams(n, F)
    learn = [[(t + i) % 5 != 4 for t in range(F)] for i in range(n)]
    words = max(wl.pack(f).shape[1] for f in frames)
    srv = spg.sp_server_create(max_streams=8, queue_depth=2, max_input_words=words,
                               device_budget_bytes=1 << 30, max_active=64)
    sids = [spg.sp_server_open_stream(srv, c.config(), state=(c.idx, c.perm, c.boost))
            for c in cases]
    packed = [wl.pack(f) for f in frames]
    d_packed = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    torch.cuda.synchronize()
    nxt = [0] * n
    got = {i: {} for i in range(n)}
    seqs = {i: [] for i in range(n)}
    done, deadline = 0, time.time() + 60
    while done < n * F and time.time() < deadline:
        todo = [i for i in range(n) if nxt[i] < F]
        if todo and device:
            st, rid = spg.sp_server_submit_many_device(
                srv, [sids[i] for i in todo], [d_packed[i][nxt[i]].data_ptr() for i in todo],
                [learn[i][nxt[i]] for i in todo], torch.cuda.current_stream())
        elif todo:
            st, rid = spg.sp_server_submit_many(srv, [sids[i] for i in todo],
                                                [packed[i][nxt[i]] for i in todo],
                                                [learn[i][nxt[i]] for i in todo])
        if todo:
            for j, i in enumerate(todo):
                assert st[j] in (0, 5)
                if st[j] == 0:
                    assert rid[j] > 0
                    nxt[i] += 1
        for r, act in spg.sp_server_poll(srv, wait_ms=1):
            assert r["status"] == 0
            i = sids.index(r["stream_id"])
            got[i][r["frame_seq"]] = act
            seqs[i].append(r["frame_seq"])
            done += 1
    assert done == n * F
    for i in range(n):
        assert seqs[i] == list(range(F)), f"stream {i} results out of order"
    # an unknown stream is refused per entry, not for the call
    st, _ = spg.sp_server_submit_many(srv, [999], [packed[0][0]], True)
    assert st[0] == 1
    for i, c in enumerate(cases):
        ref, perm, _ = _oracle_lists(c, frames[i], learn[i])
        for t in range(F):
            np.testing.assert_array_equal(got[i][t], ref[t], err_msg=f"stream {i} frame {t}")
        np.testing.assert_array_equal(
            spg.sp_server_get_permanences(srv, sids[i], (c.C, c.S)), perm)
    for sid in sids:
        spg.sp_server_close_stream(srv, sid)
    spg.sp_server_destroy(srv)


def test_native_load_generator_open_and_closed_loop():
    """The native load generator (include/sp_loadgen.h) on 6 streams: a
    closed-loop second keeps every queue full, an open-loop second offers
    Poisson arrivals at 200 fps per stream; every accepted frame comes back
    without error, arrivals are either accepted or refused, and latencies are
    positive and ordered."""
    cases, frames = _streams(6, 8)
    packed = [wl.pack(f) for f in frames]
    words = max(p.shape[1] for p in packed)
    srv = spg.sp_server_create(max_streams=8, queue_depth=4, max_input_words=words,
                               device_budget_bytes=1 << 30, max_active=64)
    sids = [spg.sp_server_open_stream(srv, c.config(), state=(c.idx, c.perm, c.boost))
            for c in cases]
    closed = spg.sp_loadgen_run(srv, sids, packed, 0.0, 1.0, producers=2, seed=1)
    assert closed["errors"] == 0 and closed["completed"] == closed["submitted"] > 0
    assert closed["frames_per_s"] > 1000
    opened = spg.sp_loadgen_run(srv, sids, packed, 200.0, 1.0, producers=3, seed=2)
    assert opened["errors"] == 0 and opened["completed"] == opened["submitted"]
    assert opened["offered"] == opened["submitted"] + opened["refused"]
    assert 0.5 * 1200 < opened["offered"] < 1.5 * 1200  # 6 streams x 200 fps x 1 s
    assert 0 < opened["p50_us"] <= opened["p99_us"] <= opened["max_us"]
    st = spg.sp_server_get_stats(srv)
    assert st["completed"] >= closed["completed"] + opened["completed"]
    for sid in sids:
        spg.sp_server_close_stream(srv, sid)
    spg.sp_server_destroy(srv)
