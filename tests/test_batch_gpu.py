"""Batches of independent SPs (one launch per batch frame) against the CPU
oracle run on each member alone, and against the members run alone on the
GPU.  Bar: bit-exact, as for single SPs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402
from helpers import dense, first_diff, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu

SWEEP_FRAMES = 200  # learning frames per combination of the sweep workload


def _member_frames(cases, dens, n):
    return [wl.bernoulli_frames(i, c.n_in, dens[i], n) for i, c in enumerate(cases)]


def _run_batch(cases, frames_u8, learn, calls, boosts=None, schedule=None):
    """Create handles + batch (schedule: (ctas_per_sm, cols_in_flight,
    member columns per warp) to pin, or None), run the batch frames split
    into `calls` (list of frame counts) through
    sp_batch_compute_overlaps_device, return per-member active [n][C], final
    perms, and overlaps of every frame [n][C]."""
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    if schedule is not None:
        spg.sp_batch_set_schedule(b, *schedule)
        assert spg.sp_batch_schedule(b, len(hs)) == (schedule[0], schedule[1],
                                                     list(schedule[2] or [0] * len(hs)))
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    oo, ow = spg.sp_batch_overlap_offsets(b)
    assert ow == sum(c.C for c in cases)
    n = frames_u8[0].shape[0]
    fw = (info["frame_words"] + 3) // 4 * 4
    bf = wl.batch_frames([wl.pack(f) for f in frames_u8], fo, fw)
    mw = info["mask_words"]
    stream = torch.cuda.current_stream()
    d = torch.from_numpy(bf.view(np.int32)).cuda()
    dm = torch.zeros((n, mw), dtype=torch.int32, device="cuda")
    dov = torch.full((n, ow), -1.0, dtype=torch.float32, device="cuda")
    t0 = 0
    for k in calls:
        spg.sp_batch_compute_overlaps_device(b, d[t0], k, fw, learn, dm[t0], mw, dov[t0], ow,
                                             stream)
        t0 += k
    assert t0 == n
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    ovr = dov.cpu().numpy()
    spg.sp_batch_destroy(b)
    acts = [dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
            for i, c in enumerate(cases)]
    perms = [spg.sp_get_permanences(h) for h in hs]
    ovs = [ovr[:, int(oo[i]):int(oo[i]) + c.C] for i, c in enumerate(cases)]
    last = [spg.sp_get_overlaps(h) for h in hs]
    for i in range(len(cases)):
        np.testing.assert_array_equal(last[i], ovs[i][-1], err_msg=f"member {i} last overlaps")
    for h in hs:
        spg.sp_destroy(h)
    return acts, perms, ovs


def _oracle_all(cases, frames_u8, learn):
    """The oracle on every member (host threads: the oracle's C code runs
    without the GIL)."""
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        return list(ex.map(lambda i: oracle_run(cases[i], frames_u8[i], learn, want_ov=True),
                           range(len(cases))))


def _check(cases, frames_u8, learn, acts, perms, ovs, label):
    """Every member, every frame: overlaps element by element, active sets,
    and the final permanences."""
    for i, (act, perm, ov) in enumerate(_oracle_all(cases, frames_u8, learn)):
        d = first_diff(ovs[i], ov)
        assert d is None, f"{label} member {i}: first differing overlap (frame, column) {d}"
        assert first_diff(acts[i], act) is None, f"{label} member {i}: frame/column {first_diff(acts[i], act)}"
        np.testing.assert_array_equal(perms[i], perm, err_msg=f"{label} member {i} perms")


def test_batch_of_identical_shapes():
    cases = [wl.small_case(seed=wl.BASE_SEED + 100 + i) for i in range(8)]
    frames = [wl.small_frames(24, seed=wl.BASE_SEED + 100 + i) for i in range(8)]
    acts, perms, ovs = _run_batch(cases, frames, True, [1, 2, 5, 16])
    _check(cases, frames, True, acts, perms, ovs, "identical")


def test_batch_uneven_shapes_and_modes():
    """Uneven columns / synapses / input sizes, plus members with local
    inhibition, non-unit boosts and S not a multiple of 4."""
    cases, dens = wl.uneven_cases(10, c_range=(128, 2048), n_in_range=(256, 4096))
    g = wl.grid_case("local", 256, 64, 7, W=320, H=180, rf=32, k=5, inhibition=1, radius=4)
    cases.append(g)
    dens.append(None)
    rag = wl.Case("ragged", 1000, 1, 300, 17, synth.pool_uniform(3, 300, 17, 1000),
                  synth.perm_uniform(4, (300, 17), 0.1, 0.3), synth.perm_uniform(5, (300,), 0.5, 2.0),
                  k=9, min_overlap=2)
    cases.append(rag)
    dens.append(0.3)
    frames = []
    for i, c in enumerate(cases):
        if c.name == "local":
            frames.append(wl.blob_frames(12, W=320, H=180, seed=11))
        else:
            frames.append(wl.bernoulli_frames(i, c.n_in, dens[i], 12))
    acts, perms, ovs = _run_batch(cases, frames, True, [3, 9])
    _check(cases, frames, True, acts, perms, ovs, "uneven")


def _schedules():
    try:
        return spg.sp_batch_schedule_list()
    except Exception:  # library not built: the test fails when it runs instead
        return [(10, 4)]


@pytest.mark.parametrize("sched", _schedules())
@pytest.mark.parametrize("split", ["default", "mixed"])
def test_batch_every_compiled_schedule(sched, split):
    """Every compiled schedule of the persistent pass (resident CTAs per SM x
    columns per warp in flight), with each member's default split and with
    per-member splits of 2 to 16 columns per warp: window-form, compact-form
    and full-form members learning over runs of several frames, against the
    oracle frame by frame."""
    cases = [wl.frame_case(seed=wl.BASE_SEED + 700 + i) for i in range(2)]
    unv, dens = wl.uneven_cases(4, c_range=(128, 1500), n_in_range=(256, 4096))
    cases += unv
    rag = wl.Case("ragged", 1000, 1, 300, 17, synth.pool_uniform(3, 300, 17, 1000),
                  synth.perm_uniform(4, (300, 17), 0.1, 0.3), synth.perm_uniform(5, (300,), 0.5, 2.0),
                  k=9, min_overlap=2)
    cases.append(rag)
    frames = [wl.blob_frames(10, seed=wl.BASE_SEED + 700 + i) for i in range(2)]
    frames += [wl.bernoulli_frames(i, c.n_in, dens[i], 10) for i, c in enumerate(unv)]
    frames.append(wl.bernoulli_frames(9, rag.n_in, 0.3, 10))
    per = None if split == "default" else [(2, 4, 8, 16)[i % 4] for i in range(len(cases))]
    acts, perms, ovs = _run_batch(cases, frames, True, [1, 4, 5],
                                  schedule=(sched[0], sched[1], per))
    _check(cases, frames, True, acts, perms, ovs, f"schedule {sched} {split}")


@pytest.mark.parametrize("cpw", ["1", "4", "8"])
def test_batch_staged_state(monkeypatch, cpw):
    """The opt-in form that brings each CTA's pools and permanences into
    shared memory by bulk copy, over uneven members (those with S not a
    multiple of 4 or whose block exceeds the cap take the streamed form)."""
    monkeypatch.setenv("SP_BATCH_STAGE_KB", "64")
    monkeypatch.setenv("SP_BATCH_COLS_PER_WARP", cpw)
    cases, dens = wl.uneven_cases(8, c_range=(64, 1500), n_in_range=(256, 4096))
    cases.append(wl.frame_case(seed=wl.BASE_SEED + 300))
    dens.append(None)
    frames = [wl.blob_frames(8, seed=wl.BASE_SEED + 300) if d is None
              else wl.bernoulli_frames(i, c.n_in, d, 8) for i, (c, d) in enumerate(zip(cases, dens))]
    acts, perms, ovs = _run_batch(cases, frames, True, [1, 7])
    _check(cases, frames, True, acts, perms, ovs, f"staged cpw={cpw}")


@pytest.mark.parametrize("window_kb", ["24", "0"])
@pytest.mark.parametrize("xspan_kb", ["0", "16"])
@pytest.mark.parametrize("compact", ["1", "0"])
def test_batch_compact_form(monkeypatch, compact, xspan_kb, window_kb):
    """Members whose pools fit 64 x 64 boxes of a frame 32k pixels wide run on
    the window form (box origin + bitmap of connected synapses, frame rows
    staged in shared memory) unless it is off; members whose synapse count is
    a multiple of 32 (<= 256) and whose pools span at most 65536 inputs run on
    16-bit offsets and connected bits; the others (a pool spread over a 960x540
    frame, S = 48) on the full form.  Every form must
    equal the oracle, learning included, with the CTAs' input words read from
    global memory or first copied to shared memory."""
    monkeypatch.setenv("SP_BATCH_COMPACT", compact)
    monkeypatch.setenv("SP_BATCH_XSPAN_KB", xspan_kb)
    monkeypatch.setenv("SP_BATCH_WINDOW_KB", window_kb)
    cases, frames = [], []
    for i, S in enumerate((32, 64, 128, 256)):
        c = wl.grid_case(f"win{S}", 256, S, wl.BASE_SEED + 400 + i, W=320, H=180, rf=32, k=6,
                         inhibition=1 if S == 64 else 0, radius=3)
        if S == 128:
            c.boost = synth.perm_uniform(wl.BASE_SEED + 7, (256,), 0.5, 2.0)
        cases.append(c)
        frames.append(wl.blob_frames(10, W=320, H=180, seed=wl.BASE_SEED + 400 + i))
    n_in = 960 * 540
    wide = wl.Case("wide", 960, 540, 128, 64,
                   synth.pool_uniform(wl.BASE_SEED + 410, 128, 64, n_in),
                   synth.perm_uniform(wl.BASE_SEED + 411, (128, 64), 0.1, 0.3),
                   np.ones(128, np.float32), k=5, min_overlap=1)
    cases.append(wide)
    frames.append(wl.blob_frames(10, seed=wl.BASE_SEED + 412))
    odd = wl.grid_case("s48", 256, 48, wl.BASE_SEED + 413, W=320, H=180, rf=32, k=6)
    cases.append(odd)
    frames.append(wl.blob_frames(10, W=320, H=180, seed=wl.BASE_SEED + 414))
    acts, perms, ovs = _run_batch(cases, frames, True, [3, 7])
    _check(cases, frames, True, acts, perms, ovs, f"compact={compact} xspan={xspan_kb}")


def test_batch_equals_members_alone_and_hands_back_state():
    """A batch, then each member continued alone: the same as the oracle over
    the whole sequence (pending learning handed back by the batch)."""
    cases = [wl.frame_case(seed=wl.BASE_SEED + 200 + i) for i in range(3)]
    frames = [wl.blob_frames(10, seed=wl.BASE_SEED + 200 + i) for i in range(3)]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    with pytest.raises(spg.SpError) as e:
        spg.sp_compute(hs[0], wl.pack(frames[0][:1])[0], True)
    assert e.value.status == 5  # SP_EBUSY while batched
    fo, mo = spg.sp_batch_offsets(b)
    info = spg.sp_batch_get_info(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    bf = wl.batch_frames([wl.pack(f[:6]) for f in frames], fo, fw)
    d = torch.from_numpy(bf.view(np.int32)).cuda()
    spg.sp_batch_compute_device(b, d, 6, fw, True, None, 0, torch.cuda.current_stream())
    spg.sp_batch_destroy(b)
    for i, (c, h) in enumerate(zip(cases, hs)):
        act, perm, _ = oracle_run(c, frames[i], True)
        for t in range(6, 10):
            spg.sp_compute(h, wl.pack(frames[i][t:t + 1])[0], True)
            np.testing.assert_array_equal(spg.sp_active_columns(h), np.flatnonzero(act[t]))
        np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
        spg.sp_destroy(h)


def test_batch_host_pipelined():
    """sp_batch_compute: pinned host batch frames in, mask records out."""
    cases, dens = wl.uneven_cases(6, c_range=(256, 1024), n_in_range=(1024, 8192))
    frames = _member_frames(cases, dens, 9)
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    bf = wl.batch_frames([wl.pack(f) for f in frames], fo, info["frame_words"])
    pinned = torch.from_numpy(bf.view(np.int32)).pin_memory()
    masks = np.zeros((9, info["mask_words"]), np.uint32)
    spg.sp_batch_compute(b, pinned.numpy().view(np.uint32), True, masks)
    spg.sp_batch_destroy(b)
    for i, c in enumerate(cases):
        act, perm, _ = oracle_run(c, frames[i], True)
        got = dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
        assert first_diff(got, act) is None, f"member {i}"
        np.testing.assert_array_equal(spg.sp_get_permanences(hs[i]), perm)
        spg.sp_destroy(hs[i])


def test_batch_rejects_bad_members():
    c = wl.small_case()
    h = spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost)
    with pytest.raises(spg.SpError):
        spg.sp_batch_create([h, h])
    b = spg.sp_batch_create([h])
    with pytest.raises(spg.SpError) as e:
        spg.sp_batch_create([h])
    assert e.value.status == 5
    spg.sp_batch_destroy(b)
    spg.sp_destroy(h)


def test_batch_autotune_keeps_state():
    """Autotuning times learning frames on every candidate (schedules and
    splits) and keeps the fastest; it puts back what the learning wrote, so
    permanences, window and compact forms, learning and duty cycles continue
    exactly as if it had not run (oracle over the real frames only).
    Window-form, compact-form and full-form members."""
    import oracle
    from helpers import oracle_params
    cases = [wl.frame_case(seed=wl.BASE_SEED + 500 + i) for i in range(2)]
    unv, dens = wl.uneven_cases(3, c_range=(200, 900), n_in_range=(512, 4096))
    cases += unv
    rag = wl.Case("ragged", 1000, 1, 300, 17, synth.pool_uniform(3, 300, 17, 1000),
                  synth.perm_uniform(4, (300, 17), 0.1, 0.3), np.ones(300, np.float32),
                  k=9, min_overlap=2)
    cases.append(rag)
    period = 25.0
    real = [wl.blob_frames(6, seed=wl.BASE_SEED + 500 + i) for i in range(2)]
    real += [wl.bernoulli_frames(i, c.n_in, dens[i], 6) for i, c in enumerate(unv)]
    real.append(wl.bernoulli_frames(7, rag.n_in, 0.3, 6))
    tune = [wl.blob_frames(3, seed=wl.BASE_SEED + 520 + i) for i in range(2)]
    tune += [wl.bernoulli_frames(i, c.n_in, dens[i], 3, start=100) for i, c in enumerate(unv)]
    tune.append(wl.bernoulli_frames(8, rag.n_in, 0.3, 3))
    hs = [spg.sp_create_from_state(c.config(duty_period=period), c.idx, c.perm, c.boost)
          for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    d_tune = torch.from_numpy(wl.batch_frames([wl.pack(f) for f in tune], fo, fw).view(np.int32)).cuda()
    cpw = spg.sp_batch_autotune(b, d_tune, 3, fw)
    assert cpw in (0, 2, 4, 8, 16, spg.SP_MIXED_SPLIT)
    ctas, cols, per = spg.sp_batch_schedule(b, len(hs))
    assert (ctas, cols) in spg.sp_batch_schedule_list()
    assert all(c in (0, 2, 4, 8, 16) for c in per)
    assert cpw == spg.SP_MIXED_SPLIT or per == [cpw] * len(hs)
    d_real = torch.from_numpy(wl.batch_frames([wl.pack(f) for f in real], fo, fw).view(np.int32)).cuda()
    mw = info["mask_words"]
    dm = torch.zeros((6, mw), dtype=torch.int32, device="cuda")
    spg.sp_batch_compute_device(b, d_real, 6, fw, True, dm, mw, torch.cuda.current_stream())
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    spg.sp_batch_destroy(b)
    for i, (c, h) in enumerate(zip(cases, hs)):
        perm = c.perm.copy()
        duty = np.zeros(c.C, np.float32)
        acts = []
        for t in range(6):
            a = oracle.run(oracle_params(c), c.idx, perm, c.boost, real[i][t:t + 1], True)[0]
            oracle.duty_update(duty, a, period)
            acts.append(a)
        got = dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
        assert first_diff(got, np.stack(acts)) is None, f"member {i}"
        np.testing.assert_array_equal(spg.sp_get_permanences(h), perm, err_msg=f"member {i}")
        np.testing.assert_array_equal(spg.sp_get_duty_cycles(h), duty, err_msg=f"member {i}")
        spg.sp_destroy(h)


@pytest.mark.parametrize("persistent", ["1", "0"])
def test_batch_long_sequence_in_one_call(monkeypatch, persistent):
    """40 learning frames of uneven members (compact and full forms, local
    inhibition, duty cycles) in one call: one persistent launch in which each
    member's frame t + 1 waits only for that member's frame t, or one launch
    per frame."""
    monkeypatch.setenv("SP_DISABLE_PERSISTENT", "0" if persistent == "1" else "1")
    cases, dens = wl.uneven_cases(5, c_range=(64, 1200), n_in_range=(256, 4096))
    g = wl.grid_case("local", 256, 64, 7, W=320, H=180, rf=32, k=5, inhibition=1, radius=4)
    cases.append(g)
    dens.append(None)
    frames = [wl.blob_frames(40, W=320, H=180, seed=11) if d is None
              else wl.bernoulli_frames(i, c.n_in, d, 40) for i, (c, d) in enumerate(zip(cases, dens))]
    acts, perms, ovs = _run_batch(cases, frames, True, [40])
    _check(cases, frames, True, acts, perms, ovs, f"persistent={persistent}")


@pytest.mark.parametrize("window_kb", ["24", "0"])
@pytest.mark.parametrize("C", [256, 1024, 4096])
def test_batch_parameter_sweep(C, window_kb, monkeypatch):
    """The sweep workload at its stated length: the 54 synapse x min_overlap x
    k x {global, 9x9 local} combinations for one column count, as members of
    one batch (window form, else compact form for S = 64 and 256 and full form
    for S = 16), 200
    learning frames of 960x540 blobbed input in one persistent launch; every
    member's overlaps and winners of every frame, and its final permanences,
    against the oracle.  Window-shaped pools run on the window form, or with it
    off on the compact form."""
    monkeypatch.setenv("SP_BATCH_WINDOW_KB", window_kb)
    frames1 = wl.blob_frames(SWEEP_FRAMES, seed=wl.BASE_SEED + 3)
    cases, frames = [], []
    for S in (16, 64, 256):
        for m in (2, 4, 8):
            for k in (8, 32, 128):
                for inh in (0, 1):
                    cases.append(wl.grid_case("sweep", C, S, wl.BASE_SEED + 3 + C + S,
                                              min_overlap=m, k=k, inhibition=inh, radius=4))
                    frames.append(frames1)
    acts, perms, ovs = _run_batch(cases, frames, True, [SWEEP_FRAMES])
    _check(cases, frames, True, acts, perms, ovs, f"sweep C{C}")
