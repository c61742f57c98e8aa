"""Dense potential pools (every column sees the whole input) computed without
learning on the tensor cores (tcgen05 kind::f8f6f4, e4m3 {0,1} operands, fp32
accumulation: exact), against the CPU oracle and against the per-frame
kernel.  Bar: bit-exact, on every frame's overlaps and winners."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402
from helpers import dense, first_diff, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu


def _dense_case(C, n_in, seed, k=20, m=4, boost=None, lo=0.1, hi=0.3, **kw):
    idx = synth.pool_dense(C, n_in)
    perm = synth.perm_uniform(synth.derive_seed(seed, 2, 0), (C, n_in), lo, hi)
    b = np.ones(C, np.float32) if boost is None else boost
    return wl.Case("dense", n_in, 1, C, n_in, idx, perm, b, k=k, min_overlap=m, **kw)


def _frames(F, n_in, p, seed):
    return np.stack([synth.frame_bernoulli(synth.derive_seed(seed, 3, t), n_in, p)
                     for t in range(F)])


def _run(case, frames, cfg_extra=None):
    packed = wl.pack(frames)
    F = packed.shape[0]
    cfg = case.config(**(cfg_extra or {}))
    h = spg.sp_create_from_state(cfg, case.idx, case.perm, case.boost)
    d = torch.from_numpy(packed.view(np.int32)).cuda()
    dm = torch.zeros((F, (case.C + 31) // 32), dtype=torch.int32, device="cuda")
    dov = torch.full((F, case.C), -1.0, dtype=torch.float32, device="cuda")
    before = spg.sp_kernel_launch_count()
    spg.sp_compute_frames_overlaps_device(h, d, F, packed.shape[1], False, dm, dov,
                                          torch.cuda.current_stream())
    spg.sp_sync(h)
    launches = spg.sp_kernel_launch_count() - before
    out = dense(dm.cpu().numpy().view(np.uint32), case.C)
    ovs = dov.cpu().numpy()
    ov = spg.sp_get_overlaps(h)
    lst = spg.sp_active_columns(h)
    duty = spg.sp_get_duty_cycles(h) if (cfg_extra or {}).get("duty_period") else None
    spg.sp_destroy(h)
    return out, ov, lst, launches, duty, ovs


def test_dense_pools_on_tensor_cores_match_oracle():
    """1024 inputs x 1024 columns over 256 frames: two 128-frame tiles x four
    256-column tiles, sixteen 64-input slices."""
    case = _dense_case(1024, 1024, 41, k=40)
    frames = _frames(256, 1024, 0.2, 42)
    act, _, ov = oracle_run(case, frames, False, want_ov=True)
    got, gov, lst, launches, _, ovs = _run(case, frames)
    assert launches <= 4  # pack, GEMM, per-frame inhibition: not 256 launches
    assert first_diff(ovs, ov) is None  # every overlap of every frame
    assert first_diff(got, act) is None
    np.testing.assert_array_equal(gov, ov[-1])
    np.testing.assert_array_equal(lst, np.flatnonzero(act[-1]))


def test_dense_ragged_tiles_and_boosts():
    """Columns, inputs and frames that fill no tile exactly; non-unit boosts
    (radix select); input bits beyond n_in in the last word are ignored."""
    boost = synth.perm_uniform(7, (300,), 0.5, 2.0)
    case = _dense_case(300, 1000, 43, k=9, m=1, boost=boost, lo=0.15, hi=0.25)
    frames = _frames(130, 1000, 0.4, 44)
    act, _, ov = oracle_run(case, frames, False, want_ov=True)
    packed = wl.pack(frames)
    packed[:, -1] |= np.uint32(0xFF000000)  # garbage in the unused high bits
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    d = torch.from_numpy(packed.view(np.int32)).cuda()
    dm = torch.zeros((130, 10), dtype=torch.int32, device="cuda")
    spg.sp_compute_frames_device(h, d, 130, packed.shape[1], False, dm, torch.cuda.current_stream())
    spg.sp_sync(h)
    assert first_diff(dense(dm.cpu().numpy().view(np.uint32), 300), act) is None
    np.testing.assert_array_equal(spg.sp_get_overlaps(h), ov[-1])
    spg.sp_destroy(h)


def test_dense_local_inhibition_and_duty(monkeypatch):
    case = _dense_case(256, 512, 45, k=3, m=2, inhibition=1, gw=16, gh=16, radius=2)
    frames = _frames(40, 512, 0.3, 46)
    act, _, _ = oracle_run(case, frames, False)
    got, _, _, _, duty, _ = _run(case, frames, {"duty_period": 10.0})
    assert first_diff(got, act) is None
    import oracle
    d = np.zeros(256, np.float32)
    for t in range(40):
        oracle.duty_update(d, act[t], 10.0)
    np.testing.assert_array_equal(duty, d)
    # the per-frame kernel gives the same
    monkeypatch.setenv("SP_DISABLE_TENSOR_CORES", "1")
    got2, _, _, launches, _, _ = _run(case, frames)
    assert launches >= 40 or launches == 1  # per-frame kernels (or one recorded graph)
    np.testing.assert_array_equal(got2, got)


def test_dense_run_after_learning_uses_learned_state():
    """Learning frames (per-frame kernel) then an inference run on the tensor
    cores: the run sees the learned permanences."""
    case = _dense_case(512, 512, 47, k=10, m=2)
    frames = _frames(40, 512, 0.3, 48)
    act_l, perm, _ = oracle_run(case, frames[:8], True)
    act_i, _, _ = oracle_run(case, frames[8:], False, perm=perm)
    packed = wl.pack(frames)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    for t in range(8):
        spg.sp_compute(h, packed[t], True)
    d = torch.from_numpy(packed[8:].view(np.int32)).cuda()
    dm = torch.zeros((32, 16), dtype=torch.int32, device="cuda")
    spg.sp_compute_frames_device(h, d, 32, packed.shape[1], False, dm, torch.cuda.current_stream())
    spg.sp_sync(h)
    assert first_diff(dense(dm.cpu().numpy().view(np.uint32), 512), act_i) is None
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


def test_batch_of_dense_sps_infers_in_two_launches():
    """Dense SPs of different shapes in one batch: all overlaps in one
    tensor-core launch, Alg. 2 for every frame and SP in one more (plus the
    operand images: the frames' every run, the connections' only when the
    permanences changed)."""
    shapes = [(1024, 1024), (300, 500), (700, 2048), (257, 999), (1024, 1024)]
    cases = [_dense_case(C, n, 50 + i, k=max(1, (2 * C + 50) // 100))
             for i, (C, n) in enumerate(shapes)]
    F = 130
    frames = [_frames(F, c.n_in, 0.02 + 0.05 * i, 60 + i) for i, c in enumerate(cases)]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    bf = wl.batch_frames([wl.pack(f) for f in frames], fo, fw)
    d = torch.from_numpy(bf.view(np.int32)).cuda()
    mw = info["mask_words"]
    oo, ow = spg.sp_batch_overlap_offsets(b)
    dm = torch.zeros((F, mw), dtype=torch.int32, device="cuda")
    before = spg.sp_kernel_launch_count()
    spg.sp_batch_infer_device(b, d, F, fw, dm, mw, torch.cuda.current_stream())
    spg.sp_batch_sync(b)
    # connection images, frame images, GEMM, inhibition
    assert spg.sp_kernel_launch_count() - before == 4
    dm.zero_()
    dov = torch.full((F, ow), -1.0, dtype=torch.float32, device="cuda")
    before = spg.sp_kernel_launch_count()
    spg.sp_batch_infer_overlaps_device(b, d, F, fw, dm, mw, dov, ow, torch.cuda.current_stream())
    spg.sp_batch_sync(b)
    assert spg.sp_kernel_launch_count() - before == 3  # the connection images are kept
    masks = dm.cpu().numpy().view(np.uint32)
    ovr = dov.cpu().numpy()
    spg.sp_batch_destroy(b)
    for i, c in enumerate(cases):
        act, _, ov = oracle_run(c, frames[i], False, want_ov=True)
        assert first_diff(ovr[:, int(oo[i]):int(oo[i]) + c.C], ov) is None, f"member {i} overlaps"
        got = dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
        assert first_diff(got, act) is None, f"member {i}"
        np.testing.assert_array_equal(spg.sp_get_overlaps(hs[i]), ov[-1])
        spg.sp_destroy(hs[i])


@pytest.mark.parametrize("C,k,m,p,unit", [
    (2000, 40, 4, 0.2, True),    # two mask words per lane of the warp select
    (2000, 25, 1, 0.3, False),   # fp32 patterns (non-unit boosts), two words per lane
    (2049, 40, 4, 0.2, True),    # wider than the warp select: one CTA per frame
    (96, 0, 1, 0.3, True),       # k = 0: no column wins
    (64, 64, 1, 0.3, True),      # k = C: every nonzero column wins
    (333, 50, 36, 0.1, True),    # frames with fewer than k nonzero overlaps, and with more
])
def test_dense_global_select_edge_cases(C, k, m, p, unit):
    """Alg. 2 with global inhibition over a dense run at the extremes of the
    per-frame select (one warp per frame up to 2048 columns)."""
    boost = None if unit else synth.perm_uniform(C + 3, (C,), 0.5, 2.0)
    case = _dense_case(C, 512, 70 + C % 97, k=k, m=m, boost=boost)
    frames = _frames(37, 512, p, 71 + k)
    act, _, ov = oracle_run(case, frames, False, want_ov=True)
    if C == 333:
        nz = (ov > 0).sum(axis=1)
        assert ((nz > 0) & (nz < k)).any() and (nz >= k).any()  # the case is what it says
    got, gov, lst, _, _, ovs = _run(case, frames)
    assert first_diff(ovs, ov) is None
    assert first_diff(got, act) is None
    np.testing.assert_array_equal(gov, ov[-1])
    np.testing.assert_array_equal(lst, np.flatnonzero(act[-1]))
    if k == 0:
        assert act.sum() == 0


def test_dense_batch_with_a_local_member_uses_the_cta_select():
    """A batch whose members mix global and local inhibition: every member's
    winners still match the oracle (the per-frame CTA kernel runs them all)."""
    cases = [_dense_case(512, 512, 80, k=12, m=2),
             _dense_case(256, 512, 81, k=3, m=2, inhibition=1, gw=16, gh=16, radius=2),
             _dense_case(1500, 512, 82, k=30, m=2)]
    F = 20
    frames = [_frames(F, 512, 0.25, 90 + i) for i in range(len(cases))]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    bf = wl.batch_frames([wl.pack(f) for f in frames], fo, fw)
    d = torch.from_numpy(bf.view(np.int32)).cuda()
    mw = info["mask_words"]
    dm = torch.zeros((F, mw), dtype=torch.int32, device="cuda")
    spg.sp_batch_infer_device(b, d, F, fw, dm, mw, torch.cuda.current_stream())
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    spg.sp_batch_destroy(b)
    for i, c in enumerate(cases):
        act, _, ov = oracle_run(c, frames[i], False, want_ov=True)
        got = dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
        assert first_diff(got, act) is None, f"member {i}"
        np.testing.assert_array_equal(spg.sp_active_columns(hs[i]), np.flatnonzero(act[-1]))
        spg.sp_destroy(hs[i])


def test_dense_connection_image_follows_learning():
    """An inference run builds the connection image; learning frames in
    between change the permanences, so the next run must rebuild it."""
    case = _dense_case(512, 512, 49, k=10, m=2)
    frames = _frames(70, 512, 0.3, 50)
    packed = wl.pack(frames)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    stream = torch.cuda.current_stream()
    d = torch.from_numpy(packed.view(np.int32)).cuda()
    dm = torch.zeros((70, 16), dtype=torch.int32, device="cuda")
    spg.sp_compute_frames_device(h, d[:30], 30, packed.shape[1], False, dm[:30], stream)
    for t in range(30, 38):
        spg.sp_compute(h, packed[t], True)
    spg.sp_compute_frames_device(h, d[38:], 32, packed.shape[1], False, dm[38:], stream)
    spg.sp_sync(h)
    act0, _, _ = oracle_run(case, frames[:30], False)
    _, perm, _ = oracle_run(case, frames[30:38], True)
    act1, _, _ = oracle_run(case, frames[38:], False, perm=perm)
    got = dense(dm.cpu().numpy().view(np.uint32), 512)
    assert first_diff(got[:30], act0) is None
    assert first_diff(got[38:], act1) is None
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


def test_dense_batch_connection_image_follows_batch_learning():
    """Batch inference, then learning frames through the batch, then
    inference again: the second inference sees the learned permanences."""
    cases = [_dense_case(256, 512, 100 + i, k=8, m=2) for i in range(3)]
    F = 24
    frames = [_frames(2 * F + 4, 512, 0.3, 110 + i) for i in range(3)]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    mw = info["mask_words"]
    stream = torch.cuda.current_stream()

    def frames_dev(lo, hi):
        bf = wl.batch_frames([wl.pack(f[lo:hi]) for f in frames], fo, fw)
        return torch.from_numpy(bf.view(np.int32)).cuda()

    dm0 = torch.zeros((F, mw), dtype=torch.int32, device="cuda")
    spg.sp_batch_infer_device(b, frames_dev(0, F), F, fw, dm0, mw, stream)
    dl = torch.zeros((4, mw), dtype=torch.int32, device="cuda")
    spg.sp_batch_compute_device(b, frames_dev(F, F + 4), 4, fw, True, dl, mw, stream)
    dm1 = torch.zeros((F, mw), dtype=torch.int32, device="cuda")
    spg.sp_batch_infer_device(b, frames_dev(F + 4, 2 * F + 4), F, fw, dm1, mw, stream)
    spg.sp_batch_sync(b)
    m0 = dm0.cpu().numpy().view(np.uint32)
    m1 = dm1.cpu().numpy().view(np.uint32)
    spg.sp_batch_destroy(b)
    for i, c in enumerate(cases):
        sl = slice(int(mo[i]), int(mo[i]) + (c.C + 31) // 32)
        a0, _, _ = oracle_run(c, frames[i][:F], False)
        _, perm, _ = oracle_run(c, frames[i][F:F + 4], True)
        a1, _, _ = oracle_run(c, frames[i][F + 4:], False, perm=perm)
        assert first_diff(dense(m0[:, sl], c.C), a0) is None, f"member {i} before"
        assert first_diff(dense(m1[:, sl], c.C), a1) is None, f"member {i} after"
        spg.sp_destroy(hs[i])


@pytest.mark.parametrize("graphs", [True, False])
def test_dense_batch_repeated_runs_replay_recorded_launches(monkeypatch, graphs):
    """Runs that repeat earlier frames, masks and buffer parity replay the
    launches recorded for them (or, with graphs off, launch them directly,
    chained by programmatic dependent launch); a longer run in between
    reallocates the run buffers, which no replay may keep using.  Winners, last-frame lists and
    duty cycles (tracked through the runs without caller masks too) against
    the oracle (the last two read once the batch is gone)."""
    import oracle
    if not graphs:
        monkeypatch.setenv("SP_DISABLE_GRAPHS", "1")
    cases = [_dense_case(256, 512, 120 + i, k=6, m=2) for i in range(2)]
    hs = [spg.sp_create_from_state(c.config(duty_period=20.0), c.idx, c.perm, c.boost)
          for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    mw = info["mask_words"]
    stream = torch.cuda.current_stream()
    sizes = {"A": 16, "B": 16, "C": 40}
    frames = {name: [_frames(F, 512, 0.25 + 0.05 * i, 130 + 10 * j + i) for i in range(2)]
              for j, (name, F) in enumerate(sizes.items())}
    dev = {name: torch.from_numpy(wl.batch_frames([wl.pack(f) for f in fr], fo, fw)
                                  .view(np.int32)).cuda() for name, fr in frames.items()}
    dm = torch.zeros((40, mw), dtype=torch.int32, device="cuda")
    duty = [np.zeros(256, np.float32) for _ in cases]
    last = [None] * len(cases)
    for name, with_masks in [("A", True), ("B", False), ("A", True), ("B", False), ("C", False),
                             ("A", True), ("B", False), ("A", True)]:
        F = sizes[name]
        dm.zero_()
        spg.sp_batch_infer_device(b, dev[name], F, fw, dm[:F] if with_masks else None, mw, stream)
        spg.sp_batch_sync(b)
        masks = dm.cpu().numpy().view(np.uint32)
        for i, c in enumerate(cases):
            act, _, _ = oracle_run(c, frames[name][i], False)
            for t in range(F):
                oracle.duty_update(duty[i], act[t], 20.0)
            if with_masks:
                got = dense(masks[:F, int(mo[i]):int(mo[i]) + c.C // 32], c.C)
                assert first_diff(got, act) is None, (name, i)
            last[i] = act[-1]
    spg.sp_batch_destroy(b)  # members answer queries again
    for i in range(len(cases)):
        np.testing.assert_array_equal(spg.sp_get_duty_cycles(hs[i]), duty[i])
        np.testing.assert_array_equal(spg.sp_active_columns(hs[i]), np.flatnonzero(last[i]))
        spg.sp_destroy(hs[i])


def _run_batch(cases, frames, F):
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    oo, ow = spg.sp_batch_overlap_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    bf = wl.batch_frames([wl.pack(f) for f in frames], fo, fw)
    d = torch.from_numpy(bf.view(np.int32)).cuda()
    mw = info["mask_words"]
    dm = torch.zeros((F, mw), dtype=torch.int32, device="cuda")
    dov = torch.full((F, ow), -1.0, dtype=torch.float32, device="cuda")
    spg.sp_batch_infer_overlaps_device(b, d, F, fw, dm, mw, dov, ow, torch.cuda.current_stream())
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    ovr = dov.cpu().numpy()
    spg.sp_batch_destroy(b)
    out = []
    for i, c in enumerate(cases):
        out.append((dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C),
                    ovr[:, int(oo[i]):int(oo[i]) + c.C], spg.sp_active_columns(hs[i]),
                    spg.sp_get_overlaps(hs[i])))
        spg.sp_destroy(hs[i])
    return out


def _check(case, frames, got, ovs, lst, gov):
    act, _, ov = oracle_run(case, frames, False, want_ov=True)
    assert first_diff(ovs, ov) is None
    assert first_diff(got, act) is None
    np.testing.assert_array_equal(lst, np.flatnonzero(act[-1]))
    np.testing.assert_array_equal(gov, ov[-1])
    return act, ov


def test_dense_select_every_overlap_equal():
    """Every synapse connected: all 1024 columns of a frame have the same
    overlap, so the k winners are decided by column order alone (the k lowest
    columns).  Zero frames in the run: no winner."""
    case = _dense_case(1024, 512, 140, k=20, m=1, lo=0.25, hi=0.3)
    frames = _frames(40, 512, 0.3, 141)
    frames[5] = 0
    frames[17] = 0
    got, gov, lst, _, _, ovs = _run(case, frames)
    act, _ = _check(case, frames, got, ovs, lst, gov)
    assert act[5].sum() == 0 and act[17].sum() == 0
    assert all(np.array_equal(np.flatnonzero(act[t]), np.arange(20)) for t in range(40)
               if t not in (5, 17))


@pytest.mark.parametrize("C,n_in,F,k,m,p", [
    (1000, 1000, 600, 32, 4, 0.2),   # five 128-frame tiles, the last ragged
    (130, 777, 257, 1, 1, 0.3),      # a column tile holding 130 columns, k = 1
    (300, 640, 140, 16, 3, 0.15),    # two column tiles, the second ragged
    (1024, 512, 50, 20, 6, 0.0),     # frames with fewer than k nonzero overlaps, and with more
    (896, 1536, 256, 24, 2, 0.05),   # four column tiles, the last one ragged, twelve slices
])
def test_dense_select_shapes(C, n_in, F, k, m, p):
    """The product and the per-frame selection at the edges of their tiling:
    column, frame and input counts that fill no tile, k at both ends of the
    range where the k-th largest lane maximum bounds the k-th overlap, runs
    with fewer than k nonzero overlaps."""
    case = _dense_case(C, n_in, 150 + C % 89, k=k, m=m)
    if p > 0:
        frames = _frames(F, n_in, p, 151 + k)
    else:
        # exactly 6 or 8 active inputs: with min_overlap 6 only the columns
        # connected to all 6 (about 1 in 64: fewer than k) or to 6 of the 8
        # (about 1 in 7) keep a nonzero overlap
        rng = np.random.default_rng(153)
        frames = np.zeros((F, n_in), np.uint8)
        for t in range(F):
            frames[t, rng.choice(n_in, 6 if t % 2 else 8, replace=False)] = 1
    got, gov, lst, launches, _, ovs = _run(case, frames)
    assert launches <= 4  # connection image, frame image, product, selection
    act, ov = _check(case, frames, got, ovs, lst, gov)
    if p == 0:
        nz = (ov > 0).sum(axis=1)
        assert ((nz > 0) & (nz < k)).any() and (nz >= k).any()  # the case is what it says


def test_dense_select_non_unit_boosts_with_ties():
    """Boosts that map different raw counts to one overlap and equal counts
    to many: ties across column tiles resolve to the lowest columns, as Alg.
    2's column order asks."""
    C = 768
    boost = np.where(np.arange(C) % 3 == 0, 1.5, 1.0).astype(np.float32)
    boost[::7] = 0.75
    case = _dense_case(C, 640, 160, k=17, m=2, boost=boost)
    frames = _frames(100, 640, 0.25, 161)
    got, gov, lst, _, _, ovs = _run(case, frames)
    _check(case, frames, got, ovs, lst, gov)


def test_dense_batch_members_of_mixed_widths_and_frames():
    """A batch whose members have 1 to 4 column tiles and different input
    sizes, over 300 frames (three frame tiles): every member's overlaps,
    winners, last list and last overlaps."""
    shapes = [(100, 300, 3), (1024, 1024, 20), (513, 700, 9), (256, 4096, 8)]
    cases = [_dense_case(C, n, 170 + i, k=k, m=3) for i, (C, n, k) in enumerate(shapes)]
    F = 300
    frames = [_frames(F, c.n_in, 0.03 + 0.06 * i, 180 + i) for i, c in enumerate(cases)]
    for i, (got, ovs, lst, gov) in enumerate(_run_batch(cases, frames, F)):
        _check(cases[i], frames[i], got, ovs, lst, gov)
