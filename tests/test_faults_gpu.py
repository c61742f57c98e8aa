"""Checkpoint / resume, bounded waits and injected allocation failures.

Failures are made on the host (a wait bound shorter than the work, an
allocation refused by the library's own allocator hook); nothing here faults,
traps or hangs the GPU."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import workloads as wl  # noqa: E402
from helpers import dense, first_diff, oracle_params  # noqa: E402

pytestmark = pytest.mark.gpu


def _frames_dev(packed):
    return torch.from_numpy(np.ascontiguousarray(packed).view(np.int32)).cuda()


def test_checkpoint_resume_equals_uninterrupted(tmp_path):
    """250 learning frames, save, load into a new handle, 250 more: the same
    active sets, permanences and duty cycles as 500 frames straight."""
    case = wl.frame_case(seed=wl.BASE_SEED + 700)
    frames = wl.blob_frames(500, seed=wl.BASE_SEED + 700)
    packed = wl.pack(frames)
    p = oracle_params(case)
    perm = case.perm.copy()
    act = oracle.run(p, case.idx, perm, case.boost, frames, True)
    duty = np.zeros(case.C, np.float32)
    for t in range(500):
        oracle.duty_update(duty, act[t], 100.0)
    cfg = case.config(duty_period=100.0)
    stream = torch.cuda.current_stream()
    h = spg.sp_create_from_state(cfg, case.idx, case.perm, case.boost)
    d = _frames_dev(packed)
    m1 = torch.zeros((250, 32), dtype=torch.int32, device="cuda")
    spg.sp_compute_frames_device(h, d, 250, packed.shape[1], True, m1, stream)
    path = os.path.join(tmp_path, "sp.ckpt")
    spg.sp_save(h, path)
    spg.sp_destroy(h)
    h2 = spg.sp_load(path)
    assert spg.sp_get_info(h2)["frames"] == 250
    m2 = torch.zeros((250, 32), dtype=torch.int32, device="cuda")
    spg.sp_compute_frames_device(h2, d[250], 250, packed.shape[1], True, m2, stream)
    spg.sp_sync(h2)
    got = np.concatenate([dense(m.cpu().numpy().view(np.uint32), case.C) for m in (m1, m2)])
    assert first_diff(got, act) is None
    np.testing.assert_array_equal(spg.sp_get_permanences(h2), perm)
    np.testing.assert_array_equal(spg.sp_get_duty_cycles(h2), duty)
    spg.sp_destroy(h2)
    with pytest.raises(spg.SpError):
        spg.sp_load(os.path.join(tmp_path, "missing.ckpt"))
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(spg.SpError):
        spg.sp_load(path)


def test_bounded_wait_expires_and_work_completes():
    """A 1 ms bound on a ~10 ms sequence: the wait returns SP_ETIMEOUT, the
    work keeps running, and a later wait with the default bound succeeds
    with the correct result."""
    case = wl.frame_case(seed=wl.BASE_SEED + 701)
    frames = wl.blob_frames(64, seed=wl.BASE_SEED + 701)
    packed = wl.pack(frames)
    reps = 40
    big = np.ascontiguousarray(np.tile(packed, (reps, 1)))
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    d = _frames_dev(big)
    spg.sp_set_timeout_ms(h, 1)
    spg.sp_compute_frames_device(h, d, big.shape[0], big.shape[1], True, None,
                                 torch.cuda.current_stream())
    with pytest.raises(spg.SpError) as e:
        spg.sp_sync(h)
    assert e.value.status == 4  # SP_ETIMEOUT
    spg.sp_set_timeout_ms(h, 0)  # back to the default bound
    spg.sp_sync(h)
    perm = case.perm.copy()
    act = oracle.run(oracle_params(case), case.idx, perm, case.boost,
                     np.tile(frames, (reps, 1)), True)
    np.testing.assert_array_equal(spg.sp_active_columns(h), np.flatnonzero(act[-1]))
    spg.sp_destroy(h)


def test_injected_allocation_failure(monkeypatch):
    case = wl.small_case()
    monkeypatch.setenv("SP_INJECT_ALLOC_FAILURE", "1")
    with pytest.raises(spg.SpError) as e:
        spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    assert e.value.status == 2  # SP_ENOMEM
    with pytest.raises(spg.SpError) as e:
        spg.sp_server_create(max_streams=2, queue_depth=2, max_input_words=64,
                             device_budget_bytes=1 << 30, max_active=16)
    assert e.value.status == 2
    monkeypatch.delenv("SP_INJECT_ALLOC_FAILURE")
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    spg.sp_compute(h, wl.pack(wl.small_frames(1))[0], True)
    assert spg.sp_active_columns(h).size <= 10
    spg.sp_destroy(h)


def test_device_wait_expires_then_the_batch_runs_clean():
    """The one wait inside a persistent batch launch (an item of a member's
    frame t + 1 waiting for that member's frame t) given a bound of 1 ns: the
    launch stops early and the batch reports SP_ETIMEOUT without hanging;
    with the default bound restored, the same batch then computes a learning
    run whose overlaps, winners and permanences equal the oracle's."""
    cases = [wl.frame_case(seed=wl.BASE_SEED + 720 + i) for i in range(4)]
    frames = [wl.blob_frames(12, seed=wl.BASE_SEED + 720 + i) for i in range(4)]
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    oo, ow = spg.sp_batch_overlap_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    d = torch.from_numpy(wl.batch_frames([wl.pack(f) for f in frames], fo, fw).view(np.int32)).cuda()
    st = torch.cuda.current_stream()
    # 4 members x 8 CTAs per frame: every frame-1 item is taken while frame 0
    # is still being computed, so it must wait, and a 1 ns bound expires
    spg.sp_batch_set_device_wait_ns(b, 1)
    spg.sp_batch_compute_device(b, d, 12, fw, False, None, 0, st)
    with pytest.raises(spg.SpError) as e:
        spg.sp_batch_sync(b)
    assert e.value.status == 4  # SP_ETIMEOUT
    spg.sp_batch_set_device_wait_ns(b, 0)  # the default bound
    mw = info["mask_words"]
    dm = torch.zeros((12, mw), dtype=torch.int32, device="cuda")
    dov = torch.full((12, ow), -1.0, dtype=torch.float32, device="cuda")
    spg.sp_batch_compute_overlaps_device(b, d, 12, fw, True, dm, mw, dov, ow, st)
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    ovr = dov.cpu().numpy()
    spg.sp_batch_destroy(b)
    for i, c in enumerate(cases):
        p = oracle_params(c)
        perm = c.perm.copy()
        act, ov = oracle.run(p, c.idx, perm, c.boost, frames[i], True, want_ov=True)
        assert first_diff(ovr[:, int(oo[i]):int(oo[i]) + c.C], ov) is None, f"member {i} overlaps"
        got = dense(masks[:, int(mo[i]):int(mo[i]) + (c.C + 31) // 32], c.C)
        assert first_diff(got, act) is None, f"member {i} winners"
        np.testing.assert_array_equal(spg.sp_get_permanences(hs[i]), perm, err_msg=f"member {i}")
        spg.sp_destroy(hs[i])
