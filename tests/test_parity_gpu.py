"""Parity of the CUDA Spatial Pooler (through the C ABI) with the CPU oracle.

Bar: bit-exact.  Overlaps are integer counts times an fp32 boost (one
rounding on both sides), the winner set is unique under (overlap desc, index
asc), and learning is one fp32 add or subtract plus a clamp per synapse, so
the oracle and the kernels must agree on every active mask, every overlap
and every permanence, frame after frame: the sequence calls record every
frame's boosted overlaps (sp_compute_frames_overlaps_device) and each one is
compared element by element.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402
from conftest import GOLDEN  # noqa: E402
from helpers import dense, first_diff, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a_u32):
    return torch.from_numpy(np.ascontiguousarray(a_u32).view(np.int32)).cuda()


def gpu_frames(case, frames_u8, learn, h=None, want=("masks", "perm", "ov")):
    """Run frames through sp_compute_frames_overlaps_device (the cluster
    sequence kernel, or one fused kernel per frame), recording every frame's
    overlaps."""
    packed = wl.pack(frames_u8)
    n = packed.shape[0]
    mw = (case.C + 31) // 32
    own = h is None
    if own:
        h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    stream = torch.cuda.current_stream()
    d = _dev(packed)
    dm = torch.zeros((n, mw), dtype=torch.int32, device="cuda")
    dov = torch.full((n, case.C), -1.0, dtype=torch.float32, device="cuda")
    spg.sp_compute_frames_overlaps_device(h, d, n, packed.shape[1], learn, dm, dov, stream)
    spg.sp_sync(h)
    out = {"masks": dense(dm.cpu().numpy().view(np.uint32), case.C),
           "ovs": dov.cpu().numpy()}
    if "perm" in want:
        out["perm"] = spg.sp_get_permanences(h)
    if "ov" in want:
        out["ov"] = spg.sp_get_overlaps(h)
    if own:
        spg.sp_destroy(h)
    return out


def assert_same(case, frames_u8, learn, label=""):
    act, perm, ov = oracle_run(case, frames_u8, learn, want_ov=True)
    g = gpu_frames(case, frames_u8, learn)
    d = first_diff(g["ovs"], ov)
    assert d is None, f"{label}: first differing overlap (frame, column) {d}"
    d = first_diff(g["masks"], act)
    assert d is None, f"{label}: first differing (frame, column) {d}"
    np.testing.assert_array_equal(g["ov"], ov[-1], err_msg=f"{label}: last-frame overlaps")
    d = first_diff(g["perm"], perm)
    assert d is None, f"{label}: first differing permanence (column, synapse) {d}"
    return act


# ------------------------------------------------------------------ golden ---

def test_golden_two_frame_example_on_gpu():
    g = json.load(open(os.path.join(GOLDEN, "sp_two_frame_example.json")))
    idx = np.array(g["idx"], np.uint32)
    perm = np.array(g["perm"], np.float32)
    cfg = spg.sp_config_init(input_w=g["n_in"], input_h=1, num_columns=4,
                             synapses_per_column=4, connect_threshold=g["connect_threshold"],
                             perm_inc=g["perm_inc"], perm_dec=g["perm_dec"],
                             min_overlap=g["min_overlap"], winners_set_size=g["winners_set_size"])
    sp = spg.SpatialPooler(cfg, state=(idx, perm, np.array(g["boost"], np.float32)))
    for x, e in zip(g["frames"], g["expected"]):
        sp.compute(synth.pack_bits(np.array(x, np.uint8)), learn=True)
        np.testing.assert_array_equal(sp.active_columns(), np.flatnonzero(e["active"]))
        np.testing.assert_array_equal(spg.sp_get_overlaps(sp.h), np.array(e["ov"], np.float32))
        np.testing.assert_array_equal(spg.sp_get_permanences(sp.h),
                                      np.array(e["perm_after"], np.float32))
    sp.close()


# --------------------------------------------------- the five workloads -----

def test_small_config_inference_then_learning():
    """32x32 Bernoulli(0.1) input, 256 columns x 16 synapses: 100 frames of
    inference, then 100 frames of learning, on one handle."""
    case = wl.small_case()
    frames = wl.small_frames(200)
    act_i, perm_i, ov_i = oracle_run(case, frames[:100], False, want_ov=True)
    act_l, perm_l, ov_l = oracle_run(case, frames[100:], True, perm=perm_i, want_ov=True)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    g1 = gpu_frames(case, frames[:100], False, h=h)
    g2 = gpu_frames(case, frames[100:], True, h=h)
    spg.sp_destroy(h)
    assert first_diff(g1["ovs"], ov_i) is None
    assert first_diff(g2["ovs"], ov_l) is None
    assert first_diff(g1["masks"], act_i) is None
    np.testing.assert_array_equal(g1["perm"], case.perm)
    assert first_diff(g2["masks"], act_l) is None
    np.testing.assert_array_equal(g2["ov"], ov_l[-1])
    np.testing.assert_array_equal(g2["perm"], perm_l)
    assert act_l.sum() > 0


def test_frame_config_full_500_frames_learning(seq_path):
    """960x540 blobbed frames, 1024 columns x 256 windowed synapses, k 40,
    500 frames with learning: the benchmark's workload, in its launch
    configuration, compared on every frame's active set and the final state."""
    case = wl.frame_case()
    frames = wl.blob_frames(500)
    act = assert_same(case, frames, True, "frame/500")
    assert (act.sum(axis=1) == 40).mean() > 0.9  # ties at rank 40 are exercised


@pytest.fixture(params=["cluster", "per-frame"])
def seq_path(request, monkeypatch):
    """Frame sequences run either in one persistent cluster launch (state in
    shared memory, when it fits) or as one fused kernel per frame."""
    if request.param == "per-frame":
        monkeypatch.setenv("SP_DISABLE_CLUSTER", "1")
    return request.param


@pytest.mark.parametrize("C", [256, 1024, 4096])
def test_parameter_sweep(C, seq_path):
    """Columns x synapses x min_overlap x k x {global, 9x9 local} on the
    960x540 blobbed input, 8 learning frames each."""
    frames = wl.blob_frames(8, seed=wl.BASE_SEED + 3)
    for S in (16, 64, 256):
        for m in (2, 4, 8):
            for k in (8, 32, 128):
                for inh in (0, 1):
                    case = wl.grid_case("sweep", C, S, wl.BASE_SEED + 3 + C + S, min_overlap=m,
                                        k=k, inhibition=inh, radius=4)
                    assert_same(case, frames, True, f"C{C} S{S} m{m} k{k} inh{inh} {seq_path}")


# ------------------------------------------------------------- edge cases ---

def _uniform_case(C, S, n_in, seed, W=None, H=1, **kw):
    idx = synth.pool_uniform(synth.derive_seed(seed, 1, 0), C, S, n_in)
    perm = synth.perm_uniform(synth.derive_seed(seed, 2, 0), (C, S), kw.pop("lo", 0.1),
                              kw.pop("hi", 0.3))
    boost = kw.pop("boost", None)
    if boost is None:
        boost = np.ones(C, np.float32)
    return wl.Case("edge", W or n_in, H, C, S, idx, perm, boost, **kw)


def _bern(n_frames, n_in, p, seed):
    return np.stack([synth.frame_bernoulli(synth.derive_seed(seed, 3, t), n_in, p)
                     for t in range(n_frames)])


def test_ragged_sizes_scalar_path_and_boost(seq_path):
    """C and n_in not multiples of 32, S not a multiple of 4 (scalar loads),
    non-unit boosts (fp32 products that are not integers), min_overlap 1."""
    boost = synth.perm_uniform(77, (1000,), 0.5, 2.0)
    case = _uniform_case(1000, 17, 1000, 31, boost=boost, min_overlap=1, k=7)
    assert_same(case, _bern(30, 1000, 0.3, 5), True, f"ragged {seq_path}")


@pytest.mark.parametrize("k", [0, 1, 5000])
def test_k_extremes(k, seq_path):
    case = _uniform_case(2000, 32, 4096, 41, k=k, min_overlap=2)
    act = assert_same(case, _bern(12, 4096, 0.2, 6), True, f"k={k} {seq_path}")
    if k == 0:
        assert act.sum() == 0


def test_all_zero_and_all_one_frames():
    case = _uniform_case(512, 24, 2048, 51, k=20, min_overlap=1)
    frames = np.stack([np.zeros(2048, np.uint8), np.ones(2048, np.uint8),
                       np.zeros(2048, np.uint8), np.ones(2048, np.uint8)])
    act = assert_same(case, frames, True, "zeros/ones")
    assert act[0].sum() == 0 and act[1].sum() == 20


@pytest.mark.parametrize("thr", [0.0, 1.5])
def test_threshold_special_cases(thr):
    case = _uniform_case(300, 20, 640, 61, thr=thr, min_overlap=0, k=12)
    assert_same(case, _bern(6, 640, 0.4, 7), True, f"thr={thr}")


def test_single_column_single_synapse():
    case = _uniform_case(1, 1, 33, 71, min_overlap=1, k=1, lo=0.15, hi=0.25)
    assert_same(case, _bern(20, 33, 0.5, 8), True, "1x1")


def test_tie_stress_global(seq_path):
    """Every synapse connected, Bernoulli(0.5) input: overlaps ~ Bin(16, 0.5)
    over 2048 columns, so dozens of columns tie at the k-th value; plus a
    frame where all columns tie (all-ones input)."""
    case = _uniform_case(2048, 16, 4096, 81, lo=0.25, hi=0.25, k=40, min_overlap=1)
    frames = np.concatenate([_bern(10, 4096, 0.5, 9), np.ones((1, 4096), np.uint8)])
    act = assert_same(case, frames, False, "ties")
    np.testing.assert_array_equal(np.flatnonzero(act[-1]), np.arange(40))


@pytest.mark.parametrize("k", [300, 700])
def test_wide_overlap_spread_global(k, seq_path):
    """Columns from never to always connected (each column's permanence range
    is shifted by its index), so a frame's overlaps spread over about a
    hundred values and the k-th largest lies several 32-value rounds below the
    largest: the cluster path's decision reads the CTAs' count histograms
    round by round from the top."""
    C, S, n = 1024, 256, 4096
    idx = synth.pool_uniform(synth.derive_seed(91, 1, 0), C, S, n)
    u = synth.perm_uniform(synth.derive_seed(91, 2, 0), (C, S), 0.0, 0.2)
    perm = (u + np.linspace(0.0, 0.4, C, dtype=np.float32)[:, None]).astype(np.float32)
    case = wl.Case("spread", n, 1, C, S, idx, perm, np.ones(C, np.float32), k=k, min_overlap=1)
    act = assert_same(case, _bern(12, n, 0.5, 10), True, f"spread k={k} {seq_path}")
    assert (act.sum(axis=1) == k).all()


def test_local_inhibition_non_square_grid_and_radius_zero(seq_path):
    for gw, gh, r, k in ((40, 25, 3, 5), (33, 7, 0, 1), (16, 16, 20, 9)):
        C = gw * gh
        idx = synth.pool_uniform(synth.derive_seed(91, 1, r), C, 32, 3000)
        perm = synth.perm_uniform(synth.derive_seed(91, 2, r), (C, 32), 0.1, 0.3)
        case = wl.Case("local", 3000, 1, C, 32, idx, perm, np.ones(C, np.float32), k=k,
                       min_overlap=2, inhibition=1, gw=gw, gh=gh, radius=r)
        assert_same(case, _bern(10, 3000, 0.3, 10 + r), True, f"local {gw}x{gh} r{r} {seq_path}")


@pytest.mark.parametrize("inh", [0, 1])
def test_max_columns(inh):
    """SP_MAX_COLUMNS columns (the largest shared-memory footprint of the
    inhibition stage), global and 9x9 local on a 128x128 grid."""
    C = spg.SP_MAX_COLUMNS
    case = _uniform_case(C, 8, 4096, 101, k=300, min_overlap=2, inhibition=inh,
                         gw=128 if inh else 0, gh=128 if inh else 0, radius=4 if inh else 0)
    assert_same(case, _bern(3, 4096, 0.3, 11), True, f"max C inh{inh}")


# ------------------------------------------------------ API equivalence -----

def test_single_frame_host_path_matches_sequence_and_mixed_learning():
    """sp_compute (host input, one frame per call) with a mixed learn pattern
    and permanence reads between frames equals the oracle."""
    case = wl.small_case(seed=wl.BASE_SEED + 11)
    frames = wl.small_frames(40, seed=wl.BASE_SEED + 11)
    learn = [(t // 3) % 2 == 0 for t in range(40)]
    perm = case.perm.copy()
    import oracle
    from helpers import oracle_params
    p = oracle_params(case)
    sp = spg.SpatialPooler(case.config(), state=(case.idx, case.perm, case.boost))
    for t in range(40):
        act = oracle.run(p, case.idx, perm, case.boost, frames[t:t + 1], learn[t])[0]
        sp.compute(synth.pack_bits(frames[t]), learn[t])
        np.testing.assert_array_equal(sp.active_columns(), np.flatnonzero(act), err_msg=f"t={t}")
        if t % 7 == 0:
            np.testing.assert_array_equal(spg.sp_get_permanences(sp.h), perm)
    np.testing.assert_array_equal(spg.sp_get_permanences(sp.h), perm)
    sp.close()


def test_device_single_frame_path_matches_oracle():
    case = wl.frame_case(seed=wl.BASE_SEED + 12)
    frames = wl.blob_frames(12, seed=wl.BASE_SEED + 12)
    act, perm, _ = oracle_run(case, frames, True)
    packed = wl.pack(frames)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    stream = torch.cuda.current_stream()
    for t in range(12):
        d = _dev(packed[t])
        spg.sp_compute_device(h, d, True, stream)
        np.testing.assert_array_equal(spg.sp_active_columns(h), np.flatnonzero(act[t]))
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


def test_host_pipelined_frames_match_oracle_across_chunks():
    """sp_compute_frames: pinned host frames, chunked H2D / compute / D2H on
    separate streams; 70 frames span three staging chunks."""
    case = wl.frame_case(seed=wl.BASE_SEED + 13)
    frames = wl.blob_frames(70, seed=wl.BASE_SEED + 13)
    act, perm, _ = oracle_run(case, frames, True)
    packed = wl.pack(frames)
    pinned = torch.from_numpy(packed.view(np.int32)).pin_memory()
    masks = torch.zeros((70, 32), dtype=torch.int32).pin_memory()
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    spg.sp_compute_frames(h, pinned.numpy().view(np.uint32), True, masks.numpy().view(np.uint32))
    assert first_diff(dense(masks.numpy().view(np.uint32), case.C), act) is None
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    # a second call continues the same sequence (pending learning carried over)
    frames2 = wl.blob_frames(5, seed=wl.BASE_SEED + 13, start=70)
    act2, perm2, _ = oracle_run(case, frames2, True, perm=perm)
    m2 = np.zeros((5, 32), np.uint32)
    spg.sp_compute_frames(h, wl.pack(frames2), True, m2)
    assert first_diff(dense(m2, case.C), act2) is None
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm2)
    spg.sp_destroy(h)


def test_seeded_create_matches_generators():
    """sp_create draws the same pools and permanences as the synth module."""
    cfg = spg.sp_config_init(input_w=960, input_h=540, num_columns=1024, col_grid_w=32,
                             col_grid_h=32, synapses_per_column=256, pool_mode=spg.SP_POOL_WINDOW,
                             rf_w=64, rf_h=64, perm_init_lo=0.1, perm_init_hi=0.3, seed=1234)
    h = spg.sp_create(cfg)
    idx = synth.pool_window(synth.derive_seed(1234, 1, 0), 32, 32, 960, 540, 64, 64, 256)
    perm = synth.perm_uniform(synth.derive_seed(1234, 2, 0), (1024, 256), 0.1, 0.3)
    np.testing.assert_array_equal(spg.sp_get_pool(h), idx)
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    np.testing.assert_array_equal(spg.sp_get_boost(h), np.ones(1024, np.float32))
    spg.sp_destroy(h)


def test_cap_too_small_reports_needed_size():
    case = _uniform_case(256, 16, 1024, 111, k=10, min_overlap=1)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    spg.sp_compute(h, synth.pack_bits(np.ones(1024, np.uint8)), False)
    with pytest.raises(spg.SpError) as e:
        spg.sp_active_columns(h, cap=3)
    assert e.value.status == 1
    assert spg.sp_active_columns(h).size == 10
    spg.sp_destroy(h)


def test_set_boost_changes_overlaps_exactly():
    case = _uniform_case(500, 32, 2048, 121, k=25, min_overlap=3)
    frames = _bern(4, 2048, 0.3, 12)
    boost = synth.perm_uniform(5, (500,), 0.25, 4.0)
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    spg.sp_set_boost(h, boost)
    case_b = wl.Case("b", case.W, 1, case.C, case.S, case.idx, case.perm, boost, k=25,
                     min_overlap=3)
    act, perm, ov = oracle_run(case_b, frames, True, want_ov=True)
    g = gpu_frames(case_b, frames, True, h=h)
    assert first_diff(g["ovs"], ov) is None
    assert first_diff(g["masks"], act) is None
    np.testing.assert_array_equal(g["ov"], ov[-1])
    np.testing.assert_array_equal(g["perm"], perm)
    spg.sp_destroy(h)


def test_recorded_sequences_replay_and_boost_change():
    """Frame sequences are recorded once as CUDA graphs and replayed: three
    passes over the same device buffers (record, record with learning
    pending, replay), then a non-unit boost (which switches the inhibition
    path baked into a recording) and two more passes."""
    case = wl.frame_case(seed=wl.BASE_SEED + 14)
    frames = wl.blob_frames(9, seed=wl.BASE_SEED + 14)
    packed = wl.pack(frames)
    stream = torch.cuda.current_stream()
    d = _dev(packed)
    dm = torch.zeros((9, 32), dtype=torch.int32, device="cuda")
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    perm = case.perm.copy()
    boost = synth.perm_uniform(99, (case.C,), 0.5, 1.5)
    for p in range(5):
        if p == 3:
            spg.sp_set_boost(h, boost)
            case = wl.Case(case.name, case.W, case.H, case.C, case.S, case.idx, case.perm, boost,
                           k=case.k, min_overlap=case.min_overlap)
        act, perm, _ = oracle_run(case, frames, True, perm=perm)
        spg.sp_compute_frames_device(h, d, 9, packed.shape[1], True, dm, stream)
        spg.sp_sync(h)
        got = dense(dm.cpu().numpy().view(np.uint32), case.C)
        assert first_diff(got, act) is None, f"pass {p}"
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


def test_pending_learning_hands_over_between_paths():
    """Single frames (per-frame kernel, learning deferred to the next frame)
    and sequences (persistent cluster launch) interleaved on one handle: the
    learning a single frame leaves pending is applied by the next sequence."""
    case = wl.frame_case(seed=wl.BASE_SEED + 15)
    frames = wl.blob_frames(40, seed=wl.BASE_SEED + 15)
    packed = wl.pack(frames)
    plan = [(0, 3, True), (3, 23, True), (23, 25, True), (25, 35, False), (35, 36, True),
            (36, 40, True)]
    perm = case.perm.copy()
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    stream = torch.cuda.current_stream()
    d = _dev(packed)
    for a0, a1, learn in plan:
        act, perm, _ = oracle_run(case, frames[a0:a1], learn, perm=perm)
        if a1 - a0 < 8:
            for t in range(a0, a1):
                spg.sp_compute_device(h, d[t], learn, stream)
                np.testing.assert_array_equal(spg.sp_active_columns(h),
                                              np.flatnonzero(act[t - a0]), err_msg=f"t={t}")
        else:
            dm = torch.zeros((a1 - a0, 32), dtype=torch.int32, device="cuda")
            spg.sp_compute_frames_device(h, d[a0], a1 - a0, packed.shape[1], learn, dm, stream)
            spg.sp_sync(h)
            got = dense(dm.cpu().numpy().view(np.uint32), case.C)
            assert first_diff(got, act) is None, f"frames {a0}..{a1}"
            np.testing.assert_array_equal(spg.sp_active_columns(h), np.flatnonzero(act[-1]))
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)


@pytest.mark.parametrize("k", [1, 7, 40, 299, 300, 400])
def test_paper_literal_inhibition(k):
    """The word-for-word reading of Alg. 2 (strict '>' against the k-th
    largest overlap of the other columns, floor 1) on the per-frame kernel:
    heavy ties at the boundary, k up to and beyond C, boosts that push some
    overlaps to 1 or below."""
    boost = np.where(np.arange(300) % 5 == 0, np.float32(0.25), np.float32(1.0)).astype(np.float32)
    case = _uniform_case(300, 12, 512, 131, k=k, min_overlap=1, lo=0.2, hi=0.2, boost=boost,
                         inhibition=2)
    frames = _bern(6, 512, 0.35, 14)
    act, perm, ov = oracle_run(case, frames, True, want_ov=True)
    assert act.sum() > 0
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    for t in range(6):
        spg.sp_compute(h, synth.pack_bits(frames[t]), True)
        np.testing.assert_array_equal(spg.sp_active_columns(h), np.flatnonzero(act[t]),
                                      err_msg=f"frame {t}")
    np.testing.assert_array_equal(spg.sp_get_permanences(h), perm)
    spg.sp_destroy(h)
