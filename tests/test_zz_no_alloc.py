"""sp_step_noalloc: one frame on caller-owned device state, allocating nothing.

Some callers cannot allocate device memory at the moment they process a
frame: a real-time video pipeline stage whose per-frame callback must not
block (cudaMalloc and cudaFree may synchronise the whole device), or a host
that runs against a fixed device-memory budget.  For them the library keeps
the step kernel's scratch in a static device array and the caller passes its
own state, input and outputs.  These tests drive that entry point through the
C ABI and require its output to equal the handle-based entry point's
(sp_compute_device) exactly -- the same bit-exact bar as every other parity
test here -- on two calls in a row, so the second call also checks that the
shared scratch left over from the first does not leak into its result.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _two_calls_against_handle(case, frames_u8, learn):
    packed = wl.pack(frames_u8)
    stream = torch.cuda.current_stream()
    cfg = case.config()
    h = spg.sp_create_from_state(cfg, case.idx, case.perm, case.boost)
    d_idx = _dev_u32(case.idx)
    d_perm = torch.from_numpy(case.perm.copy()).cuda()
    d_boost = torch.from_numpy(np.ascontiguousarray(case.boost)).cuda()
    mw = (case.C + 31) // 32
    d_mask = torch.full((mw,), -1, dtype=torch.int32, device="cuda")
    d_list = torch.full((1 + case.C,), -1, dtype=torch.int32, device="cuda")
    sizes = []
    for t in range(packed.shape[0]):
        d_x = _dev_u32(packed[t])
        spg.sp_compute_device(h, d_x, learn, stream)
        want = spg.sp_active_columns(h)
        want_perm = spg.sp_get_permanences(h)
        spg.sp_step_noalloc(cfg, d_idx, d_perm, d_boost, d_x, learn, d_mask, d_list, stream)
        torch.cuda.synchronize()
        lst = d_list.cpu().numpy().view(np.uint32)
        got = lst[1:1 + lst[0]]
        np.testing.assert_array_equal(got, want, err_msg=f"call {t}: active list")
        dense = spg.masks_to_dense(d_mask.cpu().numpy().view(np.uint32), case.C)
        ref = np.zeros(case.C, np.uint8)
        ref[want] = 1
        np.testing.assert_array_equal(dense, ref, err_msg=f"call {t}: active mask")
        np.testing.assert_array_equal(d_perm.cpu().numpy(), want_perm,
                                      err_msg=f"call {t}: permanences")
        sizes.append(len(want))
    spg.sp_destroy(h)
    return sizes


def test_noalloc_matches_handle_path_two_calls_global():
    """960x540 blobbed frames, 1024 columns x 256 windowed synapses, k = 40,
    learning on: two consecutive frames."""
    case = wl.frame_case(seed=wl.BASE_SEED + 21)
    sizes = _two_calls_against_handle(case, wl.blob_frames(2, seed=wl.BASE_SEED + 21), True)
    assert sizes == [40, 40]


def test_noalloc_matches_handle_path_two_calls_local_ragged():
    """9x9 local inhibition on a 30x20 grid, S = 17 (scalar loads), n_in not
    a multiple of 32, inference then learning."""
    C, S, n = 600, 17, 1000
    idx = synth.pool_uniform(synth.derive_seed(7, 1, 0), C, S, n)
    perm = synth.perm_uniform(synth.derive_seed(7, 2, 0), (C, S), 0.1, 0.3)
    case = wl.Case("local", n, 1, C, S, idx, perm, np.ones(C, np.float32), k=3, min_overlap=1,
                   inhibition=1, gw=30, gh=20, radius=4)
    frames = np.stack([synth.frame_bernoulli(synth.derive_seed(7, 3, t), n, 0.3) for t in range(2)])
    sizes = _two_calls_against_handle(case, frames, True)
    assert min(sizes) > 0


def test_noalloc_matches_handle_path_paper_literal_k_at_least_c():
    """The word-for-word Alg. 2 mode with winners_set_size >= C (the floor of
    1 alone decides), then with k < C and boundary ties."""
    C, S, n = 300, 12, 512
    idx = synth.pool_uniform(synth.derive_seed(9, 1, 0), C, S, n)
    perm = np.full((C, S), 0.2, np.float32)
    frames = np.stack([synth.frame_bernoulli(synth.derive_seed(9, 3, t), n, 0.35)
                       for t in range(2)])
    for k in (C, C + 50, 40):
        case = wl.Case("literal", n, 1, C, S, idx, perm, np.ones(C, np.float32), k=k,
                       min_overlap=1, inhibition=2)
        sizes = _two_calls_against_handle(case, frames, True)
        assert min(sizes) > 0


def test_noalloc_matches_handle_path_non_unit_boosts():
    """Boosts that are not 1 (the radix select over fp32 products), learning."""
    C, S, n = 700, 32, 2048
    idx = synth.pool_uniform(synth.derive_seed(11, 1, 0), C, S, n)
    perm = synth.perm_uniform(synth.derive_seed(11, 2, 0), (C, S), 0.1, 0.3)
    boost = synth.perm_uniform(synth.derive_seed(11, 4, 0), (C,), 0.5, 2.0)
    case = wl.Case("boosted", n, 1, C, S, idx, perm, boost, k=21, min_overlap=2)
    frames = np.stack([synth.frame_bernoulli(synth.derive_seed(11, 3, t), n, 0.3)
                       for t in range(2)])
    sizes = _two_calls_against_handle(case, frames, True)
    assert sizes == [21, 21]


def test_noalloc_allocates_nothing_after_setup():
    """After the first call on the device (which may load the library's device
    code), further calls leave the device's free memory unchanged."""
    case = wl.small_case()
    packed = wl.pack(wl.small_frames(6))
    cfg = case.config()
    d_idx = _dev_u32(case.idx)
    d_perm = torch.from_numpy(case.perm.copy()).cuda()
    d_boost = torch.from_numpy(case.boost).cuda()
    d_x = _dev_u32(packed)
    d_mask = torch.zeros((case.C + 31) // 32, dtype=torch.int32, device="cuda")
    d_list = torch.zeros(1 + case.C, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    spg.sp_step_noalloc(cfg, d_idx, d_perm, d_boost, d_x[0], True, d_mask, d_list, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in range(1, 6):
        spg.sp_step_noalloc(cfg, d_idx, d_perm, d_boost, d_x[t], True, d_mask, d_list, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cfg = spg.sp_config_init(input_w=4096, input_h=1, num_columns=16385, synapses_per_column=8)
    t = torch.zeros(16385 * 8, dtype=torch.int32, device="cuda")
    with pytest.raises(spg.SpError) as e:
        spg.sp_step_noalloc(cfg, t, t, t, t, False, t, t)
    assert e.value.status == 1
    assert "SP_NOALLOC_MAX_COLUMNS" in spg.sp_last_error()


@pytest.mark.parametrize("bad", [dict(reserved=1), dict(duty_period=float("nan")),
                                 dict(col_grid_w=7, col_grid_h=7)])
def test_noalloc_rejects_what_sp_create_rejects(bad):
    """The configuration checks are sp_create's: a non-zero reserved field, a
    NaN duty period, a column grid that does not match num_columns."""
    cfg = spg.sp_config_init(input_w=1024, input_h=1, num_columns=256, synapses_per_column=16,
                             **bad)
    t = torch.zeros(256 * 16, dtype=torch.int32, device="cuda")
    with pytest.raises(spg.SpError) as e:
        spg.sp_step_noalloc(cfg, t, t, t, t, False, t, t)
    assert e.value.status == 1
    with pytest.raises(spg.SpError):
        spg.sp_create(cfg)
