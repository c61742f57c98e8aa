"""Frame encoder on the GPU (Section 2; "Adaptive Video Encoder", Section
3.1) against the oracle's encoder, alone and feeding the SP.  The encoder is
integer arithmetic end to end, so the bar is bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402
from helpers import dense, first_diff, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu

SENTINEL = 0xDEADBEEF


def _frames(n, W, H, ch, seed):
    rgb = wl.rgb_frames(n, W, H, seed=seed)
    return rgb if ch == 3 else np.ascontiguousarray(rgb[..., 1])


def _oracle_bits(frames, reduce, block, offset):
    return np.stack([oracle.encode(f, reduce, block, offset).reshape(-1) for f in frames])


def _unpack(words, n_bits):
    b = np.unpackbits(words.view(np.uint8), bitorder="little")
    return b.reshape(words.shape[0], -1)[:, :n_bits]


@pytest.mark.parametrize("W,H,ch,reduce,block,offset", [
    (960, 540, 3, 1, 11, 2),    # paper-size frame, row width a multiple of 32
    (960, 540, 3, 4, 11, 2),    # reduced to 240x135: words straddle rows
    (320, 180, 1, 1, 3, -3),
    (97, 61, 3, 2, 13, 5),      # odd sizes, dropped partial blocks
    (5, 3, 3, 1, 13, 0),        # window wider than the frame, one word
    (1, 1, 1, 1, 3, 1),
    (4000, 50, 3, 1, 7, 2),     # wide: few rows per CTA
    (33, 700, 1, 1, 5, 1),      # narrow: every word crosses a row
    (1024, 64, 3, 8, 9, -1),
])
def test_encode_matches_oracle(W, H, ch, reduce, block, offset):
    n = 3
    frames = _frames(n, W, H, ch, seed=wl.BASE_SEED + 6 + W + H)
    e = spg.sp_encoder_create(spg.sp_encoder_config_init(src_w=W, src_h=H, channels=ch,
                                                         reduce=reduce, block=block,
                                                         offset=offset))
    try:
        info = spg.sp_encoder_get_info(e)
        assert (info["out_w"], info["out_h"]) == (W // reduce, H // reduce)
        fb = info["src_bytes"]
        src_stride = fb + 48
        src = np.zeros((n, src_stride), np.uint8)
        src[:, :fb] = frames.reshape(n, -1)
        words = info["out_words"]
        bstride = words + 5
        d_src = torch.from_numpy(src).cuda()
        d_bits = torch.full((n, bstride), SENTINEL - (1 << 32), dtype=torch.int32, device="cuda")
        spg.sp_encode_device(e, d_src, n, src_stride, d_bits, bstride,
                             torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = d_bits.cpu().numpy().view(np.uint32)
    finally:
        spg.sp_encoder_destroy(e)
    assert (got[:, words:] == SENTINEL).all(), "wrote past the encoded frame"
    n_bits = info["out_bits"]
    want = _oracle_bits(frames, reduce, block, offset)
    bits = _unpack(np.ascontiguousarray(got[:, :words]), words * 32)
    assert first_diff(bits[:, :n_bits], want) is None, first_diff(bits[:, :n_bits], want)
    assert not bits[:, n_bits:].any(), "unused high bits of the last word must be zero"


@pytest.mark.parametrize("reduce", [1, 4])
def test_encode_unaligned_source(reduce):
    """Frames starting at an odd byte address take the byte-load path."""
    n, W, H = 2, 256, 96
    frames = _frames(n, W, H, 3, seed=wl.BASE_SEED + 64)
    e = spg.sp_encoder_create(spg.sp_encoder_config_init(src_w=W, src_h=H, reduce=reduce))
    try:
        info = spg.sp_encoder_get_info(e)
        fb, words = info["src_bytes"], info["out_words"]
        buf = torch.zeros(n * fb + 1, dtype=torch.uint8, device="cuda")
        buf[1:] = torch.from_numpy(frames.reshape(-1)).cuda()
        d_bits = torch.zeros((n, words), dtype=torch.int32, device="cuda")
        spg.sp_encode_device(e, buf.data_ptr() + 1, n, fb, d_bits, words,
                             torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = _unpack(d_bits.cpu().numpy().view(np.uint32), info["out_bits"])
    finally:
        spg.sp_encoder_destroy(e)
    want = _oracle_bits(frames, reduce, 11, 2)
    assert first_diff(got, want) is None


def _encoded_case(Wr, Hr, C, S, seed):
    idx = synth.pool_uniform(synth.derive_seed(seed, synth.PURPOSE_POOL, 0), C, S, Wr * Hr)
    perm = synth.perm_uniform(synth.derive_seed(seed, synth.PURPOSE_PERM, 0), (C, S), 0.1, 0.3)
    return wl.Case("encoded", Wr, Hr, C, S, idx, perm, np.ones(C, np.float32), k=max(1, C // 50),
                   min_overlap=4)


@pytest.mark.parametrize("reduce,n", [(1, 40), (4, 70)])
def test_encode_then_sp_matches_oracle(reduce, n):
    """Encoder feeding the SP on the device: every frame's winners and the
    final permanences equal the oracle's encoder followed by its SP."""
    W, H = 960, 540
    frames = wl.rgb_frames(n, W, H, seed=wl.BASE_SEED + 60 + reduce)
    if reduce == 1:
        case = wl.frame_case()
    else:
        case = _encoded_case(W // reduce, H // reduce, 512, 64, wl.BASE_SEED + 61)
    e = spg.sp_encoder_create(spg.sp_encoder_config_init(reduce=reduce))
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    try:
        mw = spg.sp_get_info(h)["mask_words"]
        d_src = torch.from_numpy(frames.reshape(n, -1)).cuda()
        d_masks = torch.zeros((n, mw), dtype=torch.int32, device="cuda")
        spg.sp_encode_compute_device(e, h, d_src, n, d_src.shape[1], True, d_masks,
                                     torch.cuda.current_stream())
        spg.sp_sync(h)
        torch.cuda.synchronize()
        act = dense(d_masks.cpu().numpy().view(np.uint32), case.C)
        perm = spg.sp_get_permanences(h)
    finally:
        spg.sp_destroy(h)
        spg.sp_encoder_destroy(e)
    bits = _oracle_bits(frames, reduce, 11, 2)
    want, want_perm, _ = oracle_run(case, bits, True)
    assert first_diff(act, want) is None, first_diff(act, want)
    np.testing.assert_array_equal(perm, want_perm)


def test_encode_compute_from_host_frames():
    """sp_encode_compute: pinned host frames in, masks out, three chunks."""
    n = 70
    frames = wl.rgb_frames(n, 960, 540, seed=wl.BASE_SEED + 62)
    case = wl.frame_case(seed=wl.BASE_SEED + 63)
    e = spg.sp_encoder_create(spg.sp_encoder_config_init())
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    try:
        pinned = torch.from_numpy(frames).pin_memory()
        masks = np.zeros((n, spg.sp_get_info(h)["mask_words"]), np.uint32)
        spg.sp_encode_compute(e, h, pinned.numpy(), True, masks)
        perm = spg.sp_get_permanences(h)
    finally:
        spg.sp_destroy(h)
        spg.sp_encoder_destroy(e)
    want, want_perm, _ = oracle_run(case, _oracle_bits(frames, 1, 11, 2), True)
    got = dense(masks, case.C)
    assert first_diff(got, want) is None, first_diff(got, want)
    np.testing.assert_array_equal(perm, want_perm)


def test_encode_rejects_mismatched_sp_and_strides():
    e = spg.sp_encoder_create(spg.sp_encoder_config_init(reduce=2))
    case = wl.frame_case()
    h = spg.sp_create_from_state(case.config(), case.idx, case.perm, case.boost)
    try:
        d = torch.zeros(960 * 540 * 3, dtype=torch.uint8, device="cuda")
        with pytest.raises(spg.SpError) as ex:  # 480x270 bits into a 960x540 SP
            spg.sp_encode_compute_device(e, h, d, 1, d.numel(), False)
        assert ex.value.status == 1
        bits = torch.zeros(8192, dtype=torch.int32, device="cuda")
        with pytest.raises(spg.SpError):
            spg.sp_encode_device(e, d, 1, 100, bits, 8192)  # source stride too short
        with pytest.raises(spg.SpError):
            spg.sp_encode_device(e, d, 1, d.numel(), bits, 10)  # bit stride too short
    finally:
        spg.sp_destroy(h)
        spg.sp_encoder_destroy(e)
