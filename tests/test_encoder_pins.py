"""Pins of the oracle's frame encoder (Section 2 and "Adaptive Video Encoder"
in Section 3.1: reduction, grayscale, adaptive Gaussian threshold).

The paper names OpenCV's Gaussian adaptive threshold and gives no further
arithmetic, so the encoder is defined exactly in integers (binomial weights,
edge replication, rounded local mean; see the oracle's header).  The pins
here do not re-type that definition: the threshold is checked against
scipy's n-dimensional correlation with math.comb weights, the grayscale and
reduction steps against identities and orderings that any mistake in
channel order, rounding or block indexing breaks.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01966_gb300 import synth

scipy_ndimage = pytest.importorskip("scipy.ndimage")


def _threshold_by_scipy(gray, block, offset):
    w = np.array([math.comb(block - 1, i) for i in range(block)], np.float64)
    total = float(4 ** (block - 1))
    s = scipy_ndimage.correlate(gray.astype(np.float64), np.outer(w, w), mode="nearest")
    mean = np.floor(s / total + 0.5)  # exact: s < 2^53, total a power of two
    return (gray.astype(np.int64) > mean.astype(np.int64) - offset).astype(np.uint8)


@pytest.mark.parametrize("shape", [(1, 1), (3, 200), (200, 3), (37, 23), (64, 96)])
@pytest.mark.parametrize("block", [3, 5, 11, 13])
def test_threshold_is_gaussian_correlation_with_edge_replication(shape, block):
    rng = np.random.default_rng(block * 1000 + shape[0] * 7 + shape[1])
    gray = rng.integers(0, 256, size=shape, dtype=np.uint8)
    for offset in (-3, 0, 2, 7):
        got = oracle.encode(gray, 1, block, offset)
        np.testing.assert_array_equal(got, _threshold_by_scipy(gray, block, offset),
                                      err_msg=f"block {block} offset {offset}")


def test_threshold_on_smooth_frames_matches_scipy():
    rgb = synth.frame_rgb(synth.derive_seed(0x5EED0006, synth.PURPOSE_FRAME, 0), 160, 90)
    gray = rgb[:, :, 0]  # any 8-bit image; one channel is its own gray
    for block, offset in ((11, 2), (7, -1)):
        np.testing.assert_array_equal(oracle.encode(gray, 1, block, offset),
                                      _threshold_by_scipy(gray, block, offset))


@pytest.mark.parametrize("value", [0, 1, 77, 128, 254, 255])
def test_constant_image_mean_is_the_value(value):
    img = np.full((9, 14), value, np.uint8)
    for offset in (-2, 0, 1, 5):
        assert (oracle.encode(img, 1, 5, offset) == (1 if offset > 0 else 0)).all()
    rgb = np.full((9, 14, 3), value, np.uint8)  # gray pixels keep their value
    for offset in (0, 1):
        assert (oracle.encode(rgb, 1, 5, offset) == (1 if offset > 0 else 0)).all()


def test_gray_rgb_equals_single_channel():
    """R = G = B = v has luma exactly v (weights sum to 256, rounded)."""
    rng = np.random.default_rng(5)
    g = rng.integers(0, 256, size=(31, 45), dtype=np.uint8)
    rgb = np.repeat(g[:, :, None], 3, axis=2)
    for block, offset in ((3, 0), (11, 2), (13, -4)):
        np.testing.assert_array_equal(oracle.encode(rgb, 1, block, offset),
                                      oracle.encode(g, 1, block, offset))


def test_channel_order_and_luma_ordering():
    """Green outweighs red outweighs blue: at a boundary between two pure
    colours the brighter side's edge pixels are above their local mean and
    the darker side's below (a swap of R and B reverses the red/blue case)."""
    for top, bottom in (((255, 0, 0), (0, 0, 255)), ((0, 255, 0), (255, 0, 0)),
                        ((0, 255, 0), (0, 0, 255))):
        img = np.zeros((20, 8, 3), np.uint8)
        img[:10] = top
        img[10:] = bottom
        bits = oracle.encode(img, 1, 5, 0)
        assert bits[9].all() and not bits[10].any(), (top, bottom)
        assert not bits[0].any() and not bits[19].any()  # flat regions: g == mean


@pytest.mark.parametrize("colour,luma", [((255, 0, 0), 77), ((0, 255, 0), 149), ((0, 0, 255), 29),
                                         ((255, 255, 255), 255), ((0, 0, 0), 0)])
def test_luma_of_pure_colours(colour, luma):
    """One pixel of a pure colour on a gray background v (3 x 3 window,
    offset 0): its local mean is round(v + (L - v)/4), so it is above the
    mean for v = L - 1 and not for v = L exactly when its luma is L.
    255 x 77/256 = 76.7 rounds to 77, 255 x 150/256 = 149.4 to 149,
    255 x 29/256 = 28.9 to 29."""
    def centre_bit(v):
        img = np.full((5, 5, 3), v, np.uint8)
        img[2, 2] = colour
        return int(oracle.encode(img, 1, 3, 0)[2, 2])
    assert centre_bit(luma) == 0
    if luma > 0:
        assert centre_bit(luma - 1) == 1


def test_reduction_of_block_constant_image_is_the_small_image():
    rng = np.random.default_rng(11)
    for f in (2, 3, 4):
        small = rng.integers(0, 256, size=(12, 17, 3), dtype=np.uint8)
        big = np.repeat(np.repeat(small, f, axis=0), f, axis=1)
        np.testing.assert_array_equal(oracle.encode(big, f, 5, 2), oracle.encode(small, 1, 5, 2))


def test_reduction_rounds_half_up_and_drops_partial_blocks():
    rng = np.random.default_rng(12)
    v = rng.integers(0, 255, size=(10, 10), dtype=np.uint8)
    half = np.zeros((20, 20), np.uint8)  # each 2x2 block: v, v, v+1, v+1 (mean v + 1/2)
    half[0::2, :] = np.repeat(v, 2, axis=1)
    half[1::2, :] = np.repeat(v + 1, 2, axis=1)
    np.testing.assert_array_equal(oracle.encode(half, 2, 3, 1), oracle.encode(v + 1, 1, 3, 1))
    quarter = np.repeat(np.repeat(v, 2, axis=0), 2, axis=1)  # mean v + 1/4
    quarter[0::2, 0::2] += 1
    np.testing.assert_array_equal(oracle.encode(quarter, 2, 3, 1), oracle.encode(v, 1, 3, 1))
    # 21 x 23 with f = 2: the last row and column do not form a block
    odd = rng.integers(0, 256, size=(21, 23, 3), dtype=np.uint8)
    assert oracle.encode(odd, 2, 5, 2).shape == (10, 11)
    np.testing.assert_array_equal(oracle.encode(odd, 2, 5, 2), oracle.encode(odd[:20, :22], 2, 5, 2))


@pytest.mark.parametrize("bad", [dict(block=1), dict(block=4), dict(block=15), dict(reduce=0),
                                 dict(reduce=8)])
def test_encode_rejects_bad_parameters(bad):
    img = np.zeros((6, 6), np.uint8)
    kw = dict(reduce=1, block=3, offset=0)
    kw.update(bad)
    with pytest.raises(ValueError):
        oracle.encode(img, **kw)
