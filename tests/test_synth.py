"""Seeded input generators (include/sp_synth.h): published SplitMix64 vectors,
pool/permanence/frame recipes and the bit packing used by the library."""
import numpy as np

from paper_1608_01966_gb300 import synth


def test_splitmix64_published_vectors():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 0: the first outputs are
    # the widely published test vectors of the reference implementation.
    out, _ = synth.splitmix64(0, 3)
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_derive_seed_distinct_and_stable():
    a = [synth.derive_seed(7, p, i) for p in (1, 2, 3) for i in range(50)]
    assert len(set(a)) == len(a)
    assert synth.derive_seed(7, 3, 5) == synth.derive_seed(7, 3, 5)


def test_pool_uniform_sorted_distinct_in_range():
    idx = synth.pool_uniform(11, 64, 16, 1024)
    assert idx.shape == (64, 16)
    assert (np.diff(idx.astype(np.int64), axis=1) > 0).all()
    assert idx.max() < 1024
    # every input index reachable: over many columns the coverage is wide
    big = synth.pool_uniform(12, 2048, 16, 1024)
    assert np.unique(big).size > 1000
    np.testing.assert_array_equal(idx, synth.pool_uniform(11, 64, 16, 1024))


def test_pool_uniform_full_pool_is_identity():
    idx = synth.pool_uniform(3, 5, 32, 32)
    np.testing.assert_array_equal(idx, np.tile(np.arange(32, dtype=np.uint32), (5, 1)))


def test_pool_window_inside_clipped_window():
    gw, gh, W, H, rf = 32, 32, 960, 540, 64
    idx = synth.pool_window(5, gw, gh, W, H, rf, rf, 256)
    ys, xs = idx // W, idx % W
    for j in range(gh):
        cy = ((2 * j + 1) * H) // (2 * gh)
        y0 = min(max(cy - rf // 2, 0), H - rf)
        for i in range(gw):
            cx = ((2 * i + 1) * W) // (2 * gw)
            x0 = min(max(cx - rf // 2, 0), W - rf)
            c = j * gw + i
            assert ys[c].min() >= y0 and ys[c].max() < y0 + rf
            assert xs[c].min() >= x0 and xs[c].max() < x0 + rf
            assert np.unique(idx[c]).size == 256
    # first column's window is flush with the frame corner
    assert xs[0].min() >= 0 and ys[0].min() >= 0


def test_pool_dense():
    idx = synth.pool_dense(3, 40)
    np.testing.assert_array_equal(idx[2], np.arange(40))


def test_perm_uniform_range_and_constant():
    p = synth.perm_uniform(9, (1000,), 0.1, 0.3)
    assert p.dtype == np.float32
    assert p.min() >= np.float32(0.1) and p.max() <= np.float32(0.3)
    assert abs(float(p.mean()) - 0.2) < 0.01
    c = synth.perm_uniform(9, (10,), 0.21, 0.21)
    assert (c == np.float32(0.21)).all()


def test_pack_bits_matches_numpy_little_endian():
    rng = np.random.default_rng(0)
    for n in (1, 31, 32, 33, 100, 1024, 518400):
        bits = (rng.random(n) < 0.3).astype(np.uint8)
        w = synth.pack_bits(bits)
        ref = np.packbits(np.pad(bits, (0, (-n) % 32)), bitorder="little").view("<u4")
        np.testing.assert_array_equal(w, ref)


def test_frame_bernoulli_density():
    f = synth.frame_bernoulli(1, 100000, 0.1)
    assert abs(f.mean() - 0.1) < 0.005
    np.testing.assert_array_equal(f, synth.frame_bernoulli(1, 100000, 0.1))


def test_frame_blobbed_density_and_threshold_rule():
    for s in range(4):
        f, p = synth.frame_blobbed(synth.derive_seed(1, 3, s), 320, 180, return_p=True)
        assert 0.05 <= p <= 0.20
        # the threshold keeps at most a fraction p of the pixels
        assert f.mean() <= p + 1e-12
        assert f.mean() > 0.25 * p
        # blobbed: active pixels have many active 4-neighbours (spatial structure)
        img = f.reshape(180, 320).astype(np.int32)
        nb = img[1:-1, :-2] + img[1:-1, 2:] + img[:-2, 1:-1] + img[2:, 1:-1]
        assert nb[img[1:-1, 1:-1] == 1].mean() > 2.0
