"""Seeded SP workloads: the inputs of the tests, smoke() and the benchmark.

Only input generation lives here (pools, permanences, frames via the synth
module): no SP arithmetic.  Recipes follow the five workloads of the build:
  small     32x32 Bernoulli(0.10) input, 256 columns x 16 uniform synapses,
            perms U[0.1,0.3], threshold 0.2, min_overlap 4, k 10 global;
  frame     960x540 blobbed frames (density U[5%,20%], 7x7 box blur), 1024
            columns on a 32x32 grid of receptive-field centres, 256 synapses
            from a 64x64 window, perms U[0.1,0.3], threshold 0.2,
            min_overlap 4, k 40 global, inc 0.05 / dec 0.02;
  sweep     the frame input with columns {256,1024,4096} (square grids) x
            synapses {16,64,256} x min_overlap {2,4,8} x k {8,32,128} x
            global / 9x9 local inhibition;
  video     960x540 colour frames (blobs under an illumination ramp) for
            the frame encoder, whose output feeds a frame-shaped SP.
"""
import dataclasses

import numpy as np

from . import synth

BASE_SEED = 0x5EED0000


@dataclasses.dataclass
class Case:
    name: str
    W: int
    H: int
    C: int
    S: int
    idx: np.ndarray
    perm: np.ndarray
    boost: np.ndarray
    thr: float = 0.2
    inc: float = 0.05
    dec: float = 0.02
    min_overlap: int = 4
    k: int = 10
    inhibition: int = 0
    gw: int = 0
    gh: int = 0
    radius: int = 0

    @property
    def n_in(self):
        return self.W * self.H

    @property
    def n_words(self):
        return (self.n_in + 31) // 32

    def config(self, **extra):
        from ._binding import sp_config_init
        return sp_config_init(input_w=self.W, input_h=self.H, num_columns=self.C,
                              col_grid_w=self.gw, col_grid_h=self.gh,
                              synapses_per_column=self.S, connect_threshold=self.thr,
                              perm_inc=self.inc, perm_dec=self.dec,
                              min_overlap=self.min_overlap, winners_set_size=self.k,
                              inhibition=self.inhibition, local_radius=self.radius, **extra)


def small_case(seed=BASE_SEED + 1):
    C, S, n = 256, 16, 1024
    idx = synth.pool_uniform(synth.derive_seed(seed, synth.PURPOSE_POOL, 0), C, S, n)
    perm = synth.perm_uniform(synth.derive_seed(seed, synth.PURPOSE_PERM, 0), (C, S), 0.1, 0.3)
    return Case("small", 32, 32, C, S, idx, perm, np.ones(C, np.float32), k=10)


def small_frames(n, seed=BASE_SEED + 1, start=0):
    return np.stack([synth.frame_bernoulli(synth.derive_seed(seed, synth.PURPOSE_FRAME, t),
                                           1024, 0.10) for t in range(start, start + n)])


def grid_case(name, C, S, seed, W=960, H=540, rf=64, min_overlap=4, k=40, inhibition=0,
              radius=4, thr=0.2, lo=0.1, hi=0.3):
    g = int(round(C ** 0.5))
    assert g * g == C
    idx = synth.pool_window(synth.derive_seed(seed, synth.PURPOSE_POOL, 0), g, g, W, H, rf, rf, S)
    perm = synth.perm_uniform(synth.derive_seed(seed, synth.PURPOSE_PERM, 0), (C, S), lo, hi)
    return Case(name, W, H, C, S, idx, perm, np.ones(C, np.float32), thr=thr,
                min_overlap=min_overlap, k=k, inhibition=inhibition, gw=g, gh=g,
                radius=radius if inhibition else 0)


def frame_case(seed=BASE_SEED + 2):
    return grid_case("frame", 1024, 256, seed)


def blob_frames(n, W=960, H=540, seed=BASE_SEED + 2, start=0):
    return np.stack([synth.frame_blobbed(synth.derive_seed(seed, synth.PURPOSE_FRAME, t), W, H)
                     for t in range(start, start + n)])


def rgb_frames(n, W=960, H=540, seed=BASE_SEED + 6, start=0):
    """Colour frames uint8 [n, H, W, 3] (R, G, B)."""
    return np.stack([synth.frame_rgb(synth.derive_seed(seed, synth.PURPOSE_FRAME, t), W, H)
                     for t in range(start, start + n)])


def pack(frames):
    return synth.pack_frames(frames)


def uneven_cases(n, seed=BASE_SEED + 4, c_range=(128, 4096), s_range=(16, 256),
                 n_in_range=(256, 16384)):
    """Independent SPs of uneven shapes: columns, synapses per column and input
    bits drawn uniformly (integers) from the ranges, uniform pools,
    perms U[0.1,0.3], threshold 0.2, min_overlap 4, global inhibition with
    k = 2% of the columns rounded half up (at least 1).  Returns (cases,
    densities): each SP's input density is drawn from U[2%, 20%]."""
    cases, dens = [], []
    for i in range(n):
        st = synth.derive_seed(seed, synth.PURPOSE_SHAPE, i)
        r, st2 = synth.splitmix64(st, 4)
        C = c_range[0] + r[0] % (c_range[1] - c_range[0] + 1)
        n_in = n_in_range[0] + r[2] % (n_in_range[1] - n_in_range[0] + 1)
        S = min(s_range[0] + r[1] % (s_range[1] - s_range[0] + 1), n_in)
        p = 0.02 + 0.18 * ((r[3] >> 11) / float(1 << 53))
        k = max(1, (2 * C + 50) // 100)
        inst = synth.derive_seed(seed, synth.PURPOSE_INSTANCE, i)
        idx = synth.pool_uniform(synth.derive_seed(inst, synth.PURPOSE_POOL, 0), C, S, n_in)
        perm = synth.perm_uniform(synth.derive_seed(inst, synth.PURPOSE_PERM, 0), (C, S), 0.1, 0.3)
        cases.append(Case(f"uneven{i}", n_in, 1, C, S, idx, perm, np.ones(C, np.float32), k=k,
                          min_overlap=4))
        dens.append(p)
    return cases, dens


def bernoulli_frames(case_index, n_in, p, n, seed=BASE_SEED + 4, start=0):
    inst = synth.derive_seed(seed, synth.PURPOSE_INSTANCE, case_index)
    return np.stack([synth.frame_bernoulli(synth.derive_seed(inst, synth.PURPOSE_FRAME, t), n_in, p)
                     for t in range(start, start + n)])


def uneven_frames(cases, dens, n, seed=BASE_SEED + 4, start=0):
    """Frames of the uneven SPs: member i sees Bernoulli(dens[i]) frames drawn
    from its own instance seed."""
    return [bernoulli_frames(i, c.n_in, dens[i], n, seed=seed, start=start)
            for i, c in enumerate(cases)]


def dense_cases(members=16, frames=256, C=1024, n_in=1024, k=20, seed=BASE_SEED + 4):
    """SPs with dense potential pools (every column sees the whole input,
    S = n_in) for the tensor-core path: perms U[0.1,0.3], threshold 0.2,
    min_overlap 4, global inhibition with k winners; member i's frames are
    Bernoulli(p_i) with p_i spread evenly over [2%, 20%].  Returns (cases,
    frames uint8 [members][frames][n_in])."""
    cases, fr = [], []
    for i in range(members):
        sd = synth.derive_seed(seed, synth.PURPOSE_INSTANCE, 1000 + i)
        idx = synth.pool_dense(C, n_in)
        perm = synth.perm_uniform(synth.derive_seed(sd, synth.PURPOSE_PERM, 0), (C, n_in),
                                  0.1, 0.3)
        cases.append(Case(f"dense{i}", n_in, 1, C, n_in, idx, perm, np.ones(C, np.float32), k=k))
        p = 0.02 + 0.18 * i / max(1, members - 1)
        fr.append(np.stack([synth.frame_bernoulli(synth.derive_seed(sd, synth.PURPOSE_FRAME, t),
                                                  n_in, p) for t in range(frames)]))
    return cases, fr


SERVE_RESOLUTIONS = ((320, 180), (640, 360), (960, 540))


def serve_cases(streams=32, seed=BASE_SEED + 5):
    """The serving workload's streams: stream i at resolution i mod 3 of
    320x180 / 640x360 / 960x540, each with its own SP of 1024 columns on a
    32x32 grid x 256 synapses from 64x64 windows (k 40, min_overlap 4)."""
    cases = []
    for i in range(streams):
        W, H = SERVE_RESOLUTIONS[i % 3]
        cases.append(grid_case(f"stream{i}", 1024, 256, synth.derive_seed(seed, synth.PURPOSE_INSTANCE, i),
                               W=W, H=H))
    return cases


def serve_frames(case_index, W, H, n, seed=BASE_SEED + 5, start=0):
    """Blobbed frames of serving stream case_index."""
    return blob_frames(n, W=W, H=H, seed=synth.derive_seed(seed, synth.PURPOSE_FRAME, case_index),
                       start=start)


def batch_frames(per_member_packed, frame_off, frame_words):
    """Assemble batch frames: per_member_packed[i] is uint32 [n][words_i];
    returns uint32 [n][frame_words] with member i at word offset frame_off[i]."""
    n = per_member_packed[0].shape[0]
    out = np.zeros((n, frame_words), np.uint32)
    for i, pk in enumerate(per_member_packed):
        o = int(frame_off[i])
        out[:, o:o + pk.shape[1]] = pk
    return out
