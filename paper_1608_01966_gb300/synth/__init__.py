"""Seeded synthetic inputs (pools, permanences, binary frames) via ctypes.

Thin wrapper over libsp_synth.so (include/sp_synth.h).  Holds none of the
SP's arithmetic; used by the tests and the benchmark to draw the same inputs
for the CUDA library and for the CPU oracle.
"""
import ctypes as ct

import numpy as np

PURPOSE_POOL = 1
PURPOSE_PERM = 2
PURPOSE_FRAME = 3
PURPOSE_INSTANCE = 4
PURPOSE_SHAPE = 5

_lib = None


def lib():
    global _lib
    if _lib is None:
        from .. import build as _b
        _lib = ct.CDLL(_b.build_synth())
        _lib.synth_splitmix64.restype = ct.c_uint64
        _lib.synth_derive_seed.restype = ct.c_uint64
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


def _ok(rc, what):
    if rc != 0:
        raise ValueError(f"synth {what}: invalid argument")


def splitmix64(state: int, n: int):
    """n successive SplitMix64 outputs from `state`; returns (list, new_state)."""
    st = ct.c_uint64(state)
    out = [lib().synth_splitmix64(ct.byref(st)) for _ in range(n)]
    return out, st.value


def derive_seed(base: int, purpose: int, index: int) -> int:
    return lib().synth_derive_seed(ct.c_uint64(base), ct.c_uint64(purpose), ct.c_uint64(index))


def pool_uniform(seed, C, S, n_in):
    out = np.empty((C, S), np.uint32)
    scratch = np.empty(n_in, np.uint32)
    _ok(lib().synth_pool_uniform(ct.c_uint64(seed), ct.c_uint32(C), ct.c_uint32(S),
                                 ct.c_uint32(n_in), _p(out, ct.c_uint32),
                                 _p(scratch, ct.c_uint32)), "pool_uniform")
    return out


def pool_window(seed, gw, gh, W, H, rf_w, rf_h, S):
    out = np.empty((gw * gh, S), np.uint32)
    scratch = np.empty(rf_w * rf_h, np.uint32)
    _ok(lib().synth_pool_window(ct.c_uint64(seed), ct.c_uint32(gw), ct.c_uint32(gh),
                                ct.c_uint32(W), ct.c_uint32(H), ct.c_uint32(rf_w),
                                ct.c_uint32(rf_h), ct.c_uint32(S), _p(out, ct.c_uint32),
                                _p(scratch, ct.c_uint32)), "pool_window")
    return out


def pool_dense(C, n_in):
    out = np.empty((C, n_in), np.uint32)
    _ok(lib().synth_pool_dense(ct.c_uint32(C), ct.c_uint32(n_in), _p(out, ct.c_uint32)),
        "pool_dense")
    return out


def perm_uniform(seed, shape, lo, hi):
    out = np.empty(shape, np.float32)
    _ok(lib().synth_perm_uniform(ct.c_uint64(seed), ct.c_uint64(out.size), ct.c_float(lo),
                                 ct.c_float(hi), _p(out, ct.c_float)), "perm_uniform")
    return out


def frame_bernoulli(seed, n, p):
    out = np.empty(n, np.uint8)
    _ok(lib().synth_frame_bernoulli(ct.c_uint64(seed), ct.c_uint64(n), ct.c_double(p),
                                    _p(out, ct.c_uint8)), "frame_bernoulli")
    return out


def frame_blobbed(seed, W, H, p_lo=0.05, p_hi=0.20, return_p=False):
    out = np.empty(W * H, np.uint8)
    scratch = np.empty(2 * W * H, np.uint8)
    p = ct.c_double(0.0)
    _ok(lib().synth_frame_blobbed(ct.c_uint64(seed), ct.c_uint32(W), ct.c_uint32(H),
                                  ct.c_double(p_lo), ct.c_double(p_hi), _p(out, ct.c_uint8),
                                  _p(scratch, ct.c_uint8), ct.byref(p)), "frame_blobbed")
    return (out, p.value) if return_p else out


def frame_rgb(seed, W, H):
    """Colour frame [H, W, 3] uint8 (R, G, B): blobs under an illumination ramp."""
    out = np.empty((H, W, 3), np.uint8)
    scratch = np.empty(2 * W * H, np.uint8)
    _ok(lib().synth_frame_rgb(ct.c_uint64(seed), ct.c_uint32(W), ct.c_uint32(H),
                              _p(out, ct.c_uint8), _p(scratch, ct.c_uint8)), "frame_rgb")
    return out


def pack_bits(bits):
    bits = np.ascontiguousarray(bits, dtype=np.uint8).ravel()
    out = np.empty((bits.size + 31) // 32, np.uint32)
    _ok(lib().synth_pack_bits(_p(bits, ct.c_uint8), ct.c_uint64(bits.size),
                              _p(out, ct.c_uint32)), "pack_bits")
    return out


def pack_frames(frames):
    """uint8 [n][n_in] -> uint32 [n][ceil(n_in/32)] packed words."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    return np.stack([pack_bits(f) for f in frames]) if frames.shape[0] else \
        np.zeros((0, (frames.shape[1] + 31) // 32), np.uint32)
