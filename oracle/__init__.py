"""ctypes access to the plain CPU oracle of the Spatial Pooler hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the library package.  All arrays are
numpy; the oracle takes one byte per input bit (nonzero = 1) and returns one
byte per column for the active set.
"""
import ctypes as ct

import numpy as np

from .build import build as _build

_lib = None


class OrcParams(ct.Structure):
    _fields_ = [
        ("C", ct.c_uint32), ("S", ct.c_uint32), ("n_in", ct.c_uint64),
        ("connect_threshold", ct.c_float), ("perm_inc", ct.c_float),
        ("perm_dec", ct.c_float), ("min_overlap", ct.c_uint32),
        ("winners_set_size", ct.c_uint32), ("inhibition", ct.c_uint32),
        ("col_grid_w", ct.c_uint32), ("col_grid_h", ct.c_uint32),
        ("local_radius", ct.c_uint32),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(_build())
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ct.POINTER(ctype))


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid argument")


def params(C, S, n_in, thr=0.2, inc=0.05, dec=0.02, min_overlap=4, k=10,
           inhibition=0, grid_w=0, grid_h=0, radius=0):
    return OrcParams(C, S, n_in, thr, inc, dec, min_overlap, k, inhibition,
                     grid_w, grid_h, radius)


def overlap(idx, perm, boost, x, thr, min_overlap):
    """Alg. 1: returns (raw int32 [C], ov float32 [C])."""
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    perm = np.ascontiguousarray(perm, dtype=np.float32)
    C, S = idx.shape
    boost = np.ascontiguousarray(boost, dtype=np.float32)
    x = _u8(x)
    raw = np.zeros(C, np.int32)
    ov = np.zeros(C, np.float32)
    rc = lib().orc_overlap(ct.c_uint32(C), ct.c_uint32(S), _p(idx, ct.c_uint32),
                           _p(perm, ct.c_float), _p(boost, ct.c_float),
                           ct.c_uint64(x.size), _p(x, ct.c_uint8), ct.c_float(thr),
                           ct.c_uint32(min_overlap), _p(raw, ct.c_int32),
                           _p(ov, ct.c_float))
    _check(rc, "overlap")
    return raw, ov


def inhibit_global(ov, k):
    ov = np.ascontiguousarray(ov, dtype=np.float32)
    act = np.zeros(ov.size, np.uint8)
    _check(lib().orc_inhibit_global(ct.c_uint32(ov.size), _p(ov, ct.c_float),
                                    ct.c_uint32(k), _p(act, ct.c_uint8)), "inhibit_global")
    return act


def inhibit_local(ov, gw, gh, k, r):
    ov = np.ascontiguousarray(ov, dtype=np.float32)
    act = np.zeros(ov.size, np.uint8)
    _check(lib().orc_inhibit_local(ct.c_uint32(gw), ct.c_uint32(gh), _p(ov, ct.c_float),
                                   ct.c_uint32(k), ct.c_uint32(r), _p(act, ct.c_uint8)),
           "inhibit_local")
    return act


def inhibit_paper_literal(ov, k):
    ov = np.ascontiguousarray(ov, dtype=np.float32)
    act = np.zeros(ov.size, np.uint8)
    _check(lib().orc_inhibit_paper_literal(ct.c_uint32(ov.size), _p(ov, ct.c_float),
                                           ct.c_uint32(k), _p(act, ct.c_uint8)),
           "inhibit_paper_literal")
    return act


def learn(idx, perm, x, active, inc, dec):
    """Learning in place on perm (float32 [C][S]); returns perm."""
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    assert perm.dtype == np.float32 and perm.flags.c_contiguous
    C, S = idx.shape
    x = _u8(x)
    active = _u8(active)
    _check(lib().orc_learn(ct.c_uint32(C), ct.c_uint32(S), _p(idx, ct.c_uint32),
                           _p(perm, ct.c_float), ct.c_uint64(x.size), _p(x, ct.c_uint8),
                           _p(active, ct.c_uint8), ct.c_float(inc), ct.c_float(dec)),
           "learn")
    return perm


def run(p, idx, perm, boost, frames, learn_flag, want_ov=False):
    """n frames in sequence (frames uint8 [n][n_in]); perm updated in place.
    Returns active uint8 [n][C] (and ov float32 [n][C] when want_ov)."""
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    assert perm.dtype == np.float32 and perm.flags.c_contiguous
    boost = np.ascontiguousarray(boost, dtype=np.float32)
    frames = _u8(frames)
    n = frames.shape[0]
    act = np.zeros((n, p.C), np.uint8)
    ov = np.zeros((n, p.C), np.float32) if want_ov else None
    rc = lib().orc_run(ct.byref(p), _p(idx, ct.c_uint32), _p(perm, ct.c_float),
                       _p(boost, ct.c_float), _p(frames, ct.c_uint8), ct.c_uint32(n),
                       ct.c_int(1 if learn_flag else 0), _p(act, ct.c_uint8),
                       _p(ov, ct.c_float) if want_ov else None)
    _check(rc, "run")
    return (act, ov) if want_ov else act


def duty_update(duty, active, period):
    assert duty.dtype == np.float32 and duty.flags.c_contiguous
    active = _u8(active)
    _check(lib().orc_duty_update(ct.c_uint32(duty.size), _p(duty, ct.c_float),
                                 _p(active, ct.c_uint8), ct.c_float(period)), "duty_update")
    return duty


def encode(src, reduce=1, block=11, offset=2):
    """Frame encoder: src uint8 [H, W] (gray) or [H, W, 3] (R, G, B).
    Returns the binary image uint8 [H // reduce, W // reduce] (0/1)."""
    src = np.ascontiguousarray(src, dtype=np.uint8)
    H, W = src.shape[:2]
    ch = 1 if src.ndim == 2 else src.shape[2]
    if reduce < 1:
        raise ValueError("oracle encode: invalid argument")
    out = np.zeros((H // reduce, W // reduce), np.uint8)
    _check(lib().orc_encode(_p(src, ct.c_uint8), ct.c_uint32(W), ct.c_uint32(H),
                            ct.c_uint32(ch), ct.c_uint32(reduce), ct.c_uint32(block),
                            ct.c_int32(offset), _p(out, ct.c_uint8)), "encode")
    return out
