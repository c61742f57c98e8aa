"""ctypes binding of include/sp.h (libsp_gb300.so), same names as the C ABI.

Argument marshalling only: every step of the Spatial Pooler runs in the CUDA
library.  Host arrays are numpy; device buffers are passed as integer
addresses or as anything with ``data_ptr()`` (a torch CUDA tensor), streams as
integer ``cudaStream_t`` handles or torch streams.  A failing call raises
SpError carrying the status and the library's message.  There is no fallback:
if the library cannot be built or loaded, every call raises.
"""
import ctypes as ct
import os

import numpy as np

SP_ABI_VERSION = 2
SP_MAX_COLUMNS = 16384
SP_POOL_UNIFORM, SP_POOL_WINDOW, SP_POOL_DENSE = 0, 1, 2
SP_INHIBIT_GLOBAL, SP_INHIBIT_LOCAL, SP_INHIBIT_PAPER_LITERAL = 0, 1, 2
STATUS = {0: "SP_OK", 1: "SP_EINVAL", 2: "SP_ENOMEM", 3: "SP_ECUDA", 4: "SP_ETIMEOUT",
          5: "SP_EBUSY", 6: "SP_ENOTSUP"}


class SpError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class SpConfig(ct.Structure):
    _fields_ = [
        ("abi_version", ct.c_uint32), ("input_w", ct.c_uint32), ("input_h", ct.c_uint32),
        ("num_columns", ct.c_uint32), ("col_grid_w", ct.c_uint32), ("col_grid_h", ct.c_uint32),
        ("synapses_per_column", ct.c_uint32), ("pool_mode", ct.c_uint32),
        ("rf_w", ct.c_uint32), ("rf_h", ct.c_uint32), ("connect_threshold", ct.c_float),
        ("perm_inc", ct.c_float), ("perm_dec", ct.c_float), ("perm_init_lo", ct.c_float),
        ("perm_init_hi", ct.c_float), ("min_overlap", ct.c_uint32),
        ("winners_set_size", ct.c_uint32), ("inhibition", ct.c_uint32),
        ("local_radius", ct.c_uint32), ("seed", ct.c_uint64),
        ("duty_period", ct.c_float), ("reserved", ct.c_uint32),
    ]


class SpBatchInfo(ct.Structure):
    _fields_ = [("members", ct.c_uint32), ("ctas", ct.c_uint32), ("frame_words", ct.c_uint64),
                ("mask_words", ct.c_uint64), ("frames", ct.c_uint64)]


class SpServerConfig(ct.Structure):
    _fields_ = [("abi_version", ct.c_uint32), ("max_streams", ct.c_uint32),
                ("queue_depth", ct.c_uint32), ("max_input_words", ct.c_uint32),
                ("device_budget_bytes", ct.c_uint64), ("max_active", ct.c_uint32),
                ("reserved", ct.c_uint32)]


class SpServerResult(ct.Structure):
    _fields_ = [("request_id", ct.c_uint64), ("frame_seq", ct.c_uint64),
                ("stream_id", ct.c_uint32), ("n_active", ct.c_uint32),
                ("active_offset", ct.c_uint32), ("status", ct.c_int),
                ("latency_us", ct.c_double)]


class SpServerStats(ct.Structure):
    _fields_ = [("submitted", ct.c_uint64), ("completed", ct.c_uint64),
                ("launches", ct.c_uint64), ("frames_in_launches", ct.c_uint64),
                ("device_bytes_used", ct.c_uint64), ("open_streams", ct.c_uint32),
                ("reserved", ct.c_uint32), ("p50_us", ct.c_double), ("p99_us", ct.c_double)]


class SpLoadgenConfig(ct.Structure):
    _fields_ = [("n_streams", ct.c_uint32), ("stream_ids", ct.POINTER(ct.c_uint32)),
                ("pools", ct.POINTER(ct.c_void_p)), ("pool_frames", ct.POINTER(ct.c_uint32)),
                ("pool_stride_words", ct.POINTER(ct.c_uint64)),
                ("rate_per_stream", ct.c_double), ("seconds", ct.c_double),
                ("producers", ct.c_uint32), ("learn", ct.c_uint32), ("seed", ct.c_uint64)]


class SpLoadgenReport(ct.Structure):
    _fields_ = [("offered", ct.c_uint64), ("submitted", ct.c_uint64), ("refused", ct.c_uint64),
                ("completed", ct.c_uint64), ("errors", ct.c_uint64), ("launches", ct.c_uint64),
                ("seconds", ct.c_double), ("offered_per_s", ct.c_double),
                ("frames_per_s", ct.c_double), ("p50_us", ct.c_double), ("p90_us", ct.c_double),
                ("p99_us", ct.c_double), ("p999_us", ct.c_double), ("max_us", ct.c_double),
                ("frames_per_launch", ct.c_double)]


class SpInfo(ct.Structure):
    _fields_ = [
        ("num_columns", ct.c_uint32), ("synapses_per_column", ct.c_uint32),
        ("input_bits", ct.c_uint64), ("input_words", ct.c_uint32), ("mask_words", ct.c_uint32),
        ("max_active", ct.c_uint32), ("device", ct.c_int), ("device_bytes", ct.c_uint64),
        ("frames", ct.c_uint64),
    ]


class SpEncoderConfig(ct.Structure):
    _fields_ = [
        ("src_w", ct.c_uint32), ("src_h", ct.c_uint32), ("channels", ct.c_uint32),
        ("reduce", ct.c_uint32), ("block", ct.c_uint32), ("offset", ct.c_int32),
        ("reserved", ct.c_uint32 * 2),
    ]


class SpEncoderInfo(ct.Structure):
    _fields_ = [
        ("out_w", ct.c_uint32), ("out_h", ct.c_uint32), ("out_bits", ct.c_uint64),
        ("out_words", ct.c_uint32), ("src_bytes", ct.c_uint64),
    ]


_lib = None
_u32p = ct.POINTER(ct.c_uint32)
_f32p = ct.POINTER(ct.c_float)


def lib():
    """Load libsp_gb300.so (building it in-tree if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _b
        path = _b.build_sp() if os.environ.get("SP_NO_BUILD") != "1" else _b.SP_LIB
        L = ct.CDLL(path)
        L.sp_status_str.restype = ct.c_char_p
        L.sp_last_error.restype = ct.c_char_p
        L.sp_kernel_launch_count.restype = ct.c_uint64
        L.sp_destroy.restype = None
        vp = ct.c_void_p
        L.sp_create.argtypes = [ct.POINTER(SpConfig), ct.POINTER(vp)]
        L.sp_create_from_state.argtypes = [ct.POINTER(SpConfig), _u32p, _f32p, _f32p,
                                           ct.POINTER(vp)]
        L.sp_destroy.argtypes = [vp]
        L.sp_get_info.argtypes = [vp, ct.POINTER(SpInfo)]
        L.sp_compute.argtypes = [vp, _u32p, ct.c_int]
        L.sp_compute_device.argtypes = [vp, vp, ct.c_int, vp]
        L.sp_compute_frames_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, ct.c_int, vp, vp]
        L.sp_compute_frames.argtypes = [vp, _u32p, ct.c_uint32, ct.c_uint64, ct.c_int, _u32p]
        L.sp_compute_frames_overlaps_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64,
                                                        ct.c_int, vp, vp, vp]
        L.sp_active_columns.argtypes = [vp, _u32p, ct.c_uint32, _u32p]
        L.sp_get_overlaps.argtypes = [vp, _f32p]
        L.sp_get_permanences.argtypes = [vp, _f32p]
        L.sp_get_pool.argtypes = [vp, _u32p]
        L.sp_get_boost.argtypes = [vp, _f32p]
        L.sp_get_duty_cycles.argtypes = [vp, _f32p]
        L.sp_save.argtypes = [vp, ct.c_char_p]
        L.sp_load.argtypes = [ct.c_char_p, ct.POINTER(vp)]
        L.sp_set_boost.argtypes = [vp, _f32p]
        L.sp_sync.argtypes = [vp]
        L.sp_set_timeout_ms.argtypes = [vp, ct.c_uint32]
        L.sp_status_str.argtypes = [ct.c_int]
        L.sp_step_noalloc.argtypes = [ct.POINTER(SpConfig), vp, vp, vp, vp, ct.c_int, vp, vp, vp]
        L.sp_batch_create.argtypes = [ct.POINTER(vp), ct.c_uint32, ct.POINTER(vp)]
        L.sp_batch_destroy.argtypes = [vp]
        L.sp_batch_destroy.restype = None
        L.sp_batch_get_info.argtypes = [vp, ct.POINTER(SpBatchInfo)]
        L.sp_batch_offsets.argtypes = [vp, ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64)]
        L.sp_batch_compute_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, ct.c_int, vp,
                                              ct.c_uint64, vp]
        L.sp_batch_compute.argtypes = [vp, _u32p, ct.c_uint32, ct.c_uint64, ct.c_int, _u32p,
                                       ct.c_uint64]
        L.sp_batch_forms.argtypes = [vp, _u32p]
        L.sp_batch_overlap_offsets.argtypes = [vp, ct.POINTER(ct.c_uint64),
                                               ct.POINTER(ct.c_uint64)]
        L.sp_batch_compute_overlaps_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64,
                                                       ct.c_int, vp, ct.c_uint64, vp,
                                                       ct.c_uint64, vp]
        L.sp_batch_infer_overlaps_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, vp,
                                                     ct.c_uint64, vp, ct.c_uint64, vp]
        L.sp_batch_sync.argtypes = [vp]
        L.sp_batch_set_device_wait_ns.argtypes = [vp, ct.c_uint64]
        L.sp_batch_autotune.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, _u32p]
        L.sp_batch_schedule.argtypes = [vp, _u32p, _u32p, _u32p]
        L.sp_batch_schedule_list.argtypes = [_u32p, _u32p, ct.c_uint32, _u32p]
        L.sp_batch_set_schedule.argtypes = [vp, ct.c_uint32, ct.c_uint32, _u32p]
        L.sp_batch_infer_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, vp, ct.c_uint64, vp]
        L.sp_server_create.argtypes = [ct.POINTER(SpServerConfig), ct.POINTER(vp)]
        L.sp_server_destroy.argtypes = [vp]
        L.sp_server_destroy.restype = None
        L.sp_server_open_stream.argtypes = [vp, ct.POINTER(SpConfig), _u32p]
        L.sp_server_open_stream_from_state.argtypes = [vp, ct.POINTER(SpConfig), _u32p, _f32p,
                                                       _f32p, _u32p]
        L.sp_server_close_stream.argtypes = [vp, ct.c_uint32]
        L.sp_server_submit.argtypes = [vp, ct.c_uint32, _u32p, ct.c_int,
                                       ct.POINTER(ct.c_uint64)]
        L.sp_server_submit_many.argtypes = [vp, ct.c_uint32, _u32p, ct.POINTER(vp),
                                            ct.POINTER(ct.c_int), ct.POINTER(ct.c_uint64),
                                            ct.POINTER(ct.c_int)]
        L.sp_server_submit_many_device.argtypes = [vp, ct.c_uint32, _u32p, ct.POINTER(vp),
                                                   ct.POINTER(ct.c_int),
                                                   ct.POINTER(ct.c_uint64),
                                                   ct.POINTER(ct.c_int), vp]
        L.sp_server_poll.argtypes = [vp, ct.POINTER(SpServerResult), ct.c_uint32, _u32p,
                                     ct.c_uint32, _u32p, ct.c_uint32]
        L.sp_server_get_permanences.argtypes = [vp, ct.c_uint32, _f32p]
        L.sp_server_get_stats.argtypes = [vp, ct.POINTER(SpServerStats), ct.c_int]
        L.sp_loadgen_run.argtypes = [vp, ct.POINTER(SpLoadgenConfig), ct.POINTER(SpLoadgenReport)]
        L.sp_encoder_config_init.argtypes = [ct.POINTER(SpEncoderConfig)]
        L.sp_encoder_create.argtypes = [ct.POINTER(SpEncoderConfig), ct.POINTER(vp)]
        L.sp_encoder_destroy.argtypes = [vp]
        L.sp_encoder_destroy.restype = None
        L.sp_encoder_get_info.argtypes = [vp, ct.POINTER(SpEncoderInfo)]
        L.sp_encode_device.argtypes = [vp, vp, ct.c_uint32, ct.c_uint64, vp, ct.c_uint64, vp]
        L.sp_encode_compute_device.argtypes = [vp, vp, vp, ct.c_uint32, ct.c_uint64, ct.c_int,
                                               vp, vp]
        L.sp_encode_compute.argtypes = [vp, vp, ct.POINTER(ct.c_uint8), ct.c_uint32, ct.c_int,
                                        _u32p]
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise SpError(rc, where, lib().sp_last_error().decode())


CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy


def _addr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    """A cudaStream_t for the ABI.  None selects the handle's own stream; a
    torch stream whose handle is 0 is the legacy default stream, which the
    ABI must receive as cudaStreamLegacy (its NULL means "own stream")."""
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or CUDA_STREAM_LEGACY
    return int(s) or CUDA_STREAM_LEGACY


def _np_u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return a, a.ctypes.data_as(_u32p)


def _np_f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_f32p)


def sp_config_init(**overrides):
    cfg = SpConfig()
    _check(lib().sp_config_init(ct.byref(cfg)), "sp_config_init")
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def sp_create(cfg):
    h = ct.c_void_p()
    _check(lib().sp_create(ct.byref(cfg), ct.byref(h)), "sp_create")
    return h


def sp_create_from_state(cfg, idx, perm, boost=None):
    idx, pi = _np_u32(idx)
    perm, pp = _np_f32(perm)
    pb = None
    if boost is not None:
        boost, pb = _np_f32(boost)
    h = ct.c_void_p()
    _check(lib().sp_create_from_state(ct.byref(cfg), pi, pp, pb, ct.byref(h)),
           "sp_create_from_state")
    return h


def sp_destroy(h):
    lib().sp_destroy(h)


def sp_get_info(h):
    info = SpInfo()
    _check(lib().sp_get_info(h, ct.byref(info)), "sp_get_info")
    return {f: getattr(info, f) for f, _ in SpInfo._fields_}


def sp_compute(h, input_bits, learn):
    a, p = _np_u32(input_bits)
    _check(lib().sp_compute(h, p, 1 if learn else 0), "sp_compute")
    return a  # keep alive until the next sync


def sp_compute_device(h, d_bits, learn, stream=None):
    _check(lib().sp_compute_device(h, _addr(d_bits), 1 if learn else 0, _stream(stream)),
           "sp_compute_device")


def sp_compute_frames_device(h, d_frames, n_frames, stride_words, learn, d_active_masks=None,
                             stream=None):
    _check(lib().sp_compute_frames_device(h, _addr(d_frames), n_frames, stride_words,
                                          1 if learn else 0, _addr(d_active_masks),
                                          _stream(stream)), "sp_compute_frames_device")


def sp_compute_frames_overlaps_device(h, d_frames, n_frames, stride_words, learn,
                                      d_active_masks=None, d_overlaps=None, stream=None):
    _check(lib().sp_compute_frames_overlaps_device(h, _addr(d_frames), n_frames, stride_words,
                                                   1 if learn else 0, _addr(d_active_masks),
                                                   _addr(d_overlaps), _stream(stream)),
           "sp_compute_frames_overlaps_device")


def sp_compute_frames(h, frames, learn, masks_out=None):
    """frames: uint32 [n][stride] host array (pinned memory overlaps the copies);
    masks_out: uint32 [n][mask_words] host array or None."""
    if frames.dtype != np.uint32 or frames.ndim != 2 or not frames.flags.c_contiguous:
        raise ValueError("frames must be a C-contiguous uint32 [n][stride] array")
    pm = None
    if masks_out is not None:
        if masks_out.dtype != np.uint32 or not masks_out.flags.c_contiguous:
            raise ValueError("masks_out must be a C-contiguous uint32 array")
        pm = masks_out.ctypes.data_as(_u32p)
    _check(lib().sp_compute_frames(h, frames.ctypes.data_as(_u32p), frames.shape[0],
                                   frames.shape[1], 1 if learn else 0, pm), "sp_compute_frames")
    return masks_out


def sp_active_columns(h, cap=None):
    if cap is None:
        cap = sp_get_info(h)["max_active"]
    out = np.zeros(max(cap, 1), np.uint32)
    n = ct.c_uint32()
    _check(lib().sp_active_columns(h, out.ctypes.data_as(_u32p), cap, ct.byref(n)),
           "sp_active_columns")
    return out[: n.value].copy()


def _getter(name, dtype, shape_fn):
    def get(h):
        info = sp_get_info(h)
        out = np.empty(shape_fn(info), dtype)
        ptr = out.ctypes.data_as(_f32p if dtype == np.float32 else _u32p)
        _check(getattr(lib(), name)(h, ptr), name)
        return out
    get.__name__ = name
    return get


sp_get_overlaps = _getter("sp_get_overlaps", np.float32, lambda i: (i["num_columns"],))
sp_get_permanences = _getter("sp_get_permanences", np.float32,
                             lambda i: (i["num_columns"], i["synapses_per_column"]))
sp_get_pool = _getter("sp_get_pool", np.uint32,
                      lambda i: (i["num_columns"], i["synapses_per_column"]))
sp_get_boost = _getter("sp_get_boost", np.float32, lambda i: (i["num_columns"],))
sp_get_duty_cycles = _getter("sp_get_duty_cycles", np.float32, lambda i: (i["num_columns"],))


def sp_save(h, path):
    _check(lib().sp_save(h, os.fsencode(path)), "sp_save")


def sp_load(path):
    h = ct.c_void_p()
    _check(lib().sp_load(os.fsencode(path), ct.byref(h)), "sp_load")
    return h


def sp_set_boost(h, boost):
    b, p = _np_f32(boost)
    _check(lib().sp_set_boost(h, p), "sp_set_boost")


def sp_sync(h):
    _check(lib().sp_sync(h), "sp_sync")


def sp_set_timeout_ms(h, ms):
    _check(lib().sp_set_timeout_ms(h, ms), "sp_set_timeout_ms")


def sp_step_noalloc(cfg, d_idx, d_perm, d_boost, d_input, learn, d_active_mask, d_active_list,
                    stream=None):
    """One frame on caller-owned device buffers, allocating nothing (see
    include/sp.h): every buffer is a device address or a CUDA tensor."""
    _check(lib().sp_step_noalloc(ct.byref(cfg), _addr(d_idx), _addr(d_perm), _addr(d_boost),
                                 _addr(d_input), 1 if learn else 0, _addr(d_active_mask),
                                 _addr(d_active_list), _stream(stream)), "sp_step_noalloc")


def sp_batch_create(members):
    arr = (ct.c_void_p * len(members))(*[m.value if isinstance(m, ct.c_void_p) else m
                                          for m in members])
    b = ct.c_void_p()
    _check(lib().sp_batch_create(arr, len(members), ct.byref(b)), "sp_batch_create")
    return b


def sp_batch_destroy(b):
    lib().sp_batch_destroy(b)


def sp_batch_get_info(b):
    info = SpBatchInfo()
    _check(lib().sp_batch_get_info(b, ct.byref(info)), "sp_batch_get_info")
    return {f: getattr(info, f) for f, _ in SpBatchInfo._fields_}


def sp_batch_offsets(b):
    n = sp_batch_get_info(b)["members"]
    fo = np.zeros(n, np.uint64)
    mo = np.zeros(n, np.uint64)
    _check(lib().sp_batch_offsets(b, fo.ctypes.data_as(ct.POINTER(ct.c_uint64)),
                                  mo.ctypes.data_as(ct.POINTER(ct.c_uint64))), "sp_batch_offsets")
    return fo, mo


def sp_batch_compute_device(b, d_frames, n_frames, stride_words, learn, d_masks=None,
                            mask_stride_words=0, stream=None):
    _check(lib().sp_batch_compute_device(b, _addr(d_frames), n_frames, stride_words,
                                         1 if learn else 0, _addr(d_masks), mask_stride_words,
                                         _stream(stream)), "sp_batch_compute_device")


SP_FORM_FULL, SP_FORM_COMPACT, SP_FORM_WINDOW = 0, 1, 2
FORM_NAMES = {SP_FORM_FULL: "full", SP_FORM_COMPACT: "compact", SP_FORM_WINDOW: "window"}


def sp_batch_forms(b):
    """Per-member form of the batch state (SP_FORM_*)."""
    n = sp_batch_get_info(b)["members"]
    out = np.zeros(n, np.uint32)
    _check(lib().sp_batch_forms(b, out.ctypes.data_as(_u32p)), "sp_batch_forms")
    return out


def sp_batch_overlap_offsets(b):
    """Per-member float offsets inside a batch overlap record, and its length."""
    n = sp_batch_get_info(b)["members"]
    oo = np.zeros(n, np.uint64)
    words = ct.c_uint64()
    _check(lib().sp_batch_overlap_offsets(b, oo.ctypes.data_as(ct.POINTER(ct.c_uint64)),
                                          ct.byref(words)), "sp_batch_overlap_offsets")
    return oo, words.value


def sp_batch_compute_overlaps_device(b, d_frames, n_frames, stride_words, learn, d_masks=None,
                                     mask_stride_words=0, d_overlaps=None, ov_stride=0,
                                     stream=None):
    _check(lib().sp_batch_compute_overlaps_device(b, _addr(d_frames), n_frames, stride_words,
                                                  1 if learn else 0, _addr(d_masks),
                                                  mask_stride_words, _addr(d_overlaps),
                                                  ov_stride, _stream(stream)),
           "sp_batch_compute_overlaps_device")


def sp_batch_infer_overlaps_device(b, d_frames, n_frames, stride_words, d_masks=None,
                                   mask_stride_words=0, d_overlaps=None, ov_stride=0,
                                   stream=None):
    _check(lib().sp_batch_infer_overlaps_device(b, _addr(d_frames), n_frames, stride_words,
                                                _addr(d_masks), mask_stride_words,
                                                _addr(d_overlaps), ov_stride, _stream(stream)),
           "sp_batch_infer_overlaps_device")


SP_MIXED_SPLIT = 0xFFFFFFFF


def sp_batch_autotune(b, d_frames, n_frames, stride_words):
    """Pick the batch pass's schedule and CTA splits on device batch frames;
    returns the columns per warp chosen when every member has the same (0:
    the defaults), else SP_MIXED_SPLIT (sp_batch_schedule has each)."""
    out = ct.c_uint32(0)
    _check(lib().sp_batch_autotune(b, _addr(d_frames), n_frames, stride_words, ct.byref(out)),
           "sp_batch_autotune")
    return out.value


def sp_batch_schedule(b, members):
    """(ctas_per_sm, cols_in_flight, [columns per warp of each member, 0:
    default]) of the batch's persistent pass."""
    cps, cif = ct.c_uint32(0), ct.c_uint32(0)
    per = (ct.c_uint32 * max(1, members))()
    _check(lib().sp_batch_schedule(b, ct.byref(cps), ct.byref(cif), per), "sp_batch_schedule")
    return cps.value, cif.value, [int(per[i]) for i in range(members)]


def sp_batch_schedule_list():
    """[(ctas_per_sm, cols_in_flight)] of the compiled schedules; the first is
    the default."""
    n = ct.c_uint32(0)
    _check(lib().sp_batch_schedule_list(None, None, 0, ct.byref(n)), "sp_batch_schedule_list")
    cps = (ct.c_uint32 * max(1, n.value))()
    cif = (ct.c_uint32 * max(1, n.value))()
    _check(lib().sp_batch_schedule_list(cps, cif, n.value, None), "sp_batch_schedule_list")
    return [(int(cps[i]), int(cif[i])) for i in range(n.value)]


def sp_batch_set_schedule(b, ctas_per_sm, cols_in_flight, member_cols_per_warp=None):
    """Pin the batch's compiled schedule and each member's columns per warp
    (None: the defaults)."""
    per = None
    if member_cols_per_warp is not None:
        per = (ct.c_uint32 * len(member_cols_per_warp))(*member_cols_per_warp)
    _check(lib().sp_batch_set_schedule(b, ctas_per_sm, cols_in_flight, per),
           "sp_batch_set_schedule")


def sp_batch_compute(b, frames, learn, masks_out=None):
    """frames: uint32 [n][stride] host batch frames; masks_out: uint32 [n][mstride] or None."""
    if frames.dtype != np.uint32 or frames.ndim != 2 or not frames.flags.c_contiguous:
        raise ValueError("frames must be a C-contiguous uint32 [n][stride] array")
    pm, ms = None, 0
    if masks_out is not None:
        if masks_out.dtype != np.uint32 or masks_out.ndim != 2 or not masks_out.flags.c_contiguous:
            raise ValueError("masks_out must be a C-contiguous uint32 [n][stride] array")
        pm, ms = masks_out.ctypes.data_as(_u32p), masks_out.shape[1]
    _check(lib().sp_batch_compute(b, frames.ctypes.data_as(_u32p), frames.shape[0],
                                  frames.shape[1], 1 if learn else 0, pm, ms), "sp_batch_compute")
    return masks_out


def sp_batch_infer_device(b, d_frames, n_frames, stride_words, d_masks=None,
                          mask_stride_words=0, stream=None):
    _check(lib().sp_batch_infer_device(b, _addr(d_frames), n_frames, stride_words,
                                       _addr(d_masks), mask_stride_words, _stream(stream)),
           "sp_batch_infer_device")


def sp_batch_set_device_wait_ns(b, ns):
    _check(lib().sp_batch_set_device_wait_ns(b, ns), "sp_batch_set_device_wait_ns")


def sp_batch_sync(b):
    _check(lib().sp_batch_sync(b), "sp_batch_sync")


def sp_server_create(max_streams, queue_depth, max_input_words, device_budget_bytes,
                     max_active):
    cfg = SpServerConfig(SP_ABI_VERSION, max_streams, queue_depth, max_input_words,
                         device_budget_bytes, max_active, 0)
    s = ct.c_void_p()
    _check(lib().sp_server_create(ct.byref(cfg), ct.byref(s)), "sp_server_create")
    return s


def sp_server_destroy(s):
    lib().sp_server_destroy(s)


def sp_server_open_stream(s, cfg, state=None):
    sid = ct.c_uint32()
    if state is None:
        _check(lib().sp_server_open_stream(s, ct.byref(cfg), ct.byref(sid)),
               "sp_server_open_stream")
    else:
        idx, perm, boost = state
        idx, pi = _np_u32(idx)
        perm, pp = _np_f32(perm)
        pb = None
        if boost is not None:
            boost, pb = _np_f32(boost)
        _check(lib().sp_server_open_stream_from_state(s, ct.byref(cfg), pi, pp, pb,
                                                      ct.byref(sid)),
               "sp_server_open_stream_from_state")
    return sid.value


def sp_server_close_stream(s, sid):
    _check(lib().sp_server_close_stream(s, sid), "sp_server_close_stream")


def sp_server_submit(s, sid, frame_bits, learn):
    a, p = _np_u32(frame_bits)
    rid = ct.c_uint64()
    _check(lib().sp_server_submit(s, sid, p, 1 if learn else 0, ct.byref(rid)),
           "sp_server_submit")
    return rid.value


def sp_server_submit_many(srv, stream_ids, frames, learn=True):
    """Queue one frame per entry (frames: list of uint32 arrays, C-contiguous).
    Returns (statuses int array, request ids uint64 array)."""
    n = len(stream_ids)
    frames = [np.ascontiguousarray(f, dtype=np.uint32) for f in frames]
    ptrs = np.array([f.ctypes.data for f in frames], dtype=np.uint64)
    lf = learn if hasattr(learn, "__len__") else [learn] * n
    larr = np.array([1 if x else 0 for x in lf], dtype=np.int32)
    return sp_server_submit_many_ptrs(srv, np.asarray(stream_ids, dtype=np.uint32), ptrs, larr)


def sp_server_submit_many_ptrs(srv, stream_ids, frame_ptrs, learn):
    """sp_server_submit_many on prepared arrays: stream ids (uint32), host
    addresses of the frames (uint64; the caller keeps the frames alive until
    the call returns) and learn flags (int32).  Returns (statuses, ids)."""
    n = len(stream_ids)
    ids = np.ascontiguousarray(stream_ids, dtype=np.uint32)
    ptrs = np.ascontiguousarray(frame_ptrs, dtype=np.uint64)
    larr = np.ascontiguousarray(learn, dtype=np.int32)
    rid = np.zeros(n, np.uint64)
    st = np.zeros(n, np.int32)
    _check(lib().sp_server_submit_many(srv, n, ids.ctypes.data_as(_u32p),
                                       ptrs.ctypes.data_as(ct.POINTER(ct.c_void_p)),
                                       larr.ctypes.data_as(ct.POINTER(ct.c_int)),
                                       rid.ctypes.data_as(ct.POINTER(ct.c_uint64)),
                                       st.ctypes.data_as(ct.POINTER(ct.c_int))),
           "sp_server_submit_many")
    return st, rid


def sp_server_submit_many_device(srv, stream_ids, d_frame_ptrs, learn, stream=None):
    """sp_server_submit_many for device frames: stream ids (uint32), device
    addresses of the frames (uint64) and learn flags (int32); the copies run
    on `stream` (torch stream or handle; None = legacy default).
    Returns (statuses, request ids)."""
    n = len(stream_ids)
    ids = np.ascontiguousarray(stream_ids, dtype=np.uint32)
    ptrs = np.ascontiguousarray(d_frame_ptrs, dtype=np.uint64)
    larr = np.ascontiguousarray(learn, dtype=np.int32)
    rid = np.zeros(n, np.uint64)
    st = np.zeros(n, np.int32)
    _check(lib().sp_server_submit_many_device(
        srv, n, ids.ctypes.data_as(_u32p), ptrs.ctypes.data_as(ct.POINTER(ct.c_void_p)),
        larr.ctypes.data_as(ct.POINTER(ct.c_int)), rid.ctypes.data_as(ct.POINTER(ct.c_uint64)),
        st.ctypes.data_as(ct.POINTER(ct.c_int)), _stream(stream) or CUDA_STREAM_LEGACY),
        "sp_server_submit_many_device")
    return st, rid


def sp_server_poll(s, max_results=256, active_cap=1 << 16, wait_ms=0):
    """Returns a list of (result dict, active ndarray)."""
    res = (SpServerResult * max_results)()
    act = np.zeros(active_cap, np.uint32)
    n = ct.c_uint32()
    _check(lib().sp_server_poll(s, res, max_results, act.ctypes.data_as(_u32p), active_cap,
                                ct.byref(n), wait_ms), "sp_server_poll")
    out = []
    for i in range(n.value):
        r = res[i]
        d = {f: getattr(r, f) for f, _ in SpServerResult._fields_}
        out.append((d, act[r.active_offset:r.active_offset + r.n_active].copy()))
    return out


_drain_bufs = {}


def sp_server_drain(s, wait_ms=0, max_results=4096, active_cap=1 << 18):
    """Take up to max_results finished frames without building per-result
    objects (latency percentiles stay available from sp_server_get_stats).
    Returns (frames taken, frames whose status was not SP_OK)."""
    key = (max_results, active_cap)
    if key not in _drain_bufs:
        _drain_bufs[key] = ((SpServerResult * max_results)(), np.zeros(active_cap, np.uint32))
    res, act = _drain_bufs[key]
    n = ct.c_uint32()
    _check(lib().sp_server_poll(s, res, max_results, act.ctypes.data_as(_u32p), active_cap,
                                ct.byref(n), wait_ms), "sp_server_poll")
    bad = sum(1 for i in range(n.value) if res[i].status != 0) if n.value else 0
    return n.value, bad


def sp_server_get_permanences(s, sid, shape):
    out = np.empty(shape, np.float32)
    _check(lib().sp_server_get_permanences(s, sid, out.ctypes.data_as(_f32p)),
           "sp_server_get_permanences")
    return out


def sp_server_get_stats(s, reset=False):
    st = SpServerStats()
    _check(lib().sp_server_get_stats(s, ct.byref(st), 1 if reset else 0), "sp_server_get_stats")
    return {f: getattr(st, f) for f, _ in SpServerStats._fields_}


def sp_loadgen_run(srv, stream_ids, pools, rate_per_stream, seconds, producers=4, learn=True,
                   seed=0):
    """Drive the server with native producer threads (include/sp_loadgen.h).
    pools: one C-contiguous uint32 [frames][words] host array per stream
    (kept alive by the caller for the call).  rate_per_stream 0 = closed
    loop.  Returns the report as a dict."""
    n = len(stream_ids)
    pools = [np.ascontiguousarray(p, dtype=np.uint32) for p in pools]
    ids = np.ascontiguousarray(stream_ids, dtype=np.uint32)
    ptrs = (ct.c_void_p * n)(*[p.ctypes.data for p in pools])
    nf = np.array([p.shape[0] for p in pools], np.uint32)
    stride = np.array([p.shape[1] for p in pools], np.uint64)
    cfg = SpLoadgenConfig(n, ids.ctypes.data_as(_u32p), ptrs, nf.ctypes.data_as(_u32p),
                          stride.ctypes.data_as(ct.POINTER(ct.c_uint64)), float(rate_per_stream),
                          float(seconds), producers, 1 if learn else 0, seed)
    rep = SpLoadgenReport()
    _check(lib().sp_loadgen_run(srv, ct.byref(cfg), ct.byref(rep)), "sp_loadgen_run")
    return {f: getattr(rep, f) for f, _ in SpLoadgenReport._fields_}


def sp_kernel_launch_count():
    return lib().sp_kernel_launch_count()


def sp_status_str(s):
    return lib().sp_status_str(s).decode()


def sp_last_error():
    return lib().sp_last_error().decode()


def masks_to_dense(masks, C):
    """uint32 [..., mask_words] packed masks -> uint8 [..., C] (host helper)."""
    m = np.ascontiguousarray(masks, dtype="<u4")
    b = np.unpackbits(m.view(np.uint8), axis=-1, bitorder="little")
    return b[..., :C]


class SpatialPooler:
    """Owner of one sp_handle (destroyed with the object)."""

    def __init__(self, cfg=None, state=None, **overrides):
        self.cfg = cfg if cfg is not None else sp_config_init(**overrides)
        if state is None:
            self.h = sp_create(self.cfg)
        else:
            self.h = sp_create_from_state(self.cfg, *state)
        self.info = sp_get_info(self.h)
        self._keep = None

    def compute(self, input_bits, learn):
        self._keep = sp_compute(self.h, input_bits, learn)
        return self

    def active_columns(self):
        return sp_active_columns(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            sp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- frame encoder ----------------------------------------------------------

def sp_encoder_config_init(**kw):
    cfg = SpEncoderConfig()
    _check(lib().sp_encoder_config_init(ct.byref(cfg)), "sp_encoder_config_init")
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def sp_encoder_create(cfg):
    e = ct.c_void_p()
    _check(lib().sp_encoder_create(ct.byref(cfg), ct.byref(e)), "sp_encoder_create")
    return e


def sp_encoder_destroy(e):
    lib().sp_encoder_destroy(e)


def sp_encoder_get_info(e):
    info = SpEncoderInfo()
    _check(lib().sp_encoder_get_info(e, ct.byref(info)), "sp_encoder_get_info")
    return {f: getattr(info, f) for f, _ in SpEncoderInfo._fields_}


def sp_encode_device(e, d_src, n_frames, src_stride, d_bits, bits_stride, stream=None):
    _check(lib().sp_encode_device(e, _addr(d_src), n_frames, src_stride, _addr(d_bits),
                                  bits_stride, _stream(stream)), "sp_encode_device")


def sp_encode_compute_device(e, h, d_src, n_frames, src_stride, learn, d_active_masks=None,
                             stream=None):
    _check(lib().sp_encode_compute_device(e, h, _addr(d_src), n_frames, src_stride,
                                          1 if learn else 0, _addr(d_active_masks),
                                          _stream(stream)), "sp_encode_compute_device")


def sp_encode_compute(e, h, frames, learn, masks_out=None):
    """frames: uint8 [n, H, W(, 3)] host array, C-contiguous (pinned memory
    overlaps the copies); masks_out: uint32 [n][mask_words] or None."""
    if frames.dtype != np.uint8 or not frames.flags.c_contiguous:
        raise ValueError("frames must be a C-contiguous uint8 array")
    pm = None
    if masks_out is not None:
        if masks_out.dtype != np.uint32 or not masks_out.flags.c_contiguous:
            raise ValueError("masks_out must be a C-contiguous uint32 array")
        pm = masks_out.ctypes.data_as(_u32p)
    _check(lib().sp_encode_compute(e, h, frames.ctypes.data_as(ct.POINTER(ct.c_uint8)),
                                   frames.shape[0], 1 if learn else 0, pm), "sp_encode_compute")
    return masks_out
