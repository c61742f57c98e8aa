"""GB300 (sm_103a) Spatial Pooler hot path of Wielgosz & Pietron's
OpenCL-accelerated HTM video classifier: overlap (Alg. 1), inhibition
(Alg. 2) and winner-column permanence learning, as CUDA kernels behind the C
ABI in include/sp.h.  This package holds the ctypes binding, the in-tree
build and the seeded input generators."""
from ._binding import (  # noqa: F401
    SP_ABI_VERSION, SP_INHIBIT_GLOBAL, SP_INHIBIT_LOCAL, SP_INHIBIT_PAPER_LITERAL,
    SP_MAX_COLUMNS, SP_POOL_DENSE, SP_POOL_UNIFORM, SP_POOL_WINDOW, SpConfig, SpError,
    SpatialPooler, lib, masks_to_dense,
    sp_active_columns, sp_batch_autotune, sp_batch_schedule, sp_batch_schedule_list,
    sp_batch_set_schedule, SP_MIXED_SPLIT, sp_batch_compute,
    sp_batch_compute_device,
    sp_batch_compute_overlaps_device, sp_batch_create, sp_batch_destroy, sp_batch_get_info,
    sp_batch_infer_device, sp_batch_infer_overlaps_device, sp_batch_offsets,
    sp_batch_overlap_offsets, sp_batch_set_device_wait_ns, sp_batch_sync, sp_batch_forms,
    SP_FORM_FULL, SP_FORM_COMPACT, SP_FORM_WINDOW, FORM_NAMES,
    sp_compute, sp_compute_device, sp_compute_frames, sp_compute_frames_device,
    sp_compute_frames_overlaps_device, sp_config_init, sp_create, sp_create_from_state,
    sp_destroy, sp_get_boost, sp_get_duty_cycles, sp_get_info, sp_get_overlaps,
    sp_get_permanences, sp_get_pool, sp_kernel_launch_count, sp_last_error, sp_load, sp_save,
    sp_set_boost, sp_set_timeout_ms, sp_status_str,
    sp_server_close_stream, sp_server_create, sp_server_drain, sp_server_destroy,
    sp_server_get_permanences, sp_server_get_stats, sp_server_open_stream, sp_server_poll,
    sp_server_submit, sp_server_submit_many, sp_server_submit_many_device,
    sp_server_submit_many_ptrs,
    sp_step_noalloc, sp_sync, sp_loadgen_run,
    SpEncoderConfig, sp_encode_compute, sp_encode_compute_device, sp_encode_device,
    sp_encoder_config_init, sp_encoder_create, sp_encoder_destroy, sp_encoder_get_info,
)
