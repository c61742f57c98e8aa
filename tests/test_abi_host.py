"""C-ABI checks that need no GPU: every function declared in include/*.h is
exported by its library, configurations are validated on the host before any
CUDA call, and the status strings are stable."""
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1608_01966_gb300 as spg
from paper_1608_01966_gb300 import build
from conftest import ROOT


def _declared(header, macro):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(macro + r"\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


def _exported(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if line.strip()}


@pytest.mark.parametrize("header,macro,which", [
    ("sp.h", "SP_API", "sp"),
    ("sp_loadgen.h", "SP_API", "sp"),
    ("sp_synth.h", "SYNTH_API", "synth"),
])
def test_library_exports_every_declared_symbol(header, macro, which):
    path = build.build_sp() if which == "sp" else build.build_synth()
    names = _declared(header, macro)
    assert len(names) >= (1 if header == "sp_loadgen.h" else 8)
    missing = [n for n in names if n not in _exported(path)]
    assert not missing, f"{os.path.basename(path)} lacks {missing}"
    import ctypes
    L = ctypes.CDLL(path)
    for n in names:
        getattr(L, n)


def test_config_defaults_are_table2():
    cfg = spg.sp_config_init()
    assert cfg.abi_version == spg.SP_ABI_VERSION
    assert (cfg.num_columns, cfg.synapses_per_column) == (2048, 128)
    assert (cfg.min_overlap, cfg.winners_set_size) == (8, 40)
    assert abs(cfg.perm_inc - 0.1) < 1e-7 and abs(cfg.perm_dec - 0.1) < 1e-7
    assert abs(cfg.perm_init_lo - 0.21) < 1e-7 and cfg.perm_init_lo == cfg.perm_init_hi
    assert (cfg.input_w, cfg.input_h) == (240, 134)


@pytest.mark.parametrize("bad", [
    dict(abi_version=99),
    dict(num_columns=0),
    dict(num_columns=spg.SP_MAX_COLUMNS + 1),
    dict(synapses_per_column=0),
    dict(input_w=0),
    dict(inhibition=1),                            # local without a column grid
    dict(inhibition=7),
    dict(col_grid_w=10, col_grid_h=10),            # grid does not match C
    dict(perm_inc=-0.1),
    dict(perm_init_lo=0.5, perm_init_hi=0.4),
    dict(pool_mode=9),
    dict(synapses_per_column=40000),               # S > n_in for uniform pools
    dict(pool_mode=2),                             # dense pools need S == n_in
    dict(pool_mode=1),                             # windowed pools need a grid
    dict(connect_threshold=float("nan")),
])
def test_create_rejects_bad_config_on_host(bad):
    cfg = spg.sp_config_init(**bad)
    with pytest.raises(spg.SpError) as e:
        spg.sp_create(cfg)
    assert e.value.status == 1  # SP_EINVAL, raised before any CUDA call
    assert spg.sp_last_error()


def test_create_from_state_rejects_bad_state_on_host():
    import numpy as np
    cfg = spg.sp_config_init(input_w=16, input_h=1, num_columns=2, synapses_per_column=2)
    idx = np.array([[0, 1], [2, 16]], np.uint32)  # 16 is out of range
    perm = np.full((2, 2), 0.3, np.float32)
    with pytest.raises(spg.SpError):
        spg.sp_create_from_state(cfg, idx, perm)
    idx[1, 1] = 3
    perm[0, 0] = 1.5
    with pytest.raises(spg.SpError):
        spg.sp_create_from_state(cfg, idx, perm)
    perm[0, 0] = 0.3
    with pytest.raises(spg.SpError):
        spg.sp_create_from_state(cfg, idx, perm, np.array([1.0, -1.0], np.float32))


def test_encoder_defaults():
    cfg = spg.sp_encoder_config_init()
    assert (cfg.src_w, cfg.src_h, cfg.channels, cfg.reduce, cfg.block, cfg.offset) == \
        (960, 540, 3, 1, 11, 2)


@pytest.mark.parametrize("bad", [
    dict(block=4), dict(block=1), dict(block=15), dict(channels=2), dict(reduce=0),
    dict(reduce=9), dict(src_w=0), dict(src_h=70000), dict(src_w=7, reduce=8),
    dict(src_w=65535, src_h=65535),                # 2^32 output bits
    dict(src_w=20000, src_h=4),                    # too wide for one CTA's rows
])
def test_encoder_rejects_bad_config_on_host(bad):
    cfg = spg.sp_encoder_config_init(**bad)
    with pytest.raises(spg.SpError) as e:
        spg.sp_encoder_create(cfg)
    assert e.value.status == 1  # SP_EINVAL, raised before any CUDA call


def test_status_strings_and_null_safety():
    assert spg.sp_status_str(0) == "ok"
    assert spg.sp_status_str(4) == "timed out"
    spg.sp_destroy(None)  # NULL-safe
    spg.sp_encoder_destroy(None)
    assert spg.sp_kernel_launch_count() >= 0


def test_masks_to_dense_roundtrip():
    import numpy as np
    from paper_1608_01966_gb300 import synth
    rng = np.random.default_rng(0)
    bits = (rng.random((3, 70)) < 0.3).astype(np.uint8)
    packed = synth.pack_frames(bits)
    np.testing.assert_array_equal(spg.masks_to_dense(packed, 70), bits)


def test_load_generator_rejects_invalid_arguments():
    """Argument checks happen before any call to the server."""
    with pytest.raises(spg.SpError) as e:
        spg.sp_loadgen_run(None, [0], [np.zeros((1, 4), np.uint32)], 30.0, 1.0)
    assert e.value.status == 1
    with pytest.raises(spg.SpError) as e:
        spg.sp_loadgen_run(1, [0], [np.zeros((1, 4), np.uint32)], -1.0, 1.0)
    assert e.value.status == 1


def test_compiled_batch_schedules_are_listed():
    """The persistent batch pass is compiled in several schedules (resident
    CTAs per SM x columns per warp in flight) for the autotuner to choose
    from; the default (10 x 4) comes first and no pair repeats."""
    import paper_1608_01966_gb300 as spg
    lst = spg.sp_batch_schedule_list()
    assert lst[0] == (10, 4)
    assert len(set(lst)) == len(lst) >= 4
    assert all(8 <= c <= 12 and 2 <= f <= 8 for c, f in lst)
    with pytest.raises(spg.SpError):  # no room for the list
        import ctypes as ct
        a = (ct.c_uint32 * 1)()
        spg._binding._check(spg.lib().sp_batch_schedule_list(a, a, 1, None), "list")
    with pytest.raises(spg.SpError):  # no such batch
        spg.sp_batch_set_schedule(None, 10, 4)
