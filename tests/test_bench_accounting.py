"""The benchmark's byte accounting and its traffic gate, on CPU.

The canonical algorithmic bytes of one paper-scale SP frame (1024 columns x
256 synapses, a 960x540 frame, k = 40, learning) are the per-unit figure the
HBM roofline divides by; the compact form's own bytes are what its traffic is
compared with.  Both are checked against the figures worked out by hand from
their definitions, and the DRAM traffic from the committed ncu summary must be
reported only for the kernel and sources it was captured on."""
import json
import os

import numpy as np
import pytest

import bench
from paper_1608_01966_gb300 import synth, workloads as wl


@pytest.fixture(scope="module")
def frame_case():
    return wl.frame_case(seed=bench.instance_seed(0, 0))


def test_canonical_bytes_of_a_paper_scale_frame(frame_case):
    c = frame_case
    assert (c.C, c.S, c.n_words, c.k) == (1024, 256, 960 * 540 // 32, 40)
    # pools + permanences 2 MiB, frame 64,800 B, overlaps 4 KiB, list 160 B,
    # learned rows 40 KiB
    assert bench.algorithmic_bytes_per_frame(c) == 2 * 1048576 + 64800 + 4096 + 160 + 40960
    assert bench.algorithmic_bytes_per_frame(c) == 2207168
    assert bench.algorithmic_bytes_per_frame(c, learn=False) == 2207168 - 40960


def test_compact_bytes_of_a_paper_scale_frame(frame_case):
    c = frame_case
    assert bench.compact_form(c)  # 64x64 windows span far less than 65536 inputs
    # offsets 512 KiB, connected bits 32 KiB, bases 4 KiB, frame, overlaps,
    # list, learned rows read + written (80 KiB) and their bits (1280 B)
    want = 524288 + 32768 + 4096 + 64800 + 4096 + 160 + 81920 + 1280
    assert bench.compact_bytes_per_frame(c) == want == 713408


def test_window_bytes_of_a_paper_scale_frame(frame_case):
    c = frame_case
    # bitmaps 512 KiB, origins 4 KiB, frame 64,800 B, overlaps 4 KiB, list
    # 160 B; 40 learning columns each read 1 KiB of pool indices, read and
    # write 1 KiB of permanences and rewrite a 512-byte bitmap
    want = 524288 + 4096 + 64800 + 4096 + 160 + 40 * (1024 + 2048 + 512)
    assert bench.window_bytes_per_frame(c) == want == 740800
    assert bench.form_bytes_per_frame(c, "window") == want
    assert bench.form_bytes_per_frame(c, "compact") == 713408
    assert bench.form_bytes_per_frame(c, "full") == 2207168


def test_compact_form_pads_rows_and_needs_a_narrow_span():
    idx = synth.pool_uniform(3, 64, 17, 60000)
    ragged = wl.Case("ragged", 60000, 1, 64, 17, idx, np.zeros((64, 17), np.float32),
                     np.ones(64, np.float32), k=2)
    assert bench.compact_form(ragged)  # S = 17: rows padded to 32 synapses
    # 64 columns x 32 padded synapses x (2 + 1/8) B, bases, frame (1875
    # words), overlaps, list; 2 learners x (17 x 8 B + 32 bits)
    want = 64 * 32 * 2 + 64 * 32 // 8 + 64 * 4 + 1875 * 4 + 64 * 4 + 2 * 4 + 2 * (17 * 8 + 4)
    assert bench.compact_bytes_per_frame(ragged) == want
    big = wl.Case("big", 60000, 1, 8, 257, synth.pool_uniform(5, 8, 257, 60000),
                  np.zeros((8, 257), np.float32), np.ones(8, np.float32))
    assert not bench.compact_form(big)  # S > 256
    wide_idx = synth.pool_uniform(4, 64, 32, 200000)
    wide = wl.Case("wide", 200000, 1, 64, 32, wide_idx, np.zeros((64, 32), np.float32),
                   np.ones(64, np.float32))
    assert int((wide_idx.max(axis=1) - wide_idx.min(axis=1)).max()) > 0xFFFF
    assert not bench.compact_form(wide)


def test_traffic_reported_only_for_the_captured_kernel_and_sources(tmp_path, monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "sp_batch_step_traffic.json")) as f:
        d = json.load(f)
    # reported while the capture's sources are the current ones, else null
    if d["source_sha"] == bench.kernel_source_sha():
        assert bench.read_traffic(d["kernel"]) == d["dram_bytes_per_step"]
    else:
        assert bench.read_traffic(d["kernel"]) is None
    assert bench.read_traffic("some_other_kernel") is None
    # a capture of other sources is not reported
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    stale = dict(d, source_sha="0" * 16)
    (root / "profiles" / "sp_batch_step_traffic.json").write_text(json.dumps(stale))
    csrc = root / "paper_1608_01966_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("sp_step.cu", "sp_kernels.cuh", "sp_device.cuh", "sp_abi.cu"):
        (csrc / f).write_bytes(open(os.path.join(bench.ROOT, "paper_1608_01966_gb300", "csrc", f),
                                    "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.read_traffic(d["kernel"]) is None
