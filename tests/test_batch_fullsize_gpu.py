"""The benchmark's launch configuration at full size: 256 paper-scale frame
SPs (1024 columns x 256 synapses from 64x64 windows of 960x540 blobbed
frames, k = 40, learning on), autotuned, stepped by persistent launches over
several frames and by single-frame launches.  The oracle checks sampled
members frame by frame (every boosted overlap and the winners) and their
final permanences: bit-exact."""
import concurrent.futures as cf

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1608_01966_gb300 as spg  # noqa: E402
from paper_1608_01966_gb300 import synth, workloads as wl  # noqa: E402
from helpers import dense, first_diff, oracle_run  # noqa: E402

pytestmark = pytest.mark.gpu

N_SP = 256
SAMPLED = (0, 1, 97, 170, 255)


def test_full_size_batch_sampled_against_oracle():
    seeds = [wl.BASE_SEED + 2 + 17 * i for i in range(N_SP)]
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        cases = list(ex.map(lambda s: wl.frame_case(seed=s), seeds))
        pool = np.stack(list(ex.map(lambda t: synth.frame_blobbed(
            synth.derive_seed(wl.BASE_SEED + 2, synth.PURPOSE_FRAME, t), 960, 540), range(8))))
    packed = wl.pack(pool)
    hs = [spg.sp_create_from_state(c.config(), c.idx, c.perm, c.boost) for c in cases]
    b = spg.sp_batch_create(hs)
    info = spg.sp_batch_get_info(b)
    fo, mo = spg.sp_batch_offsets(b)
    fw = (info["frame_words"] + 3) // 4 * 4
    n_frames = 6
    # member i sees pool frame (7 i + t) mod 8 at step t
    batch = np.zeros((n_frames, fw), np.uint32)
    for t in range(n_frames):
        for i in range(N_SP):
            batch[t, int(fo[i]):int(fo[i]) + packed.shape[1]] = packed[(7 * i + t) % 8]
    d = torch.from_numpy(batch.view(np.int32)).cuda()
    mw = info["mask_words"]
    oo, ow = spg.sp_batch_overlap_offsets(b)
    dm = torch.zeros((n_frames, mw), dtype=torch.int32, device="cuda")
    dov = torch.full((n_frames, ow), -1.0, dtype=torch.float32, device="cuda")
    spg.sp_batch_autotune(b, d, 2, fw)
    st = torch.cuda.current_stream()
    # one persistent launch, then two single-frame launches
    spg.sp_batch_compute_overlaps_device(b, d[0], 4, fw, True, dm[0], mw, dov[0], ow, st)
    spg.sp_batch_compute_overlaps_device(b, d[4], 1, fw, True, dm[4], mw, dov[4], ow, st)
    spg.sp_batch_compute_overlaps_device(b, d[5], 1, fw, True, dm[5], mw, dov[5], ow, st)
    spg.sp_batch_sync(b)
    masks = dm.cpu().numpy().view(np.uint32)
    ovr = dov.cpu().numpy()
    spg.sp_batch_destroy(b)
    for i in SAMPLED:
        c = cases[i]
        frames = np.stack([pool[(7 * i + t) % 8] for t in range(n_frames)])
        want, perm, ov = oracle_run(c, frames, True, want_ov=True)
        d = first_diff(ovr[:, int(oo[i]):int(oo[i]) + c.C], ov)
        assert d is None, f"member {i}: overlap (frame, column) {d}"
        got = dense(masks[:, int(mo[i]):int(mo[i]) + 32], c.C)
        assert first_diff(got, want) is None, f"member {i}: {first_diff(got, want)}"
        assert got.sum(axis=1).max() <= c.k
        np.testing.assert_array_equal(spg.sp_get_permanences(hs[i]), perm, err_msg=f"member {i}")
    for h in hs:
        spg.sp_destroy(h)
