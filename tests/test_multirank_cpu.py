"""The multi-rank path of the benchmark on CPU (gloo, world size 2): every
rank steps its own SPs (no data exchange), the timing is the max over ranks
and the throughput the sum.  Each rank runs the oracle on its SPs here, and
a rank that raises is reported by the launcher (failure on the host, no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, fail_rank):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_1608_01966_gb300 import synth

    seeds = [bench.instance_seed(rank, i) for i in range(3)]
    cases = bench.make_cases(3, rank)
    # each rank's SPs on their own frames: the oracle stands in for the GPU step
    winners = []
    for c, sd in zip(cases, seeds):
        fr = np.stack([synth.frame_bernoulli(synth.derive_seed(sd, 3, t), c.n_in, 0.1)
                       for t in range(2)])
        p = oracle.params(c.C, c.S, c.n_in, c.thr, c.inc, c.dec, c.min_overlap, c.k)
        winners.append(int(oracle.run(p, c.idx, c.perm.copy(), c.boost, fr, True).sum()))
    if rank == fail_rank:
        raise RuntimeError("rank failed on purpose (host-side)")
    t_local = 1.0 + rank  # stands in for this rank's measured ms/step
    t_max = bench.reduce_max(t_local)
    got = [None] * world
    dist.all_gather_object(got, {"seeds": seeds, "winners": winners})
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([t_max] + [s for g in got for s in g["seeds"]], dtype=np.float64))
    dist.destroy_process_group()


def _launch(tmp_path, fail_rank=-1):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path), fail_rank))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    return codes


def test_two_ranks_shard_without_exchange(tmp_path):
    codes = _launch(tmp_path)
    assert codes == [0, 0]
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 2.0  # max over ranks of (1.0, 2.0)
    seeds = r0[1:]
    assert len(set(seeds.tolist())) == len(seeds) == 6  # disjoint SPs per rank
    np.testing.assert_array_equal(r0[1:], r1[1:])


def test_failed_rank_is_reported(tmp_path):
    """A rank that raises before the collective exits non-zero; the other
    rank's collective then fails or hangs until the join timeout, and the
    launcher sees both."""
    codes = _launch(tmp_path, fail_rank=1)
    assert codes[1] != 0
