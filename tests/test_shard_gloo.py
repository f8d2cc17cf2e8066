"""Multi-rank host logic on CPU: two gloo ranks shard a job by frame ranges of the counter-based
generator, sum their error counters and take the slowest rank's time.  The union of the ranks'
frames must be the single-process stream, the sums and the maximum exact."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1609_09358_gb300 import inputs, shard  # noqa: E402

SEED, P, B = 1609093590, 40, 37


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard.frame_range(rank, world, B)
    pay = inputs.payload_bits(SEED, first, count, P)
    counts = shard.sum_over_ranks({"frames": count, "ones": int(pay.sum()), "rank_id": rank + 1}, dist)
    slowest = shard.max_over_ranks(10.0 + 3.5 * rank, dist)
    np.save(os.path.join(out_dir, "pay%d.npy" % rank), pay)
    with open(os.path.join(out_dir, "res%d.txt" % rank), "w") as f:
        f.write("%d %d %d %d %r\n" % (first, counts["frames"], counts["ones"], counts["rank_id"], slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_reduce():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank, args=(world, _free_port(), d), nprocs=world, join=True)
        pays = [np.load(os.path.join(d, "pay%d.npy" % r)) for r in range(world)]
        res = [open(os.path.join(d, "res%d.txt" % r)).read().split() for r in range(world)]
    whole = inputs.payload_bits(SEED, 0, world * B, P)
    assert np.array_equal(np.concatenate(pays), whole)          # disjoint ranges, same stream
    for r in range(world):
        first, frames, ones, ids, slowest = res[r]
        assert int(first) == r * B
        assert int(frames) == world * B
        assert int(ones) == int(whole.sum())
        assert int(ids) == 3
        assert float(slowest) == 13.5


def test_frame_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.frame_range(2, 2, 10)
    assert shard.frame_range(0, 1, 0) == (0, 0)
