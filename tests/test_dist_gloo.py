"""Multi-process host logic of a multi-GPU run, on CPU with gloo (world size 2):
ranks own disjoint, complete shares of the work, draw distinct inputs, and
the reported rate divides all ranks' units by the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2409_16675_gb300 import dist as hd  # noqa: E402
from paper_2409_16675_gb300 import workloads as wl  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world_size, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world_size), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    ws, r, local = hd.world()
    assert (ws, r, local) == (world_size, rank, rank)
    # each rank times its own batch; rank 1 is the slow one
    local_ms = 10.0 + 5.0 * rank
    ms = hd.reduce_max(local_ms)
    rate = hd.whole_job_rate(64 * 3, ws, ms / 1000.0)
    # the units this rank owns, and the seed of its inputs
    jobs = list(hd.shard(256, rank, ws))
    seed = hd.rank_seed(wl.MASTER_SEED, rank)
    x = wl.activations(seed, (1, 3, 8, 8))
    hd.barrier()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r\n%r\n%r\n%r\n" % (ms, rate, jobs, x.tobytes().hex()))
    dist.destroy_process_group()


def test_two_ranks_shard_seed_and_time(tmp_path):
    ctx = mp.get_context("spawn")
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = []
    for r in range(2):
        lines = open(tmp_path / ("rank%d.txt" % r)).read().splitlines()
        res.append([eval(lines[0]), eval(lines[1]), eval(lines[2]), lines[3]])
    # the max over ranks, identical on every rank
    assert res[0][0] == res[1][0] == 15.0
    # whole-job rate: both ranks' 192 images over the slowest rank's 15 ms
    assert abs(res[0][1] - 2 * 192 / 0.015) < 1e-6 and res[0][1] == res[1][1]
    # disjoint shares covering every job exactly once
    assert sorted(res[0][2] + res[1][2]) == list(range(256))
    assert not set(res[0][2]) & set(res[1][2])
    # distinct inputs per rank
    assert res[0][3] != res[1][3]


def test_shard_is_balanced_and_complete():
    for n in (0, 1, 7, 64, 255, 256):
        for w in (1, 2, 3, 4, 8):
            parts = [list(hd.shard(n, r, w)) for r in range(w)]
            assert sum(parts, []) == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1


def test_single_process_reduce_is_identity():
    assert hd.reduce_max(3.5) == 3.5
    assert hd.rank_seed(11, 0) == 11 and hd.rank_seed(11, 1) != hd.rank_seed(11, 2)
