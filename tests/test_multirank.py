"""Multi-rank host logic of the benchmark, on CPU with the gloo backend
(world size 2): the job's time is its slowest rank's, its work the sum of the
ranks' work, and an ensemble is split by whole clusters with no data-path
collective."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_clusters_is_a_balanced_partition():
    import bench
    from paper_1003_3896_gb300 import ics
    sizes = ics.ensemble_sizes(512, 256, 8192, seed=0)
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_clusters(sizes, world)
        assert len(parts) == world
        allk = np.sort(np.concatenate(parts))
        assert np.array_equal(allk, np.arange(sizes.size))     # each cluster exactly once
        loads = [float((sizes[p].astype(np.float64) ** 2).sum()) for p in parts]
        # longest-processing-time bound: no rank exceeds another by more than
        # the largest single cluster
        assert max(loads) - min(loads) <= float(sizes.max()) ** 2
        assert all(np.all(np.diff(p) > 0) for p in parts)
        again = bench.shard_clusters(sizes, world)
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    assert bench.rank_env() == (world, rank, rank)
    t = 10.0 + 5.0 * rank            # rank 1 is the slower one
    work = 100.0 * (rank + 1)
    tmax = bench.max_over_ranks(t)
    wsum = bench.sum_over_ranks(work)
    # each rank integrates its own cluster: seeds differ, no data exchanged
    pos, _, m, _ = bench.workload(64, seed=rank)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([tmax, wsum, pos[0, 0], m.sum()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reductions_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 15.0          # max over ranks
    assert r0[1] == r1[1] == 300.0         # sum over ranks
    assert r0[2] != r1[2]                  # independent clusters per rank
    assert abs(r0[3] - 1.0) < 1e-12 and abs(r1[3] - 1.0) < 1e-12


def test_single_process_reductions_are_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.sum_over_ranks(2.0) == 2.0
