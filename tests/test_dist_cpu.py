"""The multi-rank plumbing of bench.py (replicas only: rank 0 builds the workload and hands it to
the other ranks, timings are reduced with a max over ranks) on two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class A:
        workload = "circle"
        scale = 1.0

    sc = bench.load_scene(A, rank, world)
    m = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    bench.barrier(world)
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), uv=sc.uv, cam_idx=sc.cam_idx, m=m)
    dist.destroy_process_group()


def test_two_rank_replicas(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    a, b = np.load(tmp_path / "r0.npz"), np.load(tmp_path / "r1.npz")
    np.testing.assert_array_equal(a["uv"], b["uv"])
    np.testing.assert_array_equal(a["cam_idx"], b["cam_idx"])
    assert float(a["m"]) == 3.0 and float(b["m"]) == 3.0
