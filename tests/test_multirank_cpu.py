"""The multi-rank path on CPU (gloo, world_size 2): query points shard by
contiguous ranges with a point_base offset and no collective on the data
path, and the gathered shards equal the unsharded result bit for bit; the
benchmark's max-over-ranks timing reduction works over gloo."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIGMA = [0.02, 0.25, 1.0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import bench
    from workloads import cornell_box, surface_queries
    m = cornell_box()
    q = surface_queries(m, 100, seed=4)
    lo, hi = rank * 50, (rank + 1) * 50
    part = {k: v[lo:hi] for k, v in q.items()}
    r = O.OracleScene.from_mesh(m).bake(part, SIGMA, 8, 8, seed=3, request_id=0, point_base=lo,
                                        nthreads=1)
    flat = torch.from_numpy(np.ascontiguousarray(r["flat"]))
    parts = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(parts, flat)
    t = bench.max_over_ranks(float(rank + 1), world, torch.device("cpu"))
    if rank == 0:
        np.save(os.path.join(out_dir, "gathered.npy"), torch.cat(parts).numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_partition_equals_single_process(tmp_path):
    sys.path.insert(0, ROOT)
    import oracle as O
    from workloads import cornell_box, surface_queries
    O.build()
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "gathered.npy")
    m = cornell_box()
    q = surface_queries(m, 100, seed=4)
    whole = O.OracleScene.from_mesh(m).bake(q, SIGMA, 8, 8, seed=3, request_id=0, nthreads=1)
    assert np.array_equal(got, whole["flat"])
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0
