"""The multi-rank path on CPU (gloo, world_size 2): query points shard by
contiguous ranges with a point_base offset and no collective on the data
path, and the gathered shards equal the unsharded result bit for bit; the
render loss and the per-triangle error, sums over all pixels, come out of
one all-reduce each equal to the unsharded sums; the benchmark's
max-over-ranks timing reduction works over gloo.  (The ranks' local
results come from the oracle here: there is no GPU.)"""
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


def _sums_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_2304_05669_gb300.sharded import global_loss, global_tri_error, shard_range
    from workloads import material_params, shading_tables
    P, T = 10007, 321
    rng = np.random.default_rng(7)
    tri = rng.integers(-1, T, P).astype(np.int32)
    Ld, Ls0, Ls1 = shading_tables(P, 3, seed=8)
    mp_, gt = material_params(P, seed=9), material_params(P, seed=10)
    Lgt, _ = O.render_forward(Ld, Ls0, Ls1, SIGMA, gt["albedo"], gt["rough"], gt["metal"])
    lo, hi = shard_range(P, rank, world)
    sl = slice(lo, hi)
    Lr, loss = O.render_forward(Ld[sl], Ls0[sl], Ls1[sl], SIGMA, mp_["albedo"][sl], mp_["rough"][sl],
                                mp_["metal"][sl], Lgt[sl])
    err, cnt = O.tri_error(tri[sl], Lr, Lgt[sl], T)
    loss_t = torch.tensor([loss], dtype=torch.float64)
    err_t = torch.from_numpy(np.ascontiguousarray(err, np.float64))
    cnt_t = torch.from_numpy(np.ascontiguousarray(cnt, np.int32))
    global_loss(loss_t)
    global_tri_error(err_t, cnt_t)
    np.save(os.path.join(out_dir, "sums%d.npy" % rank),
            np.concatenate([loss_t.numpy(), err_t.numpy(), cnt_t.numpy().astype(np.float64)]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_once():
    sys.path.insert(0, ROOT)
    from paper_2304_05669_gb300.sharded import shard_range
    for N in (0, 1, 7, 100, 1 << 20):
        for W in (1, 2, 3, 8):
            r = [shard_range(N, k, W) for k in range(W)]
            assert r[0][0] == 0 and r[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1


def test_two_rank_loss_and_tri_error_sums(tmp_path):
    sys.path.insert(0, ROOT)
    import oracle as O
    from workloads import material_params, shading_tables
    O.build()
    mp.start_processes(_sums_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    P, T = 10007, 321
    rng = np.random.default_rng(7)
    tri = rng.integers(-1, T, P).astype(np.int32)
    Ld, Ls0, Ls1 = shading_tables(P, 3, seed=8)
    mp_, gt = material_params(P, seed=9), material_params(P, seed=10)
    Lgt, _ = O.render_forward(Ld, Ls0, Ls1, SIGMA, gt["albedo"], gt["rough"], gt["metal"])
    Lr, loss = O.render_forward(Ld, Ls0, Ls1, SIGMA, mp_["albedo"], mp_["rough"], mp_["metal"], Lgt)
    err, cnt = O.tri_error(tri, Lr, Lgt, T)
    want = np.concatenate([[loss], err, cnt.astype(np.float64)])
    for r in range(2):
        got = np.load(tmp_path / ("sums%d.npy" % r))
        assert np.array_equal(got[1 + T:], want[1 + T:])                 # counts exact
        assert np.allclose(got[:1 + T], want[:1 + T], rtol=1e-12, atol=0)
