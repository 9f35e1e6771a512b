"""Serving loop (continuous batching over resident scenes in one
device-resident kernel): every request's result is bit-identical to a
standalone bake / one-pass render of the same request (chunks keep
request-local Philox counters; render items sum the loss in the render
kernels' order), sampled served bake points
agree with the FP64 oracle, requests from several scenes share batches,
admission respects the HBM budget, waits time out instead of hanging, and a
failed launch ends every request only once none of its work is in flight."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import ETA_BAKE, bake_flat, check_bake
from workloads import cornell_box, material_params, procedural_room, shading_tables, surface_queries

pytestmark = pytest.mark.gpu
SIGMA = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
REL = 1e-4


@pytest.fixture(scope="module")
def setup():
    import paper_2304_05669_gb300 as F
    scenes = [F.Scene.from_mesh(cornell_box()), F.Scene.from_mesh(procedural_room(1))]
    meshes = [cornell_box(), procedural_room(1)]
    return F, scenes, meshes


def host_queries(F, q):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
    return F.pack_queries(t(q["x"]), t(q["n"]), t(q["wo"]), t(q["tri"])).pin_memory()


def close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.maximum(np.abs(b), np.mean(np.abs(b)) if b.size else 0.0)
    return b.size == 0 or np.max(np.abs(a - b) / np.where(scale > 0, scale, 1)) <= REL


def test_mixed_requests_equal_standalone_results(setup):
    F, scenes, meshes = setup
    srv = F.Server(256 << 20, max_batch_rays=1 << 23, chunk_points=2048)
    ids = [srv.add_scene(s) for s in scenes]
    rng = np.random.default_rng(1)
    work = []
    for j in range(14):
        sc = j % 2
        n = int(rng.choice([1, 33, 1000, 5000, 20000]))
        spp = int(rng.choice([4, 8, 16]))
        work.append((sc, host_queries(F, surface_queries(meshes[sc], n, seed=100 + j)), spp, j))
    # submitted in a burst, so the scheduler finds several requests waiting
    jobs = [(srv.submit_bake(ids[sc], qh, SIGMA, spp, spp, seed=7, request_id=j), sc, qh, spp, j)
            for sc, qh, spp, j in work]
    # render requests on a resident table
    N = 50000
    Ld, Ls0, Ls1 = [torch.from_numpy(a).cuda() for a in shading_tables(N, 6, seed=3)]
    tab = srv.add_table(Ld, Ls0, Ls1, SIGMA)
    renders = []
    for j, (first, n) in enumerate([(0, 4096), (1000, 20000), (40000, 10000)]):
        mp = material_params(n, seed=50 + j)
        gt = material_params(n, seed=60 + j)
        Lgt = (np.asarray(mp["albedo"]) * 0.5 + 0.1).astype(np.float32)
        ins = [torch.from_numpy(a).pin_memory() for a in (mp["albedo"], mp["rough"], mp["metal"], Lgt)]
        renders.append((srv.submit_render(tab, first, *ins), first, n, ins))
    oracles = [O.OracleScene.from_mesh(m) for m in meshes]
    rng_s = np.random.default_rng(2)
    for t, sc, qh, spp, j in jobs:
        assert srv.wait(t) == 0
        got = srv.result(t)
        ref = F.bake(scenes[sc], qh.cuda(), SIGMA, spp, spp, seed=7, request_id=j)
        for g, r in zip((got["Ld"], got["Ls0"], got["Ls1"]), ref):
            assert np.array_equal(g.numpy(), r.cpu().numpy())
        # sampled served points against the oracle (request-local point
        # indices in the Philox counters), compared together so the
        # tolerance's floor is the mean over the sampled points
        n = qh.shape[0]
        pick = np.unique(rng_s.integers(0, n, min(n, 8)))
        qn = qh.numpy()
        rows = {k: [] for k in ("flat", "lo", "hi", "n_amb")}
        for p in pick:
            qo = {"x": qn[p:p + 1, 0:3], "n": qn[p:p + 1, 3:6], "wo": qn[p:p + 1, 6:9],
                  "tri": qn[p:p + 1, 9].copy().view(np.int32)}
            ora = oracles[sc].bake(qo, SIGMA, spp, spp, seed=7, request_id=j, point_base=int(p),
                                   eta=ETA_BAKE)
            for k in rows:
                rows[k].append(ora[k][0])
        ora = {k: np.array(v) for k, v in rows.items()}
        g_flat = bake_flat(got["Ld"].numpy(), got["Ls0"].numpy(), got["Ls1"].numpy())[pick]
        check_bake(g_flat, ora)
    for t, first, n, ins in renders:
        assert srv.wait(t) == 0
        got = srv.result(t)
        d = [x.cuda() for x in ins]
        sl = slice(first, first + n)
        Lr, loss, (ga, gr, gm) = F.render_fwd_grad(Ld[sl], Ls0[sl], Ls1[sl], SIGMA, d[0], d[1], d[2], d[3])
        assert np.array_equal(got["Lr"].numpy(), Lr.cpu().numpy())
        assert got["loss"].item() == loss.item()
        for g, r in ((got["g_albedo"], ga), (got["g_rough"], gr), (got["g_metal"], gm)):
            assert np.array_equal(g.numpy(), r.cpu().numpy())
    st = srv.stats()
    # the resident loop ran (its launches are counted as batches) and many
    # requests had work in flight on the device at once
    assert st["batches"] >= 1 and st["max_requests_per_batch"] > 2
    assert st["peak_bytes"] <= 256 << 20 and st["bytes_in_use"] == 0
    srv.close()
    F.context().sync_status()


def test_budget_admission_and_timeouts(setup):
    F, scenes, meshes = setup
    budget = 4 << 20                      # fits one ~20k-point bake at a time
    srv = F.Server(budget, max_batch_rays=1 << 22, chunk_points=4096)
    sid = srv.add_scene(scenes[1])
    q = surface_queries(meshes[1], 20000, seed=3)
    qh = host_queries(F, q)
    tickets = [srv.submit_bake(sid, qh, SIGMA, 64, 64, seed=1, request_id=i) for i in range(4)]
    # a zero timeout on work still queued reports FIPT_ERR_TIMEOUT instead of blocking
    with pytest.raises(F.FiptError) as e:
        srv.wait(tickets[-1], timeout_s=0.0)
    assert e.value.status == 5
    # a request bigger than the whole budget completes at once with FIPT_ERR_BUDGET (4)
    big = host_queries(F, surface_queries(meshes[1], 40000, seed=4))
    tb = srv.submit_bake(sid, big, SIGMA, 4, 4)
    assert srv.wait(tb, 5.0) == 4
    for t in tickets:
        assert srv.wait(t) == 0
    ref = F.bake(scenes[1], qh.cuda(), SIGMA, 64, 64, seed=1, request_id=3)
    assert close(srv.result(tickets[3])["Ld"].numpy(), ref[0].cpu().numpy())
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    # admissions were serialised by the budget: later requests were admitted
    # only after earlier ones finished
    t0 = [srv.times(t) for t in tickets]
    assert t0[1][1] >= t0[0][2] - 1e-3
    srv.close()


def test_submit_rejects_bad_requests(setup):
    F, scenes, meshes = setup
    srv = F.Server(1 << 20)
    qh = host_queries(F, surface_queries(meshes[0], 10, seed=0))
    with pytest.raises(F.FiptError):
        srv.submit_bake(3, qh, SIGMA, 4, 4)          # unknown scene
    sid = srv.add_scene(scenes[0])
    with pytest.raises(F.FiptError):
        srv.submit_bake(sid, qh, [1.5], 4, 4)        # sigma outside (0, 1]
    srv.close()


def test_failed_launch_drains_in_flight_work(setup):
    """A launch failure (injected on the host) stops the server: requests
    whose work already ran keep their results, every other request ends with
    the error, and none is reported done while its copies or kernels are
    still queued -- its host buffers no longer change once wait returns."""
    import time
    F, scenes, meshes = setup
    srv = F.Server(1 << 30, max_batch_rays=1 << 24, chunk_points=8192)
    sid = srv.add_scene(scenes[1])
    qs = [host_queries(F, surface_queries(meshes[1], 60000, seed=70 + i)) for i in range(3)]
    srv.inject_launch_failure(2)          # the third device submission fails
    tickets = [srv.submit_bake(sid, q, SIGMA, 32, 32, seed=3, request_id=i) for i, q in enumerate(qs)]
    results = [srv.wait(t, 60.0) for t in tickets]
    assert any(r == 2 for r in results), results      # FIPT_ERR_CUDA reached the requests
    snap = [{k: v.clone() for k, v in srv.result(t).items()} for t in tickets]
    time.sleep(0.3)
    for t, s in zip(tickets, snap):                    # nothing lands after completion
        for k, v in srv.result(t).items():
            assert torch.equal(v, s[k])
    for t, r, q, i in zip(tickets, results, qs, range(3)):
        if r == 0:                                     # finished before the failure: correct
            ref = F.bake(scenes[1], q.cuda(), SIGMA, 32, 32, seed=3, request_id=i)
            assert np.array_equal(srv.result(t)["Ld"].numpy(), ref[0].cpu().numpy())
    late = srv.submit_bake(sid, qs[0][:100], SIGMA, 4, 4)
    assert srv.wait(late, 10.0) == 2                   # the stopped server takes no new work
    srv.close()
    # the device is still usable
    F.bake(scenes[1], qs[0][:1000].cuda(), SIGMA, 4, 4)
    F.context().sync_status()



def test_refused_copy_ends_only_its_request(setup):
    """A request whose copies are refused (injected on the host, as a failed
    cudaMemcpyAsync call would be) ends with FIPT_ERR_CUDA -- not with
    FIPT_OK over outputs that never arrived -- while the server and the
    requests after it go on."""
    F, scenes, meshes = setup
    srv = F.Server(1 << 30, max_batch_rays=1 << 22, chunk_points=4096)
    sid = srv.add_scene(scenes[1])
    qs = [host_queries(F, surface_queries(meshes[1], 5000, seed=90 + i)) for i in range(3)]
    srv.inject_copy_failure(0)            # the next request's input copies
    t0 = srv.submit_bake(sid, qs[0], SIGMA, 8, 8, seed=2, request_id=0)
    assert srv.wait(t0, 30.0) == 2
    srv.inject_copy_failure(1)            # the next request's output copies (its inputs are step 0)
    t1 = srv.submit_bake(sid, qs[1], SIGMA, 8, 8, seed=2, request_id=1)
    assert srv.wait(t1, 30.0) == 2
    t2 = srv.submit_bake(sid, qs[2], SIGMA, 8, 8, seed=2, request_id=2)
    assert srv.wait(t2, 30.0) == 0
    ref = F.bake(scenes[1], qs[2].cuda(), SIGMA, 8, 8, seed=2, request_id=2)
    assert np.array_equal(srv.result(t2)["Ld"].numpy(), ref[0].cpu().numpy())
    assert srv.stats()["bytes_in_use"] == 0            # the refused requests gave their space back
    srv.close()

def test_loop_wait_is_bounded():
    """The resident loop on a queue nothing publishes to ends by itself: a
    warp gives up after its bounded polls and the whole launch leaves, each
    warp's item recorded for the next launch."""
    import ctypes
    from paper_2304_05669_gb300._native import check, lib
    import paper_2304_05669_gb300 as F
    F.context()
    quit_, orphans, warps = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    secs = ctypes.c_double()
    check(lib().fipt_debug_serve_wait_bound(64, ctypes.byref(quit_), ctypes.byref(orphans),
                                            ctypes.byref(warps), ctypes.byref(secs)))
    assert quit_.value == 1
    assert 1 <= orphans.value <= warps.value
    assert secs.value < 0.5, secs.value        # 64 naps of at most ~32 us each, with margin


def test_relaunched_loop_keeps_results_identical(setup):
    """Requests that arrive after the loop has stopped for want of work start
    it again (each launch first runs the items the stopped one held); results
    stay bit-identical to standalone bakes across the relaunches."""
    import time
    F, scenes, meshes = setup
    srv = F.Server(256 << 20, max_batch_rays=1 << 22, chunk_points=4096)
    ids = [srv.add_scene(s) for s in scenes]
    runs = [(0, 3000, 8), (1, 9000, 16), (1, 70, 4), (0, 20000, 8)]
    for j, (sc, n, spp) in enumerate(runs):
        qh = host_queries(F, surface_queries(meshes[sc], n, seed=200 + j))
        t = srv.submit_bake(ids[sc], qh, SIGMA, spp, spp, seed=11, request_id=j)
        assert srv.wait(t) == 0
        ref = F.bake(scenes[sc], qh.cuda(), SIGMA, spp, spp, seed=11, request_id=j)
        for g, r in zip((srv.result(t)["Ld"], srv.result(t)["Ls0"], srv.result(t)["Ls1"]), ref):
            assert np.array_equal(g.numpy(), r.cpu().numpy())
        time.sleep(0.05)                   # the loop stops after a millisecond without work
    assert srv.stats()["batches"] >= len(runs)
    srv.close()
    F.context().sync_status()


def test_scenes_with_sky_and_voxel_cache_serve_identically(setup):
    """The loop's instances that read an environment map and a voxel radiance
    cache (scenes that carry them, served side by side with a plain scene)
    give the same bits as standalone bakes."""
    F, scenes, meshes = setup
    dev = torch.device("cuda")
    rng = np.random.default_rng(12)
    sky = F.Scene.from_mesh(cornell_box())           # open front: rays leave through it
    sky.set_environment(torch.from_numpy(rng.uniform(0, 3, (16, 32, 3)).astype(np.float32)).to(dev))
    vox = F.Scene.from_mesh(meshes[1])
    qv = surface_queries(meshes[1], 30000, seed=13)
    L = torch.from_numpy(rng.uniform(0, 2, (30000, 3)).astype(np.float32)).to(dev)
    vox.set_voxel_cache(vox.voxel_cache(torch.from_numpy(qv["x"]).to(dev), L, 32))
    both = F.Scene.from_mesh(cornell_box())
    both.set_environment(torch.from_numpy(rng.uniform(0, 1, (8, 16, 3)).astype(np.float32)).to(dev))
    qb = surface_queries(cornell_box(), 4000, seed=14)
    both.set_voxel_cache(both.voxel_cache(torch.from_numpy(qb["x"]).to(dev),
                                          torch.from_numpy(rng.uniform(0, 2, (4000, 3)).astype(np.float32)).to(dev), 16))
    trio = [(sky, cornell_box()), (vox, meshes[1]), (both, cornell_box()), (scenes[1], meshes[1])]
    srv = F.Server(256 << 20, max_batch_rays=1 << 22, chunk_points=2048)
    ids = [srv.add_scene(s) for s, _ in trio]
    jobs = []
    for j, (s, m) in enumerate(trio):
        qh = host_queries(F, surface_queries(m, 5000 + 1000 * j, seed=300 + j))
        jobs.append((srv.submit_bake(ids[j], qh, SIGMA, 8, 8, seed=5, request_id=j), s, qh, j))
    for t, s, qh, j in jobs:
        assert srv.wait(t) == 0
        ref = F.bake(s, qh.cuda(), SIGMA, 8, 8, seed=5, request_id=j)
        got = srv.result(t)
        for g, r in zip((got["Ld"], got["Ls0"], got["Ls1"]), ref):
            assert np.array_equal(g.numpy(), r.cpu().numpy())
    srv.close()
    F.context().sync_status()


def test_ragged_chunks_and_mixed_levels_serve_identically(setup):
    """Chunks that do not fill their last warp (1000-point chunks), requests
    of 1, 999, 1001 and 5000 points, and roughness grids of 2, 4 and 6
    levels in one burst: every warp item finds its own chunk's level count,
    and every result equals a standalone bake bit for bit."""
    F, scenes, meshes = setup
    srv = F.Server(256 << 20, max_batch_rays=1 << 21, chunk_points=1000)
    sid = srv.add_scene(scenes[1])
    grids = [[0.1, 0.8], [0.02, 0.3, 0.6, 1.0], SIGMA]
    jobs = []
    for j, n in enumerate([1, 999, 1001, 5000, 2500, 31]):
        g = grids[j % 3]
        qh = host_queries(F, surface_queries(meshes[1], n, seed=400 + j))
        jobs.append((srv.submit_bake(sid, qh, g, 8, 4, seed=9, request_id=j), qh, g, j))
    for t, qh, g, j in jobs:
        assert srv.wait(t) == 0
        ref = F.bake(scenes[1], qh.cuda(), g, 8, 4, seed=9, request_id=j)
        got = srv.result(t)
        assert got["Ls0"].shape[1] == len(g)
        for a, b in zip((got["Ld"], got["Ls0"], got["Ls1"]), ref):
            assert np.array_equal(a.numpy(), b.cpu().numpy())
    srv.close()
    F.context().sync_status()


def test_renders_run_in_the_loop_ahead_of_bakes(setup):
    """Render requests of 0 to 100,000 rows (item edges at multiples of 512
    rows, loss blocks of 128) go through the resident loop while a large
    bake runs: each equals the one-pass render bit for bit, loss included,
    and, as render items are taken before bake items, they finish before
    the bake does."""
    F, scenes, meshes = setup
    srv = F.Server(1 << 30, max_batch_rays=1 << 24, chunk_points=16384)
    sid = srv.add_scene(scenes[1])
    N = 120000
    Ld, Ls0, Ls1 = [torch.from_numpy(a).cuda() for a in shading_tables(N, 6, seed=21)]
    tab = srv.add_table(Ld, Ls0, Ls1, SIGMA)
    qh = host_queries(F, surface_queries(meshes[1], 200000, seed=22))
    tb = srv.submit_bake(sid, qh, SIGMA, 256, 256, seed=2, request_id=77)
    jobs = []
    for j, (first, n) in enumerate([(0, 0), (5, 1), (100, 127), (0, 128), (7, 511), (9, 512), (11, 513),
                                    (200, 1537), (1000, 4096), (20000, 100000)]):
        mp = material_params(n, seed=80 + j)
        Lgt = (np.asarray(mp["albedo"]) * 0.5 + 0.1).astype(np.float32)
        ins = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (mp["albedo"], mp["rough"], mp["metal"], Lgt)]
        jobs.append((srv.submit_render(tab, first, *ins), first, n, ins))
    for t, first, n, ins in jobs:
        assert srv.wait(t) == 0
        got = srv.result(t)
        if n == 0:
            assert got["loss"].item() == 0.0
            continue
        d = [x.cuda() for x in ins]
        sl = slice(first, first + n)
        Lr, loss, (ga, gr, gm) = F.render_fwd_grad(Ld[sl], Ls0[sl], Ls1[sl], SIGMA, d[0], d[1], d[2], d[3])
        assert np.array_equal(got["Lr"].numpy(), Lr.cpu().numpy())
        assert got["loss"].item() == loss.item()
        for g, r in ((got["g_albedo"], ga), (got["g_rough"], gr), (got["g_metal"], gm)):
            assert np.array_equal(g.numpy(), r.cpu().numpy())
    assert srv.wait(tb) == 0
    t_bake = srv.times(tb)[2]
    assert max(srv.times(t)[2] for t, _, n, _ in jobs) < t_bake
    ref = F.bake(scenes[1], qh.cuda(), SIGMA, 256, 256, seed=2, request_id=77)
    assert np.array_equal(srv.result(tb)["Ld"].numpy(), ref[0].cpu().numpy())
    srv.close()
    F.context().sync_status()
