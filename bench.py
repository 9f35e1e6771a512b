#!/usr/bin/env python
"""Benchmark of the factorized shading-term bake hot path on one GB300.

Workload (default): the 2,045,464-triangle building floor (four rooms), 16
pinhole views at 512x512 whose first 2^22 hits are the query points, 256
samples per point for L_d and for each of the 6 roughness levels of
L_s0/L_s1.  ``--workload room`` selects the ~176k-triangle procedural room
(24 views at 320x208, first 2^20 hits, 128 spp).  One step runs the whole
path on device-resident inputs:

  scene build (bounds, Morton, radix sort, Karras tree, pack, refit,
  treelet restructuring, depth-first relayout)
  -> pinhole first hits -> compaction to N queries
  -> bake of L_d, L_s0, L_s1 (N * S * (1 + K) rays: 7,516,192,768 on the floor)
  -> factorized render forward (+ tone-mapped loss) and backward
  -> per-triangle rendering error.

value = rays per step / step time (Mrays/s); L2 is flushed between steps.
The e2e figure repeats the steps through the same public calls with the
inputs copied from pinned host memory and the tables, loss, gradients and
per-triangle error copied back, all inside the timed region.
``--impl reference`` times the FP64 CPU oracle on a bounded sample.

Run under torchrun for N > 1: every rank bakes its own batch (its own
Philox request id), no collective on the data path; rank 0 prints one
JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Mrays/s and shading-term points/s at 1e-4 rel. vs oracle; "
          "served p50/p99 bake latency")
SIGMA = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
WORKLOADS = {
    # name: scene, views, W, H, N, spp_d, spp_s, scene seed, view seed
    "room": dict(scene="room", views=24, W=320, H=208, N=1 << 20, spp_d=128, spp_s=128, cpu_points=16384,
                 desc="procedural room 175,926 tris; 24 views 320x208; first 2^20 hits; "
                      "128 spp; 6-level roughness grid"),
    "cornell": dict(scene="cornell", views=4, W=64, H=64, N=4096, spp_d=64, spp_s=64, surface=True,
                    cpu_points=4096,
                    desc="Cornell box 36 tris; 4096 points uniform on surfaces (seed 0); 64 spp"),
    "floor": dict(scene="floor", views=16, W=512, H=512, N=1 << 22, spp_d=256, spp_s=256, cpu_points=4096,
                  desc="building floor 2,045,464 tris; 16 views 512x512; 2^22 hits; 256 spp"),
    # the differentiation config: factorized render forward (+ loss) and
    # backward over 24 views at 640x416 with synthetic shading tables
    "render": dict(scene=None, views=24, W=640, H=416, N=24 * 640 * 416, spp_d=128, spp_s=64,
                   desc="factorized render fwd+bwd, room 175,926 tris, 24 views 640x416 = "
                        "6,389,760 pixels, tables baked once at 128/64 spp, 6-level roughness grid"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="floor", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-points", type=int, default=None,
                    help="points in the CPU-oracle sample (cpu_baseline; default: 4096 on the "
                         "floor, 16384 on the room)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--points", type=int, default=None,
                    help="override the query count (small profiling cases)")
    ap.add_argument("--spp", type=int, default=None, help="override both sample counts")
    ap.add_argument("--serve-requests", type=int, default=500,
                    help="requests in the serving trace (0 = skip the serving measurement)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, req/s")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0, help="HBM admission budget")
    ap.add_argument("--refine-points", type=int, default=1 << 18,
                    help="points of the stage-3 refinement measurement (0 = skip)")
    ap.add_argument("--refine-spp", type=int, default=32)
    ap.add_argument("--next-spp", type=int, default=32,
                    help="spp of the voxel-cache / environment bakes (0 = skip those rows)")
    return ap.parse_args()


def make_scene(name):
    from workloads import building_floor, cornell_box, procedural_room
    if name == "room":
        return procedural_room(1)
    if name == "cornell":
        return cornell_box()            # open front, as the 36-triangle config states
    return building_floor(5)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_sm_max():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def _code_only(text):
    """C/CUDA source without its comments and whitespace (string literals are
    kept), so that the digest changes with the code and not with its notes."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif c.isspace():
            i += 1
        else:
            out.append(c)
            i += 1
    return "".join(out)


def source_digest():
    """Digest of the bake kernel's code and of the tree it walks (trace.cu,
    fipt_internal.cuh, lbvh.cu, comments and whitespace left out): recorded
    ncu counters are used only while it matches."""
    h = hashlib.sha256()
    for f in ("trace.cu", "fipt_internal.cuh", "lbvh.cu"):
        with open(os.path.join(ROOT, "paper_2304_05669_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode("utf-8"))
    return h.hexdigest()[:16]


def recorded_profile(workload):
    """The bake kernel's counters from the committed ncu summary (DRAM bytes
    per ray, issue-slot activity, L2 hit rate, active lanes per warp
    instruction), or None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "bake_%s_traffic.json" % workload)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_digest") != source_digest():
        return None
    return d


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def _once(self):
        """One synchronous query (brackets timed regions shorter than the loop's period)."""
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits"],
                                 capture_output=True, text=True, timeout=20).stdout
            self.lines.extend(l.strip() for l in out.splitlines() if l.strip())
        except Exception:
            pass

    def __enter__(self):
        self._once()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        self._once()

    def summary(self):
        rows = []
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1]:
                continue
            rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        pw = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle
def oracle_sample(mesh, cams, W, H, npts, spp_d, spp_s, request_id=0, surface=False):
    """Oracle first hits of the first pixels (view-major order), then the
    oracle bake of the first ``npts`` valid points (surface workloads:
    ``npts`` seeded surface points of the same distribution).
    Returns (rays, seconds, threads, points)."""
    import oracle as O
    S = O.OracleScene.from_mesh(mesh)
    if surface:
        from workloads import surface_queries
        sq = surface_queries(mesh, npts, seed=0)
        q = {k: sq[k] for k in ("x", "n", "wo", "tri")}
        ok = np.arange(npts)
    else:
        pix = np.arange(min(len(cams) * W * H, int(npts * 1.5) + 64))
        cq = S.camera_queries(cams, W, H, pix)
        ok = np.nonzero(cq["tri"] >= 0)[0][:npts]
        q = {"x": cq["x"][ok].astype(np.float32), "n": cq["n"][ok].astype(np.float32),
             "wo": cq["wo"][ok].astype(np.float32), "tri": cq["tri"][ok].astype(np.int32)}
    threads = O.default_threads()
    t0 = time.perf_counter()
    S.bake(q, SIGMA, spp_d, spp_s, seed=0, request_id=request_id, nthreads=threads)
    dt = time.perf_counter() - t0
    rays = len(ok) * (spp_d + len(SIGMA) * spp_s)
    return rays, dt, threads, len(ok)


def run_reference_render(args, wl, world):
    """The oracle's render forward + loss + analytic gradient on a bounded
    sample of the render workload's size (the tables are drawn by the
    shading-table generator: the arithmetic does not depend on their values
    and the reference arm has no GPU bake to take them from)."""
    import oracle as O
    from workloads import material_params, shading_tables
    n = 1 << 18
    Ld, Ls0, Ls1 = shading_tables(n, K=len(SIGMA), seed=7)
    mp, gt = material_params(n, seed=3), material_params(n, seed=4)
    Lgt = O.render_forward(Ld, Ls0, Ls1, SIGMA, gt["albedo"], gt["rough"], gt["metal"])[0]

    def one():
        O.render_forward(Ld, Ls0, Ls1, SIGMA, mp["albedo"], mp["rough"], mp["metal"], Lgt)
        O.render_grad(Ld, Ls0, Ls1, SIGMA, mp["albedo"], mp["rough"], mp["metal"], Lgt)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    v = n * args.steps / dt / 1e6
    sample = "first %d pixels per step, forward + loss + analytic gradient, numpy FP64" % n
    print(json.dumps({
        "impl": "reference", "metric": "factorized render fwd+bwd pixels/s", "value": round(v, 4),
        "unit": "Mpixels/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": render_config(wl, world),
        "cpu_baseline": {"value": round(v, 4), "unit": "Mpixels/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "Mpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_reference(args, wl, world, rank):
    if rank != 0:
        return
    if wl["scene"] is None:
        run_reference_render(args, wl, world)
        return
    mesh = make_scene(wl["scene"])
    from workloads import pinhole_views
    cams = pinhole_views(mesh, wl["views"], seed=2)
    npts = max(64, min(args.cpu_points, 2048))
    for _ in range(args.warmup):
        oracle_sample(mesh, cams, wl["W"], wl["H"], 64, wl["spp_d"], wl["spp_s"],
                      surface=wl.get("surface", False))
    tot_rays, tot_t, threads, n = 0, 0.0, 1, 0
    for s in range(args.steps):
        r, dt, threads, n = oracle_sample(mesh, cams, wl["W"], wl["H"], npts, wl["spp_d"],
                                          wl["spp_s"], request_id=s, surface=wl.get("surface", False))
        tot_rays += r
        tot_t += dt
    v = tot_rays / tot_t / 1e6
    sample = "%d oracle query points (%s) per step, %d+6x%d spp, FP64" % (
        n, "surface points" if wl.get("surface") else "first hits of view 0", wl["spp_d"], wl["spp_s"])
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "Mrays/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bake_config(wl, mesh.T, world),
        "cpu_baseline": {"value": round(v, 4), "unit": "Mrays/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------- render workload
def render_config(wl, world):
    return {"workload": wl["desc"], "pixels": wl["N"], "roughness_levels": len(SIGMA),
            "scene_tris": 175926, "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "flushed between steps (512 MB write outside the timed events)"}


# one pass: Ld, the two specular rows (K = 6), albedo, rough, metal, Lgt and
# the emitter mask in; Lr and the three gradients out
RENDER_BYTES_PER_PX = (12 + 72 + 72 + 12 + 4 + 4 + 12 + 1) + (12 + 12 + 4 + 4)


def run_render(args, wl, world, rank, local):
    """Factorized render fwd (Eq. 5, 8, with the Eq. 14 loss) and backward
    over the first hits of 24 640x416 views of the room, whose shading
    tables are baked once (untimed) at 128 diffuse / 64 specular spp.
    value = pixels / step time."""
    import torch
    import paper_2304_05669_gb300 as F
    from paper_2304_05669_gb300._native import lib
    from workloads import material_params, pinhole_views
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mesh = make_scene("room")
    sc = F.Scene.from_mesh(mesh, device=dev)
    cams = torch.from_numpy(pinhole_views(mesh, wl["views"], seed=2)).to(dev)
    qa, valid = sc.camera_queries(cams, wl["W"], wl["H"])
    q, _pix, nv = F.compact_queries(qa, valid, wl["N"])
    N = int(nv.item())
    tabs = F.bake(sc, q[:N], SIGMA, wl["spp_d"], wl["spp_s"], seed=0, request_id=rank)
    F.context().sync_status()
    Ld, Ls0, Ls1 = (t.cpu().numpy() for t in tabs)
    # pixels whose first hit is an emitter are left out of the loss (an input, built once)
    tri = q[:N, 9].contiguous().view(torch.int32).cpu().numpy()
    mask = (~mesh.emitter[tri]).astype(np.uint8)
    del q, qa, valid, tabs
    mp, gt = material_params(N, seed=3), material_params(N, seed=4)
    host = {"Ld": Ld, "Ls0": Ls0, "Ls1": Ls1, "albedo": mp["albedo"], "rough": mp["rough"],
            "metal": mp["metal"], "mask": mask}
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
    d = {k: v.to(dev) for k, v in pinned.items()}
    gtd = {k: torch.from_numpy(v).to(dev) for k, v in gt.items()}
    Lgt = F.render_fwd(d["Ld"], d["Ls0"], d["Ls1"], SIGMA, gtd["albedo"], gtd["rough"], gtd["metal"])[0]
    Lgt_host = Lgt.cpu().pin_memory()
    stream = torch.cuda.current_stream()

    one = torch.ones(1, dtype=torch.float64, device=dev)     # d(step loss) / d(loss)

    def step(x, lg):
        # forward, loss and gradient in one pass over the inputs, then the
        # upstream gradient applied (the library's backward of the loss)
        Lr, loss, g = F.render_fwd_grad(x["Ld"], x["Ls0"], x["Ls1"], SIGMA, x["albedo"], x["rough"],
                                        x["metal"], lg, x["mask"])
        F.render_grad_scale(g, one)
        return loss, g

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        step(d, Lgt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    launches0 = lib().fipt_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            step(d, Lgt)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = lib().fipt_launch_count() - launches0
    ms = [a.elapsed_time(b) for a, b in ev]
    t_total = max_over_ranks(sum(ms) / 1e3, world, dev)
    F.context().sync_status()
    # e2e: tables, parameters and targets copied in, loss and gradients copied out
    e2e = None
    if not args.no_e2e:
        h2d = sum(v.numel() * v.element_size() for v in pinned.values()) + Lgt_host.numel() * 4
        out_host = None
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d2h = 0
        for s in range(args.steps):
            x = {k: v.to(dev, non_blocking=True) for k, v in pinned.items()}
            lg = Lgt_host.to(dev, non_blocking=True)
            loss, g = step(x, lg)
            res = [loss, g[0], g[1], g[2]]
            if out_host is None:
                out_host = [torch.empty(r.shape, dtype=r.dtype, pin_memory=True) for r in res]
            for h, r in zip(out_host, res):
                h.copy_(r, non_blocking=True)
            d2h = sum(r.numel() * r.element_size() for r in res)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
        e2e = {"value": round(world * N * args.steps / t_e2e / 1e6, 3), "unit": "Mpixels/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        n = 1 << 20
        sl = slice(0, n)
        t0 = time.perf_counter()
        O.render_forward(Ld[sl], Ls0[sl], Ls1[sl], SIGMA, mp["albedo"][sl], mp["rough"][sl], mp["metal"][sl],
                         Lgt_host.numpy()[sl], mask[sl])
        O.render_grad(Ld[sl], Ls0[sl], Ls1[sl], SIGMA, mp["albedo"][sl], mp["rough"][sl], mp["metal"][sl],
                      Lgt_host.numpy()[sl], mask[sl])
        dt = time.perf_counter() - t0
        cpu = {"value": round(n / dt / 1e6, 4), "unit": "Mpixels/s", "cores": 1, "kind": "oracle",
               "sample": "first %d pixels, forward + loss + analytic gradient, numpy FP64, %.1f s" % (n, dt)}
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    step_s = t_total / args.steps
    achieved = RENDER_BYTES_PER_PX * N / step_s / 1e9
    print(json.dumps({
        "metric": "factorized render fwd+bwd pixels/s", "value": round(world * N * args.steps / t_total / 1e6, 3),
        "unit": "Mpixels/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * step_s, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": render_config(wl, world),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "k_render_fwd_grad + k_render_grad_scale", "peak_kind": peak_kind,
                     "alg_bytes_per_pixel": RENDER_BYTES_PER_PX},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
    }))


# ---------------------------------------------------------------- serving
def run_serving(args, F, dev):
    """Poisson trace of bake and render requests over four resident scenes
    (the 36-triangle Cornell box, the 175,926-triangle room, two rooms of the
    floor at 1,022,732 triangles and the 2,045,464-triangle floor), served
    with continuous batching, then the same trace one request at a time,
    then the trace slowed to a sustainable rate (utilisation 0.7 of the
    serial service time)."""
    import torch
    from workloads import (building_floor, cornell_box, material_params, pinhole_views,
                           procedural_room, shading_tables)
    rng = np.random.default_rng(6)
    meshes = [cornell_box(), procedural_room(1), building_floor(5, rooms=2),
              building_floor(5, rooms=4)]
    scenes = [F.Scene.from_mesh(m) for m in meshes]
    # query pools: pinhole first hits of each scene, kept in pinned host memory
    pools = []
    for m, sc in zip(meshes, scenes):
        cams = torch.from_numpy(pinhole_views(m, 16, seed=8)).to(dev)
        qa, valid = sc.camera_queries(cams, 512, 256)
        q, _pix, n = F.compact_queries(qa, valid, 2_000_000)
        pools.append(q[:int(n.item())].cpu().pin_memory())
    tab_n = 266_240
    tabs = [torch.from_numpy(a).to(dev) for a in shading_tables(tab_n, len(SIGMA), seed=9)]
    mp = material_params(tab_n, seed=10)
    params = [torch.from_numpy(mp[k]).pin_memory() for k in ("albedo", "rough", "metal")]
    Lgt = torch.from_numpy(mp["albedo"] * 0.5 + 0.05).pin_memory()
    trace = []
    t = 0.0
    for i in range(args.serve_requests):
        t += rng.exponential(1.0 / args.serve_rate)
        sc = int(rng.integers(0, 4))
        if rng.random() < 0.5:
            pool = pools[sc]
            n = int(min(len(pool), np.exp(rng.uniform(np.log(1e3), np.log(2e6)))))
            spp = int(rng.choice([16, 64, 256]))
            off = int(rng.integers(0, len(pool) - n + 1))
            trace.append(("bake", t, sc, off, n, spp, i))
        else:
            n = int(np.exp(rng.uniform(np.log(4096), np.log(266_240))))
            first = int(rng.integers(0, tab_n - n + 1))
            trace.append(("render", t, 0, first, n, 0, i))
    bake_rays = sum(r[4] * r[5] * (1 + len(SIGMA)) for r in trace if r[0] == "bake")

    def serve(serial, tr):
        srv = F.Server(int(args.serve_budget_gb * (1 << 30)))
        sids = [srv.add_scene(s) for s in scenes]
        tid = srv.add_table(*tabs, SIGMA)

        def submit(r):
            kind, _t, sc, off, n, spp, i = r
            if kind == "bake":
                return srv.submit_bake(sids[sc], pools[sc][off:off + n], SIGMA, spp, spp,
                                       seed=0, request_id=i)
            sl = slice(off, off + n)
            return srv.submit_render(tid, off, params[0][sl], params[1][sl], params[2][sl], Lgt[sl])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for r in tr:
            if serial:
                tk = submit(r)
                if srv.wait(tk) != 0:
                    raise RuntimeError("request failed")
                tickets.append(tk)
            else:
                delay = t0 + r[1] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(submit(r))
        for tk in tickets:
            if srv.wait(tk) != 0:
                raise RuntimeError("request failed")
        wall = time.perf_counter() - t0
        lat = [srv.times(tk)[2] - srv.times(tk)[0] for tk in tickets]
        st = srv.stats()
        srv.close()
        return wall, lat, st

    wall_b, lat_b, st_b = serve(False, trace)
    wall_s, lat_s, _ = serve(True, trace)
    # a sustainable arrival rate: utilisation 0.7 of the serial service time
    lam = 0.7 * len(trace) / wall_s
    scale = args.serve_rate / lam
    trace_s = [(r[0], r[1] * scale) + tuple(r[2:]) for r in trace]
    wall_u, lat_u, _ = serve(False, trace_s)
    return {"requests": len(trace), "rate_per_s": args.serve_rate,
            "budget_gb": args.serve_budget_gb,
            "scenes_tris": [m.T for m in meshes],
            "p50_ms": round(1e3 * float(np.percentile(lat_b, 50)), 2),
            "p99_ms": round(1e3 * float(np.percentile(lat_b, 99)), 2),
            "mrays_per_s_batched": round(bake_rays / wall_b / 1e6, 2),
            "mrays_per_s_serial": round(bake_rays / wall_s / 1e6, 2),
            "serial_p50_ms": round(1e3 * float(np.percentile(lat_s, 50)), 2),
            "wall_s_batched": round(wall_b, 3), "wall_s_serial": round(wall_s, 3),
            "batches": int(st_b["batches"]),
            "max_requests_per_batch": int(st_b["max_requests_per_batch"]),
            "sustainable": {"rate_per_s": round(lam, 2), "utilisation": 0.7,
                            "p50_ms": round(1e3 * float(np.percentile(lat_u, 50)), 2),
                            "p99_ms": round(1e3 * float(np.percentile(lat_u, 99)), 2),
                            "wall_s": round(wall_u, 3),
                            "mrays_per_s": round(bake_rays / wall_u / 1e6, 2)},
            "note": "latency = completion - submission (host steady clock); "
                    "serial = same trace, one request at a time, no arrival gaps"}


# ---------------------------------------------------------------- stage-3 refinement
def refine_materials(mesh, seed=11):
    """Per-triangle stage-2-like materials: albedo U[0,1]^3, roughness
    U[0.02,1] (so ~60% of surfaces continue paths at sigma_c = 0.6),
    metallic U[0,1]."""
    rng = np.random.default_rng(seed)
    T = mesh.T
    return (rng.uniform(0, 1, (T, 3)).astype(np.float32),
            rng.uniform(0.02, 1.0, T).astype(np.float32),
            rng.uniform(0, 1, T).astype(np.float32))


def run_refine(args, F, dev, mesh, sc, q_all, with_cpu):
    """Stage-3 path-traced refinement (Sec. 4.3, Eq. 10, MIS) of the first
    --refine-points queries at --refine-spp, timed with CUDA events."""
    import torch
    N, S = args.refine_points, args.refine_spp
    a, r, m = refine_materials(mesh)
    sc.set_materials(*[torch.from_numpy(x).to(dev) for x in (a, r, m)])
    q = q_all[:N].contiguous()
    for _ in range(2):
        F.bake_refine(sc, q, SIGMA, S, S)
    torch.cuda.synchronize()
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        F.bake_refine(sc, q, SIGMA, S, S)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    st = torch.zeros(4, dtype=torch.int64, device=dev)     # instrumented, untimed
    F.bake_refine(sc, q, SIGMA, S, S, stats=st)
    F.context().sync_status()
    n_rays, n_nodes, n_tris, max_sp = [int(x) for x in st.cpu().tolist()]
    t = float(np.median(ts))
    samples = N * S * (1 + len(SIGMA))
    alg = 64.0 * n_nodes + 48.0 * n_tris + 24.0 * n_rays + N * (40 + 12 * (1 + 2 * len(SIGMA)))
    peak, peak_kind = measured_peaks()
    out = {"points": N, "spp": S, "sigma_c": 0.6, "max_depth": 8, "mis": True,
           "ms": round(1e3 * t, 3),
           "msamples_per_s": round(samples / t / 1e6, 2),
           "points_per_s": round(N / t, 1),
           "rays_per_sample": round(n_rays / samples, 3), "mrays_per_s": round(n_rays / t / 1e6, 1),
           "nodes_per_ray": round(n_nodes / max(n_rays, 1), 2), "max_stack": max_sp,
           "roofline": {"bound": "l1l2_algorithmic", "achieved": round(alg / t / 1e9, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(alg / t / 1e9 / peak, 4), "peak_kind": peak_kind,
                        "kernel": "whole call: k_rf_gen, k_rf_trace, k_rf_shade, k_rf_reduce",
                        "note": "algorithmic node + triangle + gather + path-state bytes / call time; the "
                                "traversal (75 % of the call) is served by L1/L2 and bound by issue"}}
    if with_cpu:
        import oracle as O
        cams = pinhole_views_for(mesh)
        S_o = O.OracleScene.from_mesh(mesh)
        npts = 1024
        cq = S_o.camera_queries(cams, 320, 208, np.arange(int(npts * 1.5)))
        ok = np.nonzero(cq["tri"] >= 0)[0][:npts]
        qo = {k: cq[k][ok].astype(np.float32 if k != "tri" else np.int32)
              for k in ("x", "n", "wo", "tri")}
        t0 = time.perf_counter()
        S_o.refine(qo, SIGMA, S, S, a, r, m, nthreads=O.default_threads())
        dt = time.perf_counter() - t0
        out["cpu_oracle_msamples_per_s"] = round(len(ok) * S * (1 + len(SIGMA)) / dt / 1e6, 4)
        out["cpu_oracle_sample"] = "%d oracle first hits, %d spp, %d threads, %.1f s" % (
            len(ok), S, O.default_threads(), dt)
    return out


# ---------------------------------------------------------------- next rows (f2-f4)
def _device_time(fn, reps=5, warm=2):
    """Median CUDA-event seconds of fn() on the current stream."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(ts))


def _sort_passes(bits):
    return (bits + 7) // 8


def run_next_rows(args, F, dev, mesh, sc, q, Lgt, qa, with_cpu, peak):
    """Voxel radiance cache (Sec. 4.2), environment light (Sec. 8 window
    light) and emitter extraction (Sec. 4.4, Eq. 12), each timed with CUDA
    events (median of 5) on the benchmark's scene, with its algorithmic
    bytes against the measured HBM copy rate and the FP64 oracle timed on a
    sample beside it."""
    import torch
    out = {}
    N = q.shape[0]
    K = len(SIGMA)
    spp = args.next_spp

    def bake_rate(scene, qq, stats_too=True):
        t = _device_time(lambda: F.bake(scene, qq, SIGMA, spp, spp, seed=5), reps=3, warm=1)
        rays = qq.shape[0] * spp * (1 + K)
        st = torch.zeros(4, dtype=torch.int64, device=dev)
        F.bake(scene, qq, SIGMA, spp, spp, seed=5, stats=st)
        n_rays, n_nodes, n_tris, _ = [int(x) for x in st.cpu().tolist()]
        alg = 64.0 * n_nodes + 48.0 * n_tris + 24.0 * n_rays + qq.shape[0] * (40 + 12 * (1 + 2 * K))
        return t, rays, alg

    # ---- f3: voxel cache over the N pixels' first hits and radiance
    R = 256
    grid = sc.voxel_cache(q, Lgt, R)
    t_pool = _device_time(lambda: sc.voxel_cache(q, Lgt, R))
    nonempty = int((grid[..., 3] > 0).sum().item())
    bits = max(8, int(np.ceil(np.log2(R ** 3))))
    pool_bytes = 16.0 * R ** 3 + N * (24 + 8 + 24 * _sort_passes(bits) + 20) + 16.0 * nonempty
    t_plain, rays, _ = bake_rate(sc, q)
    sc.set_voxel_cache(grid)
    t_vox, _, alg_vox = bake_rate(sc, q)
    sc.set_voxel_cache(None)
    vox = {"R": R, "pixels": N, "nonempty_voxels": nonempty,
           "pool_ms": round(1e3 * t_pool, 3), "pool_mpixels_per_s": round(N / t_pool / 1e6, 1),
           "pool_alg_bytes": int(pool_bytes),
           "pool_roofline": {"bound": "hbm", "achieved": round(pool_bytes / t_pool / 1e9, 1),
                             "peak": peak, "unit": "GB/s",
                             "frac": round(pool_bytes / t_pool / 1e9 / peak, 4)},
           "bake_spp": spp, "bake_plain_mrays_per_s": round(rays / t_plain / 1e6, 1),
           "bake_voxel_mrays_per_s": round(rays / t_vox / 1e6, 1),
           "bake_voxel_cache_served_frac": round(alg_vox / t_vox / 1e9 / peak, 4)}
    # ---- f4: environment map, open Cornell box (rays leave through the front)
    from workloads import cornell_box, surface_queries
    cb = cornell_box()
    scb = F.Scene.from_mesh(cb, device=dev)
    nq = 1 << 20
    sq = surface_queries(cb, nq, seed=12)
    qc = F.pack_queries(*[torch.from_numpy(np.ascontiguousarray(sq[k])).to(dev)
                          for k in ("x", "n", "wo", "tri")])
    rng = np.random.default_rng(13)
    env = torch.from_numpy(rng.uniform(0, 3, (512, 1024, 3)).astype(np.float32)).to(dev)
    t_noenv, rays_c, _ = bake_rate(scb, qc)
    scb.set_environment(env)
    t_env, _, alg_env = bake_rate(scb, qc)
    envr = {"scene": "open Cornell box 36 tris", "points": nq, "spp": spp, "env": [512, 1024],
            "bake_without_env_mrays_per_s": round(rays_c / t_noenv / 1e6, 1),
            "bake_env_mrays_per_s": round(rays_c / t_env / 1e6, 1),
            "bake_env_cache_served_frac": round(alg_env / t_env / 1e9 / peak, 4)}
    # ---- f2: emitter extraction on the benchmark scene
    n_per = 100
    T = mesh.T
    Pq = qa.shape[0]
    rgb = torch.rand((Pq, 3), device=dev, generator=torch.Generator(device=dev).manual_seed(14)) * 4

    def alpha_fn(x):
        return (x[:, 1] > 2.9).float() * 0.05

    pts = sc.emitter_points(n_per)
    alpha = alpha_fn(pts)
    t_pts = _device_time(lambda: sc.emitter_points(n_per))
    t_cls = _device_time(lambda: F.emitter_classify(alpha, n_per, 0.01))
    flag, _ = F.emitter_classify(alpha, n_per, 0.01)
    t_rad = _device_time(lambda: F.emitter_radiance(qa, rgb, flag))
    M = int(F.emitter_radiance(qa, rgb, flag)[1].sum().item())     # pixels on emitter triangles
    # triangle id + flag per pixel in the count and scatter passes; per
    # emitter pixel its rgb, the three key rows and four 8-bit selection
    # passes over them; per triangle its count, segment, L_e and pixel count
    rad_bytes = Pq * 2 * (4 + 1) + M * (12 + 12 + 3 * 4 * 4) + T * (4 + 8 + 12 + 4)
    b_pts = 12.0 * T * n_per + 52.0 * T
    b_cls = 4.0 * T * n_per + 9.0 * T
    em = {"triangles": T, "samples_per_triangle": n_per, "pixels": Pq,
          "emitters_found": int(flag.sum().item()), "emitter_pixels": M,
          "points_ms": round(1e3 * t_pts, 3), "classify_ms": round(1e3 * t_cls, 3),
          "radiance_ms": round(1e3 * t_rad, 3),
          "points_roofline_frac": round(b_pts / t_pts / 1e9 / peak, 4),
          "classify_roofline_frac": round(b_cls / t_cls / 1e9 / peak, 4),
          "radiance_roofline_frac": round(rad_bytes / t_rad / 1e9 / peak, 4),
          "radiance_mpixels_per_s": round(Pq / t_rad / 1e6, 1)}
    if with_cpu:
        import oracle as O
        S = O.OracleScene.from_mesh(mesh)
        xh = q[:, :3].cpu().numpy().copy()
        Lh = Lgt.cpu().numpy()
        t0 = time.perf_counter()
        S.voxel_pool(xh, Lh, R)
        vox["cpu_oracle_pool_mpixels_per_s"] = round(N / (time.perf_counter() - t0) / 1e6, 2)
        t0 = time.perf_counter()
        S.emitter_points(n_per)
        em["cpu_oracle_points_ms"] = round(1e3 * (time.perf_counter() - t0), 1)
        ah = alpha.cpu().numpy()
        t0 = time.perf_counter()
        fo, _ = O.emitter_classify(ah, n_per, 0.01)
        em["cpu_oracle_classify_ms"] = round(1e3 * (time.perf_counter() - t0), 1)
        trih = qa[:, 9].contiguous().view(torch.int32).cpu().numpy()
        rgbh = rgb.cpu().numpy()
        t0 = time.perf_counter()
        O.emitter_radiance(trih, rgbh, fo)
        em["cpu_oracle_radiance_ms"] = round(1e3 * (time.perf_counter() - t0), 1)
        em["cpu_oracle_threads"] = 1
        vox["cpu_oracle_threads"] = 1
    F.context().sync_status()
    out["voxel_cache"] = vox
    out["environment"] = envr
    out["emitter_extraction"] = em
    return out


def bake_config(wl, scene_tris, world):
    """The workload description both arms print (identical dicts, so the
    two lines describe the same configuration)."""
    K = len(SIGMA)
    surface = wl.get("surface", False)
    return {"workload": wl["desc"], "scene_tris": int(scene_tris), "points": wl["N"],
            "spp_diffuse": wl["spp_d"], "spp_specular": wl["spp_s"], "roughness_levels": K,
            "rays_per_step": wl["N"] * (wl["spp_d"] + K * wl["spp_s"]), "views": wl["views"],
            "resolution": [wl["W"], wl["H"]],
            "l2": "flushed between steps (512 MB write outside the timed events)",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "step": ("scene build + bake + render fwd/bwd + per-triangle error" if surface else
                     "scene build + first hits + compaction + bake + render fwd/bwd + "
                     "per-triangle error")}


def bake_roofline(prof, rays_per_step, n_rays_traced, alg_bytes, bake_s, sm_mhz, n_sm):
    """Ceilings of the bake kernel.  The one that binds is instruction
    issue: one warp instruction per scheduler per SM clock (4 schedulers
    per SM), so peak = SMs x 4 x the SM clock sampled during the timed
    region.  Issued warp instructions, DRAM bytes and active lanes per warp
    instruction come from the committed ncu capture of the same kernel
    source (per nominal ray, scaled to this launch).  Beside it: DRAM
    traffic against the measured HBM copy rate, and the algorithmic node /
    triangle bytes of the walk, which L1 and L2 serve (so that figure is a
    cache-served rate, not HBM traffic)."""
    hbm, hbm_kind = measured_peaks()
    cache = {"bound": "l1l2_algorithmic", "achieved": round(alg_bytes / bake_s / 1e9, 1),
             "peak": hbm, "unit": "GB/s", "frac": round(alg_bytes / bake_s / 1e9 / hbm, 4),
             "peak_kind": hbm_kind,
             "note": "algorithmic node + triangle + gather bytes per ray / bake time; served by L1/L2"}
    if prof is None or "warp_inst_per_ray" not in prof:
        out = dict(cache)
        out.update({"traffic": None, "kernel": "k_bake",
                    "note": cache["note"] + "; no ncu capture of the current kernel source"})
        return out
    traffic = float(prof["dram_bytes_per_ray"]) * rays_per_step
    inst = float(prof["warp_inst_per_ray"]) * rays_per_step
    peak_issue = n_sm * 4 * sm_mhz / 1e3                # G warp instructions / s
    ach_issue = inst / bake_s / 1e9
    lanes = float(prof["lanes_per_warp_inst"])
    return {"bound": "alu", "achieved": round(ach_issue, 1), "peak": round(peak_issue, 1),
            "unit": "Gwarp-inst/s", "frac": round(ach_issue / peak_issue, 4),
            "traffic": int(round(traffic)), "kernel": "k_bake",
            "peak_kind": "derived: %d SMs x 4 schedulers x %.0f MHz sampled SM clock" % (n_sm, sm_mhz),
            "what": "warp-instruction issue (the walk is bound by issue and divergence, not by HBM)",
            "warp_inst_per_ray": round(float(prof["warp_inst_per_ray"]), 2),
            "lanes_per_warp_inst": lanes,
            "lane_frac": round(ach_issue / peak_issue * lanes / 32.0, 4),
            "dram": {"achieved": round(traffic / bake_s / 1e9, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(traffic / bake_s / 1e9 / hbm, 4), "peak_kind": hbm_kind,
                     "bytes_per_ray": round(float(prof["dram_bytes_per_ray"]), 2)},
            "cache_served": cache,
            "ncu": {k: prof[k] for k in ("issue_active_pct", "l1_hit_pct", "l2_hit_pct", "capture")
                    if k in prof}}


def pinhole_views_for(mesh):
    from workloads import pinhole_views
    return pinhole_views(mesh, 24, seed=2)


# ---------------------------------------------------------------- GPU arm
def run_ours(args, wl, world, rank, local):
    import torch
    import paper_2304_05669_gb300 as F
    from paper_2304_05669_gb300._native import lib
    from paper_2304_05669_gb300.sharded import global_loss, global_tri_error

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mesh = make_scene(wl["scene"])
    from workloads import material_params, pinhole_views
    cams = pinhole_views(mesh, wl["views"], seed=2)
    N, W, H = wl["N"], wl["W"], wl["H"]
    spp_d, spp_s = wl["spp_d"], wl["spp_s"]
    K = len(SIGMA)
    rays_per_step = N * (spp_d + K * spp_s)

    host = {"V": mesh.V, "F": mesh.F, "Le": mesh.Le, "cache": mesh.cache, "cams": cams}
    surface = wl.get("surface", False)
    if surface:          # query records of points drawn uniformly on the surfaces
        from workloads import surface_queries
        sq = surface_queries(mesh, N, seed=0)
        rec = np.zeros((N, 10), np.float32)
        rec[:, 0:3], rec[:, 3:6], rec[:, 6:9] = sq["x"], sq["n"], sq["wo"]
        rec[:, 9] = sq["tri"].astype(np.int32).view(np.float32)
        host["q"] = rec
    mp = material_params(N, seed=3)
    gt = material_params(N, seed=4)
    host.update({"albedo": mp["albedo"], "rough": mp["rough"], "metal": mp["metal"]})
    pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in host.items()}
    dv = {k: v.to(dev) for k, v in pinned.items()}
    gt_d = {k: torch.from_numpy(v).to(dev) for k, v in gt.items()}
    stream = torch.cuda.current_stream()
    one = torch.ones(1, dtype=torch.float64, device=dev)     # d(step loss) / d(loss)
    ctx = F.context(local)
    request_id = rank

    def step(d, Lgt, ev=None):
        sc = F.Scene(d["V"], d["F"], d["Le"], d["cache"], ctx=ctx)
        if surface:
            q = d["q"]
        else:
            qa, valid = sc.camera_queries(d["cams"], W, H)
            q, _pix, _n = F.compact_queries(qa, valid, N)
        if ev is not None:
            ev[0].record(stream)
        Ld, Ls0, Ls1 = F.bake(sc, q, SIGMA, spp_d, spp_s, seed=0, request_id=request_id)
        if ev is not None:
            ev[1].record(stream)
        if Lgt is None:
            return sc, (Ld, Ls0, Ls1), q
        # render forward, loss and gradient in one pass, then the upstream gradient
        Lr, loss, grads = F.render_fwd_grad(Ld, Ls0, Ls1, SIGMA, d["albedo"], d["rough"], d["metal"], Lgt)
        F.render_grad_scale(grads, one)
        err, cnt = F.tri_error(q, Lr, Lgt, mesh.T)
        if world > 1:        # the two sums over all ranks' pixels (one all-reduce each)
            global_loss(loss)
            global_tri_error(err, cnt)
        return sc, (Ld, Ls0, Ls1), q, loss, grads, (err, cnt)

    # ground-truth images for the render loss: the same tables rendered with
    # a second set of material parameters (computed once, an input)
    sc0, tabs0, q0 = step(dv, None)
    Lgt = F.render_fwd(*tabs0, SIGMA, gt_d["albedo"], gt_d["rough"], gt_d["metal"])[0].clone()
    n_valid = N if surface else int(F.compact_queries(*sc0.camera_queries(dv["cams"], W, H), N)[2].item())
    ctx.sync_status()
    if n_valid < N:
        raise RuntimeError("workload has only %d hits < %d" % (n_valid, N))

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    for _ in range(args.warmup):
        flush.zero_()
        step(dv, Lgt)
    torch.cuda.synchronize()

    # -------------------------------------------------- timed: device-resident
    ev_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    ev_bake = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    launches0 = lib().fipt_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(uuid) as clk:
        for s in range(args.steps):
            flush.zero_()
            ev_step[s][0].record(stream)
            step(dv, Lgt, ev_bake[s])
            ev_step[s][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = lib().fipt_launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    bake_ms = [a.elapsed_time(b) for a, b in ev_bake]
    t_total = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    ctx.sync_status()

    # -------------------------------------------------- e2e: host in, host out
    e2e = None
    if not args.no_e2e:
        out_host = None
        in_keys = ["V", "F", "Le", "cache", "cams", "albedo", "rough", "metal"] + (["q"] if surface else [])
        Lgt_host = Lgt.cpu().pin_memory()
        h2d = sum(pinned[k].numel() * pinned[k].element_size() for k in in_keys) \
            + Lgt_host.numel() * 4
        d2h = 0
        # copies run on their own streams so they overlap the compute: a
        # step's inputs go up while the previous step computes, and its
        # results come back while the next one computes (double-buffered
        # pinned host outputs); the timed region ends when the last
        # step's results are on the host
        h2d_stream = torch.cuda.Stream(device=dev)
        d2h_stream = torch.cuda.Stream(device=dev)
        out_host = [None, None]
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_steps = min(args.steps, 5)
        e0.record(stream)
        h2d_stream.wait_event(e0)
        d2h_stream.wait_event(e0)
        for s in range(e2e_steps):
            with torch.cuda.stream(h2d_stream):
                d = {k: pinned[k].to(dev, non_blocking=True) for k in in_keys}
                Lg = Lgt_host.to(dev, non_blocking=True)
            stream.wait_stream(h2d_stream)
            for t in list(d.values()) + [Lg]:
                t.record_stream(stream)
            _sc, (Ld, Ls0, Ls1), _q, loss, grads, (err, cnt) = step(d, Lg)
            res = [Ld, Ls0, Ls1, loss, grads[0], grads[1], grads[2], err, cnt]
            if out_host[s % 2] is None:
                out_host[s % 2] = [torch.empty(r.shape, dtype=r.dtype, pin_memory=True) for r in res]
            d2h_stream.wait_stream(stream)
            with torch.cuda.stream(d2h_stream):
                for h, r in zip(out_host[s % 2], res):
                    h.copy_(r, non_blocking=True)
                    r.record_stream(d2h_stream)
            d2h = sum(r.numel() * r.element_size() for r in res)
        stream.wait_stream(d2h_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
        e2e = {"value": round(world * rays_per_step * e2e_steps / t_e2e / 1e6, 3),
               "unit": "Mrays/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(1e3 * t_e2e / e2e_steps, 3), "steps": e2e_steps,
               "copies": "pinned host buffers; inputs and results on two copy streams that overlap "
                         "the compute of the neighbouring steps"}

    # -------------------------------------------------- roofline of the bake
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    F.bake(sc0, q0, SIGMA, spp_d, spp_s, seed=0, request_id=request_id, stats=stats)
    ctx.sync_status()
    n_rays, n_nodes, n_tris, max_depth = [int(x) for x in stats.cpu().tolist()]
    bytes_per_ray = (64.0 * n_nodes + 48.0 * n_tris + 24.0 * n_rays) / max(n_rays, 1)
    alg_bytes = bytes_per_ray * n_rays + N * (40 + 4 * 3 * (1 + 2 * K))
    bake_s = float(np.mean(bake_ms)) / 1e3
    prof = recorded_profile(args.workload) if args.points is None and args.spp is None else None
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or measured_sm_max()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof = bake_roofline(prof, rays_per_step, n_rays, alg_bytes, bake_s, sm_mhz, n_sm)
    roof.update({"alg_bytes_per_ray": round(bytes_per_ray, 1),
                 "nodes_per_ray": round(n_nodes / max(n_rays, 1), 2),
                 "tris_per_ray": round(n_tris / max(n_rays, 1), 2), "max_stack": max_depth})

    # -------------------------------------------------- CPU baseline (rank 0, N=1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, dt, threads, n = oracle_sample(mesh, cams, W, H, min(args.cpu_points, N), spp_d, spp_s,
                                          surface=surface)
        cpu = {"value": round(r / dt / 1e6, 4), "unit": "Mrays/s", "cores": threads,
               "kind": "oracle",
               "sample": "%d oracle query points (%s), %d+6x%d spp, FP64, %.1f s" %
                         (n, "surface points" if surface else "first hits of view 0", spp_d, spp_s, dt)}

    refine = None
    if rank == 0 and world == 1 and args.refine_points > 0:
        refine = run_refine(args, F, dev, mesh, sc0, q0, not args.no_cpu_baseline)

    next_rows = None
    if rank == 0 and world == 1 and args.next_spp > 0:
        qa0, _v = sc0.camera_queries(dv["cams"], W, H)
        next_rows = run_next_rows(args, F, dev, mesh, sc0, q0, Lgt, qa0, not args.no_cpu_baseline,
                                  measured_peaks()[0])

    serving = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        serving = run_serving(args, F, dev)

    if rank != 0:
        return
    value = world * rays_per_step * args.steps / t_total / 1e6
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bake_config(wl, mesh.T, world),
        "points_per_s": round(world * N * args.steps / t_total, 1),
        "bake_ms": round(1e3 * bake_s, 3),
        "bake_mrays_per_s": round(rays_per_step / bake_s / 1e6, 3),
        # rays = N * S * (1 + K) samples; specular samples with n.wi <= 0 or
        # wo.h <= 0 contribute zero and trace nothing
        "traced_rays_per_step": int(n_rays),
        "bake_traced_mrays_per_s": round(n_rays / bake_s / 1e6, 3),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "refine": refine,
        "next_rows": next_rows,
        "serving": serving,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(out))


def main():
    args = parse()
    wl = dict(WORKLOADS[args.workload])
    if args.cpu_points is None:
        args.cpu_points = wl.get("cpu_points", 4096)
    if args.points:
        wl["N"] = args.points
        wl["desc"] += "; overridden to %d points" % args.points
    if args.spp:
        wl["spp_d"] = wl["spp_s"] = args.spp
        wl["desc"] += "; overridden to %d spp" % args.spp
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
    elif args.workload == "render":
        run_render(args, wl, world, rank, local)
    else:
        run_ours(args, wl, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
