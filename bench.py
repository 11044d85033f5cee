#!/usr/bin/env python
"""Benchmark of the RTSDF hot path on one GB300 (per rank).

A step is one frame of the whole path on the paper-shaped 400x200x400 room scene
(ground quad + 40 tessellated primitives, ~109k triangles): voxelize -> LBVH ->
10 jump-flooding passes (256..1 plus one extra 1) -> resolve + refine with 8 rays
per masked voxel (accumulated over frames) -> 1920x1080 soft-shadow raymarch.
Inputs are resident in HBM when the timed region starts; the per-frame working
set (~1.4 GB of grids) is far larger than L2, so no L2 flush is needed.

  python bench.py [--steps K] [--warmup W] [--workload room|tiny] [--impl reference]

Under torchrun every rank runs an independent replica (the path has no exchange
step); value = frames of all ranks / max-over-ranks time, expressed in ms/frame.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SDF rebuild ms/frame @400x200x400, GVoxel/s, %HBM roof; bwd+batch vs plain"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the ten flooding passes of one
# room frame, from one ncu capture, with the SHA-256 (first 16 hex digits) of the code of the
# flooding sources it was taken on (comments stripped); the bench reports it only while that
# code is unchanged
JFA_ROOM_TRAFFIC = {"bytes_per_frame": 2_211_134_720, "sources_sha256_16": "13f05a812ff87b66"}
JFA_SOURCES = ("paper_2210_06160_gb300/csrc/jfa_core.cuh", "paper_2210_06160_gb300/csrc/jfa.cu")
# algorithmic operations per unit of refinement work (counted by the kernel in rtsdf_counters):
# a ray is a Philox4x32-10 draw and Marsaglia's direction (about 20 FP32 and 40 integer
# operations); a BVH child-box test about 25; a (voxel, triangle) reach test 7 (a squared
# distance and a compare); a (pair, ray) plane/sphere filter test 10; a Moller-Trumbore test 35
REFINE_OPS_PER_UNIT = {"ray": 60, "node_test": 25, "reach_test": 7, "filter_ray_test": 10, "exact_test": 35}


def code_text(src: str) -> str:
    """C/CUDA source without its comments and with whitespace collapsed: what the
    compiler sees, so that edits to comments do not count as changes of the kernel."""
    import re
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def sources_hash(paths) -> str:
    """SHA-256 prefix of the code (comments stripped) of the given source files."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), encoding="utf-8") as f:
            h.update(code_text(f.read()).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="room", choices=["room", "tiny"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extensions", action="store_true", help="skip the backward and batched sections")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the benchmark: stage times over grid size x rays and mask distance x rays")
    return ap.parse_args()


def load_scene(workload: str):
    from paper_2210_06160_gb300 import scenes
    return scenes.scene_room() if workload == "room" else scenes.scene_tiny()


def workload_config(sc, workload: str) -> dict:
    g = sc.grid
    return {"workload": ("room scene 400x200x400 (ground quad + 40 primitives), 8 rays/voxel/frame "
                         "accumulated, 1920x1080 shadow, 96 steps" if workload == "room" else
                         "icosphere 64^3, 16 rays/voxel, 256x256 shadow, 64 steps"),
            "grid": [g.nx, g.ny, g.nz], "triangles": int(len(sc.tris)), "jfa_passes": len(sc.jfa_steps),
            "rays_per_voxel": sc.refine.rays_per_voxel, "receivers": int(len(sc.recv_pos)),
            "raymarch_steps": sc.shadow.steps,
            "l2": ("working set > L2 (grids of 128 MB each); no flush" if workload == "room" else
                   "working set < L2: a 256 MB buffer is written before each timed frame (outside its events); "
                   "ms/frame is the mean of the per-frame event spans")}


# ------------------------------------------------------------------ ranks

def rank_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (the slowest replica's time); no-op alone."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_ms_per_frame(t_max_ms: float, frames_per_rank: int, world: int) -> float:
    """Whole-job time per frame: every rank rebuilds its own replica (no exchange), so
    the job does frames_per_rank * world frames in the slowest rank's time."""
    return t_max_ms / (frames_per_rank * world)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle

def oracle_frame_sample(sc, threads: int | None = None, n_refine: int | None = None, full: bool = False) -> dict:
    """The oracle as it stands, timed stage by stage on `threads` host threads (all
    when None), on a bounded sample of one frame scaled to the whole frame: voxelize
    and resolve in full; the flooding passes in full (all threads) or the first and
    last pass scaled to all of them (one thread); ray sampling of `n_refine` masked
    voxels (brute force over every triangle per ray) scaled to all masked voxels; the
    shadow of a prefix of the receivers, scaled.  `full` runs everything in full (the
    small workloads)."""
    import numpy as np

    import oracle
    g, rp = sc.grid, sc.refine
    nproc = os.cpu_count() or 1
    oracle.set_num_threads(threads or nproc)
    used = oracle.num_threads()
    single = used == 1
    t, note = {}, []
    t0 = time.perf_counter()
    vv = oracle.to_voxel(sc.verts, g)
    seed, rep, _ = oracle.voxelize(vv, sc.tris, g)
    t["voxelize"] = time.perf_counter() - t0
    steps = list(sc.jfa_steps)
    if full or not single:
        t0 = time.perf_counter()
        near = oracle.jfa(g, seed, steps)
        t["jfa"] = time.perf_counter() - t0
    else:
        # one thread: time the first and the last pass (the cheapest and the dearest), scale
        near = seed
        t0 = time.perf_counter()
        first = oracle.jfa_pass(g, seed, steps[0])
        t_first = time.perf_counter() - t0
        oracle.set_num_threads(nproc)
        near = oracle.jfa(g, first, steps[1:])  # the field for resolve, not timed (all threads)
        oracle.set_num_threads(used)
        t0 = time.perf_counter()
        oracle.jfa_pass(g, near, steps[-1])
        t_last = time.perf_counter() - t0
        t["jfa"] = 0.5 * (t_first + t_last) * len(steps)
        note.append(f"JFA: passes {steps[0]} and {steps[-1]} timed, scaled to {len(steps)}")
    t0 = time.perf_counter()
    u_c, mask = oracle.resolve(g, vv, sc.tris, near, rep, rp.mask_vox)
    t["resolve"] = time.perf_counter() - t0
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    nsub = len(masked) if (full or n_refine is None or n_refine >= len(masked)) else max(1, n_refine)
    sub = masked[:: max(1, len(masked) // nsub)][:nsub]
    d, f, b = (x.ravel() for x in oracle.init_refine_state(u_c, mask)[:3])
    t0 = time.perf_counter()
    oracle.refine_voxels(g, vv, sc.tris, sub, rp, 0, d, f, b)
    t["refine"] = (time.perf_counter() - t0) * len(masked) / max(1, len(sub))
    sdf = (u_c - np.float32(rp.beta_vox)).astype(np.float32)
    npix = len(sc.recv_pos) if full else min(len(sc.recv_pos), 50_000 if not single else 10_000)
    t0 = time.perf_counter()
    oracle.shadow(g, sdf, sc.recv_pos[:npix], sc.recv_nrm[:npix], sc.shadow)
    t["shadow"] = (time.perf_counter() - t0) * len(sc.recv_pos) / max(1, npix)
    oracle.set_num_threads(nproc)
    total_ms = 1e3 * sum(t.values())
    sample = (f"voxelize + resolve in full; JFA ({len(steps)} passes) "
              + ("in full" if not note else "first and last pass scaled")
              + f"; ray sampling of {len(sub)} of {len(masked)} masked voxels (brute force over {len(sc.tris)} "
              f"triangles per ray){'' if len(sub) == len(masked) else ' scaled'}; shadow of {npix} of "
              f"{len(sc.recv_pos)} receivers{'' if npix == len(sc.recv_pos) else ' scaled'}")
    return {"value": total_ms, "unit": "ms/frame", "cores": used, "nproc": nproc, "kind": "oracle",
            "sample": sample, "refined_voxels": int(len(sub)), "stage_s": {k: round(v, 3) for k, v in t.items()}}


def cpu_baseline(sc, workload: str) -> dict:
    """The oracle on all host threads (ray sampling of at least 4,096 masked voxels) and
    on one thread (a smaller sample), both scaled to one frame."""
    full = workload != "room"
    allc = oracle_frame_sample(sc, None, n_refine=4096, full=full)
    one = oracle_frame_sample(sc, 1, n_refine=96, full=full)
    allc["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample", "stage_s")}
    return allc


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return
    sc = load_scene(args.workload)
    # each step a bounded sample of the frame (512 ray-sampled voxels on the room), all host threads
    n_ref = 512 if args.workload == "room" else None
    for _ in range(args.warmup):
        oracle_frame_sample(sc, None, n_refine=n_ref, full=args.workload != "room")
    vals, stage = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle_frame_sample(sc, None, n_refine=n_ref, full=args.workload != "room")
        vals.append(r["value"])
        stage = r
    wall = time.perf_counter() - t0
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/frame", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sc, args.workload),
            "cpu_baseline": {"value": v, "unit": "ms/frame", "cores": stage["cores"], "nproc": stage["nproc"],
                             "kind": "oracle", "sample": stage["sample"]},
            "e2e": {"value": v, "unit": "ms/frame", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 2)}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ghosting (Sec. 2.5.1)

def tri_dist64_pairs(P, A, B, C):
    """FP64 distance from point P[i] to triangle (A[i], B[i], C[i]), for every i: the
    plane foot when it lies inside the triangle, else the nearest of the three edges."""
    import numpy as np
    e1, e2, ap = B - A, C - A, P - A
    d00, d01, d11 = (e1 * e1).sum(1), (e1 * e2).sum(1), (e2 * e2).sum(1)
    d20, d21 = (ap * e1).sum(1), (ap * e2).sum(1)
    den = d00 * d11 - d01 * d01
    ok = den > 1e-300
    sden = np.where(ok, den, 1.0)
    u = (d11 * d20 - d01 * d21) / sden
    v = (d00 * d21 - d01 * d20) / sden
    inside = ok & (u >= 0) & (v >= 0) & (u + v <= 1)
    foot = A + u[:, None] * e1 + v[:, None] * e2
    best = np.where(inside, np.linalg.norm(P - foot, axis=1), np.inf)
    for a, b in ((A, B), (B, C), (C, A)):
        ab = b - a
        L = (ab * ab).sum(1)
        t = np.clip(((P - a) * ab).sum(1) / np.where(L > 0, L, 1.0), 0.0, 1.0)
        best = np.minimum(best, np.linalg.norm(P - (a + t[:, None] * ab), axis=1))
    return best


def true_distance_f64(vv, tris, pts, reach: float, small: float = 8.0):
    """FP64 unsigned distance (voxel units) from each point to the mesh with voxel-space
    vertices vv, for points known to lie within `reach` of some triangle.  Triangles
    of circumradius-about-centroid up to `small` are found through a k-d tree of their
    centroids; larger ones are tested against every point."""
    import numpy as np
    from scipy.spatial import cKDTree
    V = np.asarray(vv, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)
    T = T[(T >= 0).all(1) & (T < len(V)).all(1)]
    A, B, C = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    good = np.isfinite(A).all(1) & np.isfinite(B).all(1) & np.isfinite(C).all(1)
    A, B, C = A[good], B[good], C[good]
    P = np.asarray(pts, dtype=np.float64)
    cen = (A + B + C) / 3.0
    rad = np.sqrt(np.maximum(np.maximum(((A - cen) ** 2).sum(1), ((B - cen) ** 2).sum(1)), ((C - cen) ** 2).sum(1)))
    big = np.flatnonzero(rad > small)
    sm = np.flatnonzero(rad <= small)
    pp, tt = [], []
    if len(sm):
        lists = cKDTree(cen[sm]).query_ball_point(P, reach + float(rad[sm].max()))
        cnt = np.array([len(l) for l in lists])
        pp.append(np.repeat(np.arange(len(P)), cnt))
        tt.append(sm[np.concatenate([np.asarray(l, dtype=np.int64) for l in lists])] if cnt.sum() else
                  np.zeros(0, np.int64))
    if len(big):
        pp.append(np.repeat(np.arange(len(P)), len(big)))
        tt.append(np.tile(big, len(P)))
    out = np.full(len(P), np.inf)
    if pp:
        pi, ti = np.concatenate(pp), np.concatenate(tt)
        np.minimum.at(out, pi, tri_dist64_pairs(P[pi], A[ti], B[ti], C[ti]))
    return out


def ghost_stats(values, truth, tol: float = 1e-4) -> dict:
    """Ghosting of a field at sampled voxels: the fraction whose value lies below the
    current frame's true distance (by more than FP32 rounding, `tol` voxel), and the
    mean error value - truth (voxels)."""
    import numpy as np
    v = np.asarray(values, dtype=np.float64)
    t = np.asarray(truth, dtype=np.float64)
    return {"ghost_fraction": float(np.mean(v < t - tol)) if len(v) else 0.0,
            "mean_error_vox": float(np.mean(v - t)) if len(v) else 0.0, "samples": int(len(v))}


# ------------------------------------------------------------------ GPU path

def bench_dynamic(dev, frames: int = 120, warmup: int = 3, ghost_every: int = 4, ghost_samples: int = 16384) -> dict:
    """The room animated over `frames` frames (seeded linear and angular motion, 10
    deforming primitives): every frame re-voxelizes, rebuilds the BVH, floods and refines
    with 4 rays per voxel, then shades 1920x1080 receivers. Per-frame vertex arrays
    are uploaded before timing; each frame is timed with events. Run three ways: fresh
    per frame (no carry-over), with the Eq. (1) decay (alpha 0.95), and with the plain
    minimum over frames (the accumulation of the static scene).

    Ghosting (Sec. 2.5.1): on every `ghost_every`-th frame, seeded uniform voxels are read
    back after the frame (outside its timed span); at those inside the frame's ray mask
    the refined distance is compared with the FP64 distance to that frame's mesh.  The
    ghost fraction is the share below it (by more than FP32 rounding): distances left
    over from where a surface was.  Fresh frames cannot ghost (every value is a hit
    distance or a coarse distance on the current mesh); the decay fades old values."""
    import numpy as np
    import torch

    from paper_2210_06160_gb300 import rtsdf as rt
    from paper_2210_06160_gb300 import scenes

    anim = scenes.room_animation()
    sc = anim.scene
    g = sc.grid
    host_verts = [scenes.room_frame(anim, f) for f in range(frames)]
    verts = [torch.from_numpy(v).to(dev) for v in host_verts]
    tris = torch.from_numpy(sc.tris).to(dev)
    pos = torch.from_numpy(sc.recv_pos).to(dev)
    nrm = torch.from_numpy(sc.recv_nrm).to(dev)
    P = rt.Pipeline(g, len(sc.verts), len(sc.tris), device=dev)
    vis = torch.empty(len(sc.recv_pos), dtype=torch.float32, device=dev)
    sp = rt.make_shadow_params(sc.shadow)
    stream = torch.cuda.current_stream()
    ghost_frames = list(range(0, frames, ghost_every))
    rng = np.random.default_rng(2510)
    samples = {f: np.sort(rng.choice(g.nvox, ghost_samples, replace=False)) for f in ghost_frames}
    sample_dev = {f: torch.from_numpy(samples[f].astype(np.int64)).to(dev) for f in ghost_frames}
    out = {"workload": (f"room 400x200x400 animated, {frames} frames, {len(sc.tris)} triangles, "
                        f"{sc.refine.rays_per_voxel} rays/voxel, full rebuild + 1920x1080 shadow per frame")}
    reads = {}
    for label, mode in (("fresh", 0), ("decay", 2), ("minimum", 1)):
        def frame(f):
            rp = rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=f,
                                                           accumulate=mode if f > 0 else 0))
            P.rebuild(verts[f], tris, sc.jfa_steps, rp)
            P.shadow(pos, nrm, sp, vis)

        for f in range(warmup):
            frame(f)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
        got = {}
        for f in range(frames):
            evs[f][0].record(stream)
            frame(f)
            evs[f][1].record(stream)
            if f in sample_dev:
                got[f] = (P.dist_bits.view(-1).index_select(0, sample_dev[f]),
                          P.nearest.view(-1).index_select(0, sample_dev[f]))
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        out[label] = {"p50_ms": round(float(np.percentile(ms, 50)), 4), "p99_ms": round(float(np.percentile(ms, 99)), 4),
                      "mean_ms": round(float(ms.mean()), 4), "max_ms": round(float(ms.max()), 4)}
        reads[label] = {f: (d.cpu().numpy().view(np.uint32).view(np.float32), n.cpu().numpy()) for f, (d, n) in got.items()}
    del P, verts
    torch.cuda.empty_cache()
    # FP64 truth at the masked samples of each read frame (the same for every mode)
    D = float(sc.refine.mask_vox)
    per_frame = {label: [] for label in reads}
    errs = {label: [] for label in reads}
    n_masked = 0
    for f in ghost_frames:
        lin = samples[f]
        k, j, i = lin // (g.nx * g.ny), (lin // g.nx) % g.ny, lin % g.nx
        s = reads["fresh"][f][1].astype(np.int64)
        d2 = (i - (s & 1023)) ** 2 + (j - ((s >> 10) & 1023)) ** 2 + (k - (s >> 20)) ** 2
        m = (s >= 0) & (d2 <= D * D)  # the frame's ray mask (the same seeds in every mode)
        pts = np.stack([i[m], j[m], k[m]], 1) + 0.5
        vv = (host_verts[f].astype(np.float64) - np.array(g.origin)) / g.h
        truth = true_distance_f64(vv, sc.tris, pts, reach=D + 1.0)
        n_masked += int(m.sum())
        for label in reads:
            val = reads[label][f][0][m]
            st = ghost_stats(val, truth)
            per_frame[label].append(round(st["ghost_fraction"], 5))
            errs[label].append(st["mean_error_vox"])
    out["ghosting"] = {
        "frames_read": ghost_frames, "samples_per_frame": ghost_samples, "masked_samples": n_masked,
        "definition": ("share of sampled masked voxels whose refined distance is below the FP64 distance to the "
                       "current frame's mesh by more than 1e-4 voxel; mean error = refined - FP64 truth (voxels)"),
        **{f"ghosting_{label}": {"mean": round(float(np.mean(v)), 5), "max": round(float(np.max(v)), 5),
                                 "per_frame": v, "mean_error_vox": round(float(np.mean(errs[label])), 4)}
           for label, v in per_frame.items()}}
    return out


def bench_two_res(dev, steps: int = 10, warmup: int = 3) -> dict:
    """Sec. 2.5.1 two resolutions on the room: seeds and jump flooding on a 200x100x200
    coarse grid, coarse field, mask (2 coarse voxels = 4 fine) and refinement (8 rays,
    accumulated) on the 400x200x400 fine grid, then the 1920x1080 shadow."""
    import torch

    from paper_2210_06160_gb300 import rtsdf as rt
    from paper_2210_06160_gb300 import scenes

    sc = scenes.scene_room()
    gf = sc.grid
    gc = scenes.Grid(gf.nx // 2, gf.ny // 2, gf.nz // 2, gf.origin, gf.h * 2)
    steps_c = scenes.jfa_steps(gc, extra_one=True)
    verts = torch.from_numpy(sc.verts).to(dev)
    tris = torch.from_numpy(sc.tris).to(dev)
    pos = torch.from_numpy(sc.recv_pos).to(dev)
    nrm = torch.from_numpy(sc.recv_nrm).to(dev)
    P = rt.TwoResPipeline(gf, gc, len(sc.verts), len(sc.tris), device=dev)
    sp = rt.make_shadow_params(sc.shadow)
    vis = torch.empty(len(sc.recv_pos), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def frame(f, ev=None):
        rp = rt.make_refine_params(dataclasses.replace(sc.refine, mask_vox=2.0, frame_index=f, accumulate=f > 0))
        if ev:
            ev[0].record(stream)
        P.coarse.voxelize(verts, tris)
        P.fine.build_bvh(verts, tris)
        near = P.coarse.jfa(steps_c)
        if ev:
            ev[1].record(stream)
        f_ = P.fine
        rt.rtsdf_refine_2res(P.gf, P.gc, verts, tris, f_.bvh, near, P.coarse.rep_tri, rp, f_.dist_bits, f_.front,
                             f_.back, f_.sdf, f_.ws_refine, f_.counters)
        if ev:
            ev[2].record(stream)
        P.shadow(pos, nrm, sp, vis)
        if ev:
            ev[3].record(stream)

    for f in range(warmup):
        frame(f)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for i in range(steps):
        frame(warmup + i, evs[i])
    torch.cuda.synchronize()
    mean = lambda a, b: statistics.mean(e[a].elapsed_time(e[b]) for e in evs)
    out = {"workload": "room, coarse 200x100x200 (voxelize + JFA), fine 400x200x400 (BVH, resolve, refine 8 rays, "
                       "field), 1920x1080 shadow",
           "frame_ms": round(mean(0, 3), 4), "voxelize_bvh_jfa_ms": round(mean(0, 1), 4),
           "refine_ms": round(mean(1, 2), 4), "shadow_ms": round(mean(2, 3), 4), "steps": steps}
    del P
    torch.cuda.empty_cache()
    return out


def bench_batch(dev, steps: int = 5, warmup: int = 2) -> dict:
    """48 seeded scenes of uneven sizes (dims from 32^3 .. 256x128x256, 500-60k
    triangles, 8 rays/voxel): one batched rebuild (voxelize + BVH + JFA + refine,
    autotuned refine shape, JFA chain from a CUDA graph) against 48 sequential
    single-scene rebuilds on the same GPU."""
    import torch

    from paper_2210_06160_gb300 import rtsdf as rt
    from paper_2210_06160_gb300 import scenes

    scs = scenes.scene_batch()
    nvox = sum(sc.grid.nvox for sc in scs)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    # sequential single-scene builds
    pipes = []
    for sc in scs:
        v, t = torch.from_numpy(sc.verts).to(dev), torch.from_numpy(sc.tris).to(dev)
        pipes.append((rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris), device=dev), v, t, sc,
                      rt.make_refine_params(sc.refine)))

    def sequential():
        for P, v, t, sc, rp in pipes:
            P.rebuild(v, t, sc.jfa_steps, rp)

    for _ in range(warmup):
        sequential()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        sequential()
    ev[1].record(stream)
    torch.cuda.synchronize()
    seq_ms = ev[0].elapsed_time(ev[1]) / steps
    seq_launches0 = rt.rtsdf_kernel_launches()
    sequential()
    torch.cuda.synchronize()
    seq_launches = rt.rtsdf_kernel_launches() - seq_launches0
    del pipes
    torch.cuda.empty_cache()
    # batched
    B = rt.Batch(scs, device=dev)
    tune_ms = B.autotune(reps=2)
    for _ in range(warmup):
        B.rebuild(0, False)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        B.rebuild(0, False)
    ev[1].record(stream)
    torch.cuda.synchronize()
    batch_ms = ev[0].elapsed_time(ev[1]) / steps
    l0 = rt.rtsdf_kernel_launches()
    B.rebuild(0, False)
    torch.cuda.synchronize()
    batch_launches = rt.rtsdf_kernel_launches() - l0
    tri = sum(len(sc.tris) for sc in scs)
    out = {"workload": f"{len(scs)} scenes, dims from {sorted(set(scenes.BATCH_DIMS))}, {tri} triangles, "
                       f"{scs[0].refine.rays_per_voxel} rays/voxel, {nvox / 1e6:.1f} M voxels",
           "batched_ms": round(batch_ms, 4), "sequential_ms": round(seq_ms, 4),
           "batched_gvoxel_per_s": round(nvox / (batch_ms * 1e-3) / 1e9, 3),
           "sequential_gvoxel_per_s": round(nvox / (seq_ms * 1e-3) / 1e9, 3),
           "speedup": round(seq_ms / batch_ms, 3), "tuning": B.tuning, "autotune_refine_ms": round(tune_ms, 4),
           "launches_batched": int(batch_launches), "launches_sequential": int(seq_launches), "steps": steps}
    del B
    torch.cuda.empty_cache()
    return out


def bench_backward(dev, steps: int = 10, warmup: int = 3) -> dict:
    """Forward + adjoint on the 128^3 differentiation workload (8 icospheres s3 +
    2 boxes, 65,536 field samples, 512x512 shadow image, 1 frame of 8 rays), against
    the plain forward (untracked refine) of the same scene.  L = sum (s - s*)^2 +
    sum (v - v*)^2 with fixed targets (not timed)."""
    import torch

    from paper_2210_06160_gb300 import rtsdf as rt
    from paper_2210_06160_gb300 import scenes

    ds = scenes.scene_diff()
    sc = ds.scene
    g = sc.grid
    verts = torch.from_numpy(sc.verts).to(dev)
    tris = torch.from_numpy(sc.tris).to(dev)
    pts = torch.from_numpy(ds.pts).to(dev)
    pos = torch.from_numpy(sc.recv_pos).to(dev)
    nrm = torch.from_numpy(sc.recv_nrm).to(dev)
    rp = rt.make_refine_params(sc.refine)
    sp = rt.make_shadow_params(sc.shadow)
    frames = [sc.refine]
    plain = rt.Pipeline(g, len(sc.verts), len(sc.tris), device=dev)
    tracked = rt.Pipeline(g, len(sc.verts), len(sc.tris), device=dev, track=True)
    s_tgt = torch.zeros(len(ds.pts), dtype=torch.float32, device=dev)
    v_tgt = torch.full((len(sc.recv_pos),), 0.5, dtype=torch.float32, device=dev)
    # the light lives on the GPU, as a trained parameter would: the kernels read it there, so
    # the forward and backward enqueue without a host round trip
    light = torch.tensor(sc.shadow.light_dir, dtype=torch.float32, device=dev, requires_grad=True)
    stream = torch.cuda.current_stream()

    def plain_fwd():
        plain.rebuild(verts, tris, sc.jfa_steps, rp)
        plain.sample(pts)
        plain.shadow(pos, nrm, sp)

    def fwd_bwd(ev=None):
        v = verts.clone().requires_grad_(True)
        if ev:
            ev[0].record(stream)
        samples, vis = rt.sdf_shadow(v, light, tracked, tris, sc.jfa_steps, frames, pts, pos, nrm, sc.shadow)
        loss = ((samples - s_tgt) ** 2).sum() + ((vis - v_tgt) ** 2).sum()
        if ev:
            ev[1].record(stream)
        loss.backward()
        if ev:
            ev[2].record(stream)
        light.grad = None

    for _ in range(warmup):
        plain_fwd()
        fwd_bwd()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record(stream)
    for _ in range(steps):
        plain_fwd()
    e[1].record(stream)
    torch.cuda.synchronize()
    plain_ms = e[0].elapsed_time(e[1]) / steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(steps):
        fwd_bwd(evs[i])
    torch.cuda.synchronize()
    fwd_ms = statistics.mean(x[0].elapsed_time(x[1]) for x in evs)
    bwd_ms = statistics.mean(x[1].elapsed_time(x[2]) for x in evs)
    # the adjoint call alone (the state of the last forward is still in `tracked`)
    d_verts = torch.empty_like(verts)
    d_light = torch.empty(3, dtype=torch.float32, device=dev)
    ws = torch.empty(rt.rtsdf_backward_workspace(tracked.g), dtype=torch.uint8, device=dev)
    ds_ = torch.ones(len(ds.pts), dtype=torch.float32, device=dev)
    dv_ = torch.ones(len(sc.recv_pos), dtype=torch.float32, device=dev)
    sp_l = rt.make_shadow_params(sc.shadow)

    def adj():
        rt.rtsdf_backward(tracked.g, verts, tris, tracked.nearest, tracked.rep_tri, tracked.front, tracked.back,
                          tracked.win_ray, tracked.win_tri, rp, tracked.sdf, pts, ds_, pos, nrm, sp_l, dv_, d_verts,
                          d_light, ws)

    for _ in range(warmup):
        adj()
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(steps):
        adj()
    e[1].record(stream)
    torch.cuda.synchronize()
    adj_ms = e[0].elapsed_time(e[1]) / steps
    return {"workload": (f"differentiation {g.nx}^3, {len(sc.tris)} triangles (8 icospheres s3 + 2 boxes), "
                         f"{len(ds.pts)} samples, {int(len(sc.recv_pos) ** 0.5)}^2 shadow, "
                         f"{sc.refine.rays_per_voxel} rays/voxel"),
            "plain_forward_ms": round(plain_ms, 4), "tracked_forward_ms": round(fwd_ms, 4),
            "backward_ms": round(bwd_ms, 4), "rtsdf_backward_ms": round(adj_ms, 4),
            "fwd_bwd_gvoxel_per_s": round(g.nvox / ((fwd_ms + bwd_ms) * 1e-3) / 1e9, 3),
            "plain_gvoxel_per_s": round(g.nvox / (plain_ms * 1e-3) / 1e9, 3),
            "fwd_bwd_vs_plain": round((fwd_ms + bwd_ms) / plain_ms, 3), "steps": steps}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2210_06160_gb300 import build
    from paper_2210_06160_gb300 import rtsdf as rt

    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    rt.lib()

    sc = load_scene(args.workload)
    g = sc.grid
    dev = torch.device("cuda", local)
    verts = torch.from_numpy(sc.verts).to(dev)
    tris = torch.from_numpy(sc.tris).to(dev)
    pos = torch.from_numpy(sc.recv_pos).to(dev)
    nrm = torch.from_numpy(sc.recv_nrm).to(dev)
    P = rt.Pipeline(g, len(sc.verts), len(sc.tris), device=dev)
    vis = torch.empty(len(sc.recv_pos), dtype=torch.float32, device=dev)
    sp = rt.make_shadow_params(sc.shadow)
    stream = torch.cuda.current_stream()

    def params(f):
        return rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=f, accumulate=f > 0))

    side = P.side_stream()
    copy = torch.cuda.Stream(device=dev)
    pending = [None]  # a copy of the previous frame's field and visibility still in flight

    def frame(f, ev=None):
        # the BVH builds on a second stream while voxelize + JFA run (Pipeline.rebuild)
        ev0 = ev[0] if ev else torch.cuda.Event()
        ev0.record(stream)
        side.wait_event(ev0)
        if ev:
            ev[6].record(side)
        P.build_bvh(verts, tris, side)
        built = ev[7] if ev else torch.cuda.Event()
        built.record(side)
        P.voxelize(verts, tris, stream)
        if ev:
            ev[1].record(stream)
        P.jfa(sc.jfa_steps, stream)
        if ev:
            ev[2].record(stream)
        stream.wait_event(built)
        if pending[0] is not None:  # the refinement rewrites the field being copied out
            stream.wait_event(pending[0])
            pending[0] = None
        P.refine(verts, tris, params(f), stream)
        if ev:
            ev[3].record(stream)
        P.shadow(pos, nrm, sp, vis, stream)
        if ev:
            ev[4].record(stream)

    f = 0
    for _ in range(args.warmup):
        frame(f)
        f += 1
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    n_launch0 = rt.rtsdf_kernel_launches()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # a grid set that fits in L2 would stay cached between frames: flush it before each one
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if args.workload != "room" else None
    start.record(stream)
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xFF)
        frame(f, evs[i])
        f += 1
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = rt.rtsdf_kernel_launches() - n_launch0
    clk = clocks.stop()
    # one more frame, outside the timed region, with the refinement counting its work units
    work0 = rt.counters_dict(P.counters)
    P.refine(verts, tris, rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=f, accumulate=True),
                                                count_work=True), stream)
    torch.cuda.synchronize()
    f += 1
    work1 = rt.counters_dict(P.counters)
    t_ms = max_over_ranks(start.elapsed_time(end), world, dev)
    def span(a, b):
        return statistics.mean(evs[i][a].elapsed_time(evs[i][b]) for i in range(args.steps))

    # stage events on the frame's stream; the BVH's own span on the side stream, which overlaps
    # voxelize + JFA (rebuild_ms is the overlapped wall time of voxelize + BVH + JFA + refine)
    stage = {"voxelize": span(0, 1), "jfa": span(1, 2), "refine": span(2, 3), "shadow": span(3, 4),
             "bvh_side_stream": span(6, 7)}
    if flush is not None:  # the frames' own spans, without the flushes between them
        t_ms = max_over_ranks(sum(evs[i][0].elapsed_time(evs[i][4]) for i in range(args.steps)), world, dev)
        del flush
    ms_per_step = t_ms / args.steps
    value = replica_ms_per_frame(t_ms, args.steps, world)
    rebuild_ms = span(0, 3)
    nvox = g.nvox

    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak_src = "measured"
    try:
        hbm_peak = float(json.load(open(peaks_path))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm_peak, peak_src = 6800.0, "fallback"
    jfa_bytes = 8.0 * nvox * len(sc.jfa_steps)  # 4 B read + 4 B write per voxel per pass
    jfa_gbs = jfa_bytes / (stage["jfa"] * 1e-3) / 1e9
    # DRAM traffic of the passes from one ncu capture, while the flooding sources are the ones captured
    traffic = None
    if args.workload == "room" and JFA_ROOM_TRAFFIC["sources_sha256_16"] == sources_hash(JFA_SOURCES):
        traffic = JFA_ROOM_TRAFFIC["bytes_per_frame"]
    roofline = {"kernel": "k_jfa_pass + k_jfa_pass_grouped (all passes of a frame)", "bound": "hbm", "achieved": round(jfa_gbs, 1),
                "peak": hbm_peak, "unit": "GB/s", "frac": round(jfa_gbs / hbm_peak, 4), "traffic": traffic,
                "peak_source": peak_src, "algorithmic_bytes_per_frame": jfa_bytes,
                "per": f"frame: the {len(sc.jfa_steps)} flooding launches together (achieved = their bytes / "
                       f"their summed time, the launch-weighted mean rate; traffic likewise per frame)",
                "limit": "instruction issue (27 candidates per voxel, an exact (distance, seed) argmin each), not HBM"}

    # the dominant kernel by time, k_refine: the work it counts (rtsdf_counters, one counted frame)
    # per frame, as rates and as algorithmic operations per second against the FP32 lanes' rate at
    # the sampled SM clock; timed by the refine stage of the timed (uncounted) frames, which also
    # holds k_resolve and k_refine_report, so the rates are lower bounds on k_refine's own
    sm_mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    wide = ("node_tests", "reach_tests", "filter_pairs", "exact_tests")  # 64-bit counters; the others wrap at 2^32
    per_frame = {k: ((work1[k] - work0[k]) if k in wide else (work1[k] - work0[k]) & 0xFFFFFFFF)
                 for k in ("masked_voxels", "rays_hit", "near_edge_hits") + wide}
    units = {"ray": per_frame["masked_voxels"] * sc.refine.rays_per_voxel, "node_test": per_frame["node_tests"],
             "reach_test": per_frame["reach_tests"],
             "filter_ray_test": per_frame["filter_pairs"] * sc.refine.rays_per_voxel,
             "exact_test": per_frame["exact_tests"]}
    ops = sum(units[u] * REFINE_OPS_PER_UNIT[u] for u in units)
    t_ref = stage["refine"] * 1e-3
    lane_peak = 128.0 * nsm * sm_mhz * 1e6  # FP32 lanes per SM x SMs x clock: one operation each per cycle
    roofline_refine = {"kernel": "k_refine (timed with k_resolve in the refine stage)", "bound": "alu",
                       "achieved": round(ops / t_ref / 1e12, 3), "peak": round(lane_peak / 1e12, 3),
                       "unit": "T lane-operations/s", "frac": round(ops / t_ref / lane_peak, 4),
                       "peak_source": f"128 FP32 lanes x {nsm} SMs x median SM clock {sm_mhz:.0f} MHz",
                       "ops_per_unit": REFINE_OPS_PER_UNIT,
                       "units_per_frame": {k: int(v) for k, v in units.items()},
                       "rates_per_s": {f"{k}s": round(v / t_ref, 1) for k, v in units.items()},
                       "near_edge_hits_per_frame": per_frame["near_edge_hits"],
                       "rays_hit_per_frame": per_frame["rays_hit"]}

    counters = rt.counters_dict(P.counters)

    # the shadow through the texture path on the last frame's field (not part of the frame)
    tex = None
    if not args.no_extensions:
        T = rt.SdfTexture(g)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        for _ in range(3):
            T.upload(P.sdf)
            T.shadow(pos, nrm, sp, vis)
        torch.cuda.synchronize()
        reps = 10
        e[0].record(stream)
        for _ in range(reps):
            T.upload(P.sdf)
        e[1].record(stream)
        for _ in range(reps):
            T.shadow(pos, nrm, sp, vis)
        e[2].record(stream)
        torch.cuda.synchronize()
        tex = {"workload": "1920x1080 shadow, 96 steps, field as a 3D texture (hardware trilinear)",
               "shadow_ms": round(e[1].elapsed_time(e[2]) / reps, 4), "upload_ms": round(e[0].elapsed_time(e[1]) / reps, 4),
               "software_shadow_ms": round(stage["shadow"], 4)}
        del T

    # end to end through the C-ABI with host buffers: H2D of the mesh, D2H of sdf + visibility
    e2e = None
    if not args.no_e2e:
        h_verts = torch.from_numpy(sc.verts).pin_memory()
        h_tris = torch.from_numpy(sc.tris).pin_memory()
        h_sdf = torch.empty(P.sdf.shape, dtype=torch.float32).pin_memory()
        h_vis = torch.empty(vis.shape, dtype=torch.float32).pin_memory()
        ke = max(3, min(args.steps, 10))

        def e2e_frame(fi):
            verts.copy_(h_verts, non_blocking=True)
            tris.copy_(h_tris, non_blocking=True)
            frame(fi)
            # device -> host copies of the frame's results on a copy stream, overlapping the
            # next frame's voxelize + BVH + JFA; the next refinement waits for them
            done = torch.cuda.Event()
            done.record(stream)
            copy.wait_event(done)
            with torch.cuda.stream(copy):
                h_sdf.copy_(P.sdf, non_blocking=True)
                h_vis.copy_(vis, non_blocking=True)
                read = torch.cuda.Event()
                read.record(copy)
            pending[0] = read

        for _ in range(2):
            e2e_frame(f)
            f += 1
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            e2e_frame(f)
            f += 1
        stream.wait_event(pending[0])
        pending[0] = None
        e1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1), world, dev)
        e2e = {"value": replica_ms_per_frame(te, ke, world), "unit": "ms/frame",
               "h2d_bytes_per_step": int(h_verts.numel() * 4 + h_tris.numel() * 4),
               "d2h_bytes_per_step": int(h_sdf.numel() * 4 + h_vis.numel() * 4), "steps": ke}

    bwd = batch = dyn = two = None
    if args.workload == "room" and not args.no_extensions:
        bwd = bench_backward(dev)
        batch = bench_batch(dev)
        dyn = bench_dynamic(dev)
        two = bench_two_res(dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, args.workload)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "ms/frame", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": workload_config(sc, args.workload),
                "gvoxel_per_s": round(nvox / (rebuild_ms * 1e-3) / 1e9, 3),
                "rebuild_ms": round(rebuild_ms, 4),
                "stage_ms": {k: round(v, 4) for k, v in stage.items()},
                "roofline": roofline, "roofline_refine": roofline_refine, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "backward": bwd, "batch": batch, "dynamic": dyn, "two_resolution": two, "shadow_texture": tex,
                "clocks": clk, "counters": counters, "impl": "ours"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    del np


def run_sweep(args):
    """Stage times of the room scene (ms, CUDA events, mean of 5 frames after 2 warm-up
    frames, fresh refine state each frame) over (a) grid size x rays per voxel and (b)
    ray-mask distance x rays per voxel at 256x128x256: the axes of the paper's Table 3
    (size x rays) and Table 4 (mask distance d x rays), on one grid instead of the
    paper's coarse + fine pair.  Each point also reports the refinement's counted work per
    masked voxel (staged triangles reach-tested, pairs within reach) and exact tests per ray."""
    import torch

    from paper_2210_06160_gb300 import build
    from paper_2210_06160_gb300 import rtsdf as rt
    from paper_2210_06160_gb300 import scenes

    build.build()
    dev = torch.device("cuda", 0)

    def stages(sc, rays, mask_vox, frames=5, warmup=2):
        verts = torch.from_numpy(sc.verts).to(dev)
        tris = torch.from_numpy(sc.tris).to(dev)
        P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris), device=dev)
        rp = rt.make_refine_params(dataclasses.replace(sc.refine, rays_per_voxel=rays, mask_vox=mask_vox,
                                                       accumulate=0))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        acc = [0.0] * 4
        for i in range(warmup + frames):
            ev[0].record()
            P.voxelize(verts, tris)
            ev[1].record()
            P.build_bvh(verts, tris)
            ev[2].record()
            P.jfa(sc.jfa_steps)
            ev[3].record()
            P.refine(verts, tris, rp)
            ev[4].record()
            torch.cuda.synchronize()
            if i >= warmup:
                for j in range(4):
                    acc[j] += ev[j].elapsed_time(ev[j + 1]) / frames
        c = rt.counters_dict(P.counters)
        # one more refinement that counts its work units (not timed)
        P.refine(verts, tris, rt.make_refine_params(dataclasses.replace(sc.refine, rays_per_voxel=rays,
                                                                        mask_vox=mask_vox, accumulate=0),
                                                    count_work=True))
        torch.cuda.synchronize()
        w = rt.counters_dict(P.counters)
        nm = max(1, w["masked_voxels"] - c["masked_voxels"])
        work = {"staged_per_voxel": round((w["reach_tests"] - c["reach_tests"]) / nm, 1),
                "pairs_per_voxel": round((w["filter_pairs"] - c["filter_pairs"]) / nm, 1),
                "exact_per_ray": round((w["exact_tests"] - c["exact_tests"]) / (nm * rays), 2)}
        del P
        torch.cuda.empty_cache()
        return {"voxelize": round(acc[0], 3), "bvh": round(acc[1], 3), "jfa": round(acc[2], 3),
                "refine": round(acc[3], 3), "masked_voxels": c["masked_voxels"] // (warmup + frames), **work}

    size_rays = []
    for nx in (128, 256, 512):
        sc = scenes.scene_room(nx=nx, ny=nx // 2, nz=nx, shadow_w=64, shadow_h=36)
        for rays in (1, 5, 10):
            size_rays.append({"grid": [nx, nx // 2, nx], "rays": rays, **stages(sc, rays, 4.0)})
    sc = scenes.scene_room(nx=256, ny=128, nz=256, shadow_w=64, shadow_h=36)
    h = sc.grid.h
    mask_rays = []
    for d in (0.01, 0.05, 0.1, 0.5, None):
        mv = 1e6 if d is None else d / h
        for rays in (1, 5, 10, 15):
            mask_rays.append({"d_world": d, "mask_vox": round(mv, 3) if d is not None else "all", "rays": rays,
                              **stages(sc, rays, mv)})
    print(json.dumps({"sweep": "room scene", "size_x_rays": size_rays, "mask_x_rays_256x128x256": mask_rays}))


def main():
    args = parse()
    if args.sweep:
        run_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
