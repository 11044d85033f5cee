"""Small, fixed workloads for kernel profiling (ncu), sized so a full capture of one
launch ends quickly while the kernel sees the benchmark's voxel size and scene.

    python -m paper_2210_06160_gb300.profile_cases jfa
        voxelize the 400x200x400 room, then run its 10 flooding passes (only the
        two 128 MB flooding buffers stay resident)
    python -m paper_2210_06160_gb300.profile_cases refine-subbox [frames]
        the room's refinement on a 200^3 sub-box at the benchmark's voxel size
        (same triangles and brick statistics, ~8 M voxels); a last frame counts
        the refinement's work units
    python -m paper_2210_06160_gb300.profile_cases shadow
        the 1920x1080 shadow raymarch of the room on its rebuilt 400x200x400
        field (only the field and the receivers stay resident)
    python -m paper_2210_06160_gb300.profile_cases shadow-coherent
        the same with rtsdf_shadow_coherent: three calls, the second and third
        regrouped by the march lengths of the call before
    python -m paper_2210_06160_gb300.profile_cases adjoint
        the 128^3 differentiation workload: one tracked forward, then three
        rtsdf_backward calls (65,536 samples, 512x512 shadow image)
    python -m paper_2210_06160_gb300.profile_cases batch
        the 48-scene batch (118.8 M voxels): two batched rebuilds
    python -m paper_2210_06160_gb300.profile_cases refine-coarse
        the room on a 128x64x128 grid with 5 rays per voxel, three fresh frames:
        each refinement is two k_refine launches, the staged one (which leaves
        the bricks whose walk overflows to the next) and the per-ray walk
"""
from __future__ import annotations

import dataclasses
import sys

import torch

from paper_2210_06160_gb300 import build
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes


def case_jfa() -> None:
    sc = scenes.scene_room(shadow_w=64, shadow_h=36)
    g = rt.make_grid(sc.grid)
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda()
    seed = torch.empty(sc.grid.shape_zyx, dtype=torch.int32, device="cuda")
    rep = torch.empty_like(seed)
    ws = torch.empty(rt.rtsdf_voxelize_workspace(len(sc.tris), g), dtype=torch.uint8, device="cuda")
    rt.rtsdf_voxelize(v, t, g, seed, rep, ws)
    del ws, rep
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    out = rt.rtsdf_jfa(g, seed, torch.empty_like(seed), sc.jfa_steps)
    torch.cuda.synchronize()
    print("jfa ok", int((out >= 0).sum()))


def case_refine_subbox(frames: int = 3) -> None:
    sc = scenes.scene_room(shadow_w=64, shadow_h=36)
    g = scenes.Grid(200, 200, 200, (0.5, 0.0, 0.5), 0.005)
    steps = scenes.jfa_steps(g, extra_one=True)
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda()
    P = rt.Pipeline(g, len(sc.verts), len(sc.tris))
    for f in range(frames):
        P.rebuild(v, t, steps, rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=f, accumulate=f > 0)))
    torch.cuda.synchronize()
    # one more frame whose refinement counts its work units (the instantiation k_refine<0, 8, 1>)
    c0 = rt.counters_dict(P.counters)
    P.rebuild(v, t, steps, rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=frames, accumulate=True),
                                                 count_work=True))
    torch.cuda.synchronize()
    c1 = rt.counters_dict(P.counters)
    work = {k: c1[k] - c0[k] for k in ("masked_voxels", "node_tests", "reach_tests", "filter_pairs", "exact_tests")}
    print("refine-subbox ok", work)


def case_refine_coarse(frames: int = 3) -> None:
    sc = scenes.scene_room(nx=128, ny=64, nz=128, shadow_w=64, shadow_h=36)
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda()
    P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris))
    rp = dataclasses.replace(sc.refine, rays_per_voxel=5, accumulate=False)
    for f in range(frames):
        P.rebuild(v, t, sc.jfa_steps, rt.make_refine_params(dataclasses.replace(rp, frame_index=f)))
    torch.cuda.synchronize()
    print("refine-coarse ok", rt.counters_dict(P.counters))


def case_shadow(coherent: bool = False) -> None:
    sc = scenes.scene_room()
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda()
    P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris))
    for f in range(2):
        P.rebuild(v, t, sc.jfa_steps,
                  rt.make_refine_params(dataclasses.replace(sc.refine, frame_index=f, accumulate=f > 0)))
    sdf = P.sdf.clone()
    del P
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    pos, nrm = torch.from_numpy(sc.recv_pos).cuda(), torch.from_numpy(sc.recv_nrm).cuda()
    vis = torch.empty(len(sc.recv_pos), dtype=torch.float32, device="cuda")
    g, sp = rt.make_grid(sc.grid), rt.make_shadow_params(sc.shadow)
    if coherent:
        steps = torch.zeros(len(sc.recv_pos), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            rt.rtsdf_shadow_coherent(g, sdf, pos, nrm, sp, vis, steps)
    else:
        for _ in range(3):
            rt.rtsdf_shadow(g, sdf, pos, nrm, sp, vis)
    torch.cuda.synchronize()
    print("shadow ok", float(vis.mean()))


def case_adjoint() -> None:
    ds = scenes.scene_diff()
    sc = ds.scene
    v, t = torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda()
    pts = torch.from_numpy(ds.pts).cuda()
    pos, nrm = torch.from_numpy(sc.recv_pos).cuda(), torch.from_numpy(sc.recv_nrm).cuda()
    P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris), track=True)
    rp, sp = rt.make_refine_params(sc.refine), rt.make_shadow_params(sc.shadow)
    P.rebuild(v, t, sc.jfa_steps, rp)
    ones_s = torch.ones(len(ds.pts), dtype=torch.float32, device="cuda")
    ones_v = torch.ones(len(sc.recv_pos), dtype=torch.float32, device="cuda")
    dv = torch.empty_like(v)
    dl = torch.empty(3, dtype=torch.float32, device="cuda")
    ws = torch.empty(rt.rtsdf_backward_workspace(P.g), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        rt.rtsdf_backward(P.g, v, t, P.nearest, P.rep_tri, P.front, P.back, P.win_ray, P.win_tri, rp, P.sdf, pts,
                          ones_s, pos, nrm, sp, ones_v, dv, dl, ws)
    torch.cuda.synchronize()
    print("adjoint ok", float(dv.abs().sum()), dl.tolist())


def case_batch() -> None:
    B = rt.Batch(scenes.scene_batch())
    for _ in range(2):
        B.rebuild(0, False)
    torch.cuda.synchronize()
    print("batch ok", rt.counters_dict(B.counters))


if __name__ == "__main__":
    build.build()
    which = sys.argv[1] if len(sys.argv) > 1 else "jfa"
    if which == "jfa":
        case_jfa()
    elif which == "shadow":
        case_shadow()
    elif which == "shadow-coherent":
        case_shadow(coherent=True)
    elif which == "adjoint":
        case_adjoint()
    elif which == "batch":
        case_batch()
    elif which == "refine-coarse":
        case_refine_coarse()
    elif which == "refine-subbox":
        case_refine_subbox(int(sys.argv[2]) if len(sys.argv) > 2 else 3)
    else:
        raise SystemExit(f"unknown case {which}")
