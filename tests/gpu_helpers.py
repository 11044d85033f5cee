"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI and
the oracle on the same seeded inputs."""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2210_06160_gb300 import build
    build.build()
    rt.lib()


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_rebuild(sc: scenes.Scene, frames: int | None = None, frame0: int = 0, count_work: bool = True):
    """Voxelize, BVH, JFA and `frames` refine frames on the GPU; returns numpy copies.
    count_work=False runs the uncounted kernels (the ones the benchmark times)."""
    nf = sc.frames if frames is None else frames
    verts, tris = to_dev(sc.verts), to_dev(sc.tris)
    P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris))
    P.voxelize(verts, tris)
    seed = P.buf_a.cpu().numpy().copy()
    rep = P.rep_tri.cpu().numpy().copy()
    P.build_bvh(verts, tris)
    P.jfa(sc.jfa_steps)
    nearest = P.nearest.cpu().numpy().copy()
    for f in range(nf):
        rp = dataclasses.replace(sc.refine, frame_index=frame0 + f,
                                 accumulate=int(sc.refine.accumulate) if f > 0 else 0)
        P.refine(verts, tris, rt.make_refine_params(rp, count_work=count_work))
    torch.cuda.synchronize()
    out = dict(seed=seed, rep_tri=rep, nearest=nearest,
               dist_bits=P.dist_bits.cpu().numpy().view(np.uint32).copy(),
               front=P.front.cpu().numpy().view(np.uint32).copy(),
               back=P.back.cpu().numpy().view(np.uint32).copy(),
               sdf=P.sdf.cpu().numpy().copy(), counters=rt.counters_dict(P.counters))
    return out, P


def gpu_shadow(grid, sdf: np.ndarray, pos: np.ndarray, nrm: np.ndarray, sp) -> np.ndarray:
    g = rt.make_grid(grid)
    vis = torch.empty(len(pos), dtype=torch.float32, device="cuda")
    rt.rtsdf_shadow(g, to_dev(sdf.astype(np.float32)), to_dev(pos), to_dev(nrm), rt.make_shadow_params(sp), vis)
    return vis.cpu().numpy()


def compare_rebuild(ref: dict, got: dict, sdf_tol: float = 1e-5, voxels=None):
    """Bit-exact seeds, rep-tri, flooded seeds; bit-exact refine state and votes (every
    voxel, or the given sample of masked voxels); signed field within sdf_tol voxel."""
    np.testing.assert_array_equal(got["seed"], ref["seed"])
    np.testing.assert_array_equal(got["rep_tri"], ref["rep_tri"])
    np.testing.assert_array_equal(got["nearest"], ref["nearest"])
    sel = np.arange(ref["mask"].size) if voxels is None else np.asarray(voxels)
    for k in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(got[k].ravel()[sel], ref[k].ravel()[sel], err_msg=k)
    if voxels is None:
        d = np.abs(got["sdf"].astype(np.float64) - ref["sdf"].astype(np.float64))
        assert d.max() <= sdf_tol, (d.max(), np.unravel_index(d.argmax(), d.shape))
        # hits within 1e-6 of a triangle edge: the GPU tests only the triangles its filters
        # keep, the oracle every triangle, and the counts agree
        if "near_edge" in ref and "counters" in got:
            assert got["counters"]["near_edge_hits"] == ref["near_edge"], (got["counters"], ref["near_edge"])
    else:
        d = np.abs(got["sdf"].ravel()[sel].astype(np.float64) - ref["sdf"].ravel()[sel].astype(np.float64))
        assert d.max() <= sdf_tol
