"""Two resolutions (Sec. 2.5.1: coarse jump flooding, fine refinement) through
rtsdf_refine_2res against the oracle's two-grid rebuild: whole grids on a small
room (coarse 24x12x24, fine 48x24x48, two accumulated frames); one frame of the
room at coarse 200x100x200 / fine 400x200x400 on sampled voxels."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _coarse(g, r):
    return scenes.Grid((g.nx + r - 1) // r, (g.ny + r - 1) // r, (g.nz + r - 1) // r, g.origin, g.h * r)


def _gpu_2res(sc, gc, steps_c, frames, frame0=0):
    verts, tris = to_dev(sc.verts), to_dev(sc.tris)
    P = rt.TwoResPipeline(sc.grid, gc, len(sc.verts), len(sc.tris))
    for f in range(frames):
        rp = dataclasses.replace(sc.refine, frame_index=frame0 + f, accumulate=int(sc.refine.accumulate) if f else 0)
        P.rebuild(verts, tris, steps_c, rt.make_refine_params(rp))
    torch.cuda.synchronize()
    return dict(nearest_c=P.coarse.nearest.cpu().numpy(), rep_c=P.coarse.rep_tri.cpu().numpy(),
                dist_bits=P.fine.dist_bits.cpu().numpy().view(np.uint32),
                front=P.fine.front.cpu().numpy().view(np.uint32), back=P.fine.back.cpu().numpy().view(np.uint32),
                sdf=P.sdf.cpu().numpy(), counters=rt.counters_dict(P.fine.counters))


def test_two_res_small_room_whole_grids():
    sc = scenes.scene_small_room()
    sc = dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, mask_vox=2.0))
    gc = _coarse(sc.grid, 2)
    steps_c = scenes.jfa_steps(gc, extra_one=True)
    ref = oracle.rebuild_2res(sc, gc, steps_c, frames=2)
    got = _gpu_2res(sc, gc, steps_c, frames=2)
    np.testing.assert_array_equal(got["nearest_c"], ref["nearest_c"])
    np.testing.assert_array_equal(got["rep_c"], ref["rep_c"])
    for k in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert np.abs(got["sdf"].astype(np.float64) - ref["sdf"]).max() <= 1e-5
    assert got["counters"]["masked_voxels"] == 2 * int(ref["mask"].sum()) > 1000
    assert ref["back"].sum() > 0


def test_two_res_room_sampled():
    sc = scenes.scene_room(shadow_w=64, shadow_h=36)
    sc = dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, mask_vox=2.0))
    gc = _coarse(sc.grid, 2)
    steps_c = scenes.jfa_steps(gc, extra_one=True)
    got = _gpu_2res(sc, gc, steps_c, frames=1)
    # oracle: full coarse flood and fine resolve, ray sampling of 64 masked voxels
    vv_c = oracle.to_voxel(sc.verts, gc)
    seed_c, rep_c, _ = oracle.voxelize(vv_c, sc.tris, gc)
    near_c = oracle.jfa(gc, seed_c, steps_c)
    np.testing.assert_array_equal(got["nearest_c"], near_c)
    np.testing.assert_array_equal(got["rep_c"], rep_c)
    vv = oracle.to_voxel(sc.verts, sc.grid)
    u_c, mask = oracle.resolve_2res(sc.grid, gc, 2, vv, sc.tris, near_c, rep_c, sc.refine.mask_vox)
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    sample = np.sort(np.random.default_rng(5).choice(masked, 64, replace=False)).astype(np.int32)
    d, fr, bk = (a.ravel() for a in oracle.init_refine_state(u_c, mask)[:3])
    oracle.refine_voxels(sc.grid, vv, sc.tris, sample, sc.refine, 0, d, fr, bk)
    for k, want in (("dist_bits", d), ("front", fr), ("back", bk)):
        np.testing.assert_array_equal(got[k].ravel()[sample], want[sample], err_msg=k)
    um = ~mask.ravel()
    np.testing.assert_array_equal(got["dist_bits"].ravel()[um], d[um])
    np.testing.assert_allclose(got["sdf"].ravel()[um], (u_c.ravel()[um] - np.float32(1.0)), rtol=0, atol=1e-5)
