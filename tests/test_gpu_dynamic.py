"""The dynamic workload (the room animated frame by frame, every frame rebuilt from
scratch with 4 rays per voxel) and the decayed accumulation of Eq. (1) (Sec. 2.5.1),
against the oracle: whole grids on a small animated room, sampled voxels at
400x200x400."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import compare_rebuild, gpu_rebuild, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _small_anim():
    return scenes.room_animation(nx=48, ny=24, nz=48, n_prims=4, target_tris=None, shadow_w=32, shadow_h=18)


def _frame_scene(anim, f, **refine):
    return dataclasses.replace(anim.scene, verts=scenes.room_frame(anim, f),
                               refine=dataclasses.replace(anim.scene.refine, frame_index=f, **refine))


@pytest.mark.parametrize("f", [0, 23, 61])
def test_dynamic_small_room_frame(f):
    sc = _frame_scene(_small_anim(), f)
    ref = oracle.rebuild(sc, frames=1, frame0=f)
    got, _ = gpu_rebuild(sc, frames=1, frame0=f)
    compare_rebuild(ref, got)
    assert ref["mask"].sum() > 1000


def test_decay_sequence_small_room():
    """Frame 30 fresh, frames 31-33 with the Eq. (1) decay (alpha 0.95) while the scene
    moves: refine state bit-exact on the whole grid, field within 1e-5."""
    anim = _small_anim()
    g = anim.scene.grid
    P = rt.Pipeline(g, len(anim.scene.verts), len(anim.scene.tris))
    tris = to_dev(anim.scene.tris)
    state = None
    for f in range(30, 34):
        mode = 0 if f == 30 else 2
        sc = _frame_scene(anim, f, accumulate=mode)
        verts = to_dev(sc.verts)
        P.voxelize(verts, tris)
        P.build_bvh(verts, tris)
        P.jfa(sc.jfa_steps)
        P.refine(verts, tris, rt.make_refine_params(sc.refine))
        vv = oracle.to_voxel(sc.verts, g)
        seed, rep, _ = oracle.voxelize(vv, sc.tris, g)
        near = oracle.jfa(g, seed, sc.jfa_steps)
        u_c, mask = oracle.resolve(g, vv, sc.tris, near, rep, sc.refine.mask_vox)
        state = oracle.init_refine_state(u_c, mask, state, accumulate=mode, alpha=sc.refine.decay_alpha)
        d, fr, bk = (a.ravel().copy() for a in state[:3])
        oracle.refine_voxels(g, vv, sc.tris, np.flatnonzero(mask.ravel()).astype(np.int32), sc.refine, f, d, fr, bk)
        state = (d.reshape(g.shape_zyx), fr.reshape(g.shape_zyx), bk.reshape(g.shape_zyx)) + tuple(state[3:])
        sdf = oracle.finalize(g, vv, sc.tris, near, rep, mask, u_c, *state[:3], sc.refine)
        torch.cuda.synchronize()
        for name, want in (("dist_bits", d), ("front", fr), ("back", bk)):
            np.testing.assert_array_equal(getattr(P, name).cpu().numpy().view(np.uint32).ravel(), want,
                                          err_msg=f"frame {f} {name}")
        assert np.abs(P.sdf.cpu().numpy().astype(np.float64) - sdf).max() <= 1e-5
    # the decay really blended: some masked voxel holds neither its coarse distance nor a hit
    m = mask.astype(bool).ravel()
    assert np.any(d.view(np.float32)[m] < u_c.ravel()[m])


def test_dynamic_room_full_size_sampled():
    """Frame 77 of the 400x200x400 animated room, 4 rays: whole-grid seeds, representative
    triangles and flooded seeds; refine state at 64 sampled masked voxels."""
    anim = scenes.room_animation(shadow_w=64, shadow_h=36)
    f = 77
    sc = _frame_scene(anim, f)
    g, rp = sc.grid, sc.refine
    got, _ = gpu_rebuild(sc, frames=1, frame0=f)
    vv = oracle.to_voxel(sc.verts, g)
    seed, rep, _ = oracle.voxelize(vv, sc.tris, g)
    np.testing.assert_array_equal(got["seed"], seed)
    np.testing.assert_array_equal(got["rep_tri"], rep)
    near = oracle.jfa(g, seed, sc.jfa_steps)
    np.testing.assert_array_equal(got["nearest"], near)
    u_c, mask = oracle.resolve(g, vv, sc.tris, near, rep, rp.mask_vox)
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    sample = np.sort(np.random.default_rng(77).choice(masked, 64, replace=False)).astype(np.int32)
    d, fr, bk = (a.ravel() for a in oracle.init_refine_state(u_c, mask)[:3])
    oracle.refine_voxels(g, vv, sc.tris, sample, rp, f, d, fr, bk)
    for name, want in (("dist_bits", d), ("front", fr), ("back", bk)):
        np.testing.assert_array_equal(got[name].ravel()[sample], want[sample], err_msg=name)
    np.testing.assert_array_equal(got["dist_bits"].ravel()[~mask.ravel()], d[~mask.ravel()])


def test_ghosting_matches_the_oracle():
    """The Eq. (1) decay over the small animated room (5-frame stride): the GPU's
    refined distances at the sampled masked voxels equal the oracle's bit for bit, so
    the ghost fraction against the FP64 truth is the same on both sides."""
    import bench
    from tests import test_ghosting as tg
    anim = tg._anim()
    sc, g = anim.scene, anim.scene.grid
    vv0 = oracle.to_voxel(scenes.room_frame(anim, tg.FRAMES[0]), g)
    seed, rep, _ = oracle.voxelize(vv0, sc.tris, g)
    near = oracle.jfa(g, seed, sc.jfa_steps)
    _, mask = oracle.resolve(g, vv0, sc.tris, near, rep, sc.refine.mask_vox)
    voxels = np.sort(np.random.default_rng(5).choice(np.flatnonzero(mask.ravel()), 1000, replace=False))
    seq = tg._oracle_sequence(oracle, anim, 2, tg.FRAMES, voxels)
    want, _ = tg._fractions(g, sc.tris, seq, voxels, sc.refine.mask_vox + 1.0)
    P = rt.Pipeline(g, len(sc.verts), len(sc.tris))
    tris = to_dev(sc.tris)
    got_seq = []
    for n, f in enumerate(tg.FRAMES):
        verts = scenes.room_frame(anim, f)
        rp = dataclasses.replace(sc.refine, frame_index=f, accumulate=2 if n > 0 else 0, decay_alpha=0.95)
        P.rebuild(to_dev(verts), tris, sc.jfa_steps, rt.make_refine_params(rp))
        torch.cuda.synchronize()
        d = P.dist_bits.cpu().numpy().view(np.uint32).ravel().view(np.float32).copy()
        got_seq.append((verts, seq[n][1], d))
        sel = np.asarray([v for v in voxels if seq[n][1][v]])
        np.testing.assert_array_equal(d[sel].view(np.uint32), seq[n][2][sel].view(np.uint32), err_msg=f"frame {f}")
    got, _ = tg._fractions(g, sc.tris, got_seq, voxels, sc.refine.mask_vox + 1.0)
    assert got == want and max(got) > 0.0
