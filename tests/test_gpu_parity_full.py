"""Parity at the full 400x200x400 room workload, in the launch configuration the
benchmark times (the same Pipeline, the same per-frame parameters).

Whole-grid comparisons where the oracle finishes in seconds (seeds,
representative triangles, flooded seeds, the unmasked part of the field);
8,192 sampled masked voxels for ray sampling over two accumulated frames (the
oracle is brute force over all ~109k triangles per ray); sampled receivers for the
shadow, both sides marching the same field: the oracle-built coarse field, and the
field the GPU refined.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import gpu_shadow, require_gpu, to_dev

pytestmark = pytest.mark.gpu

FRAMES = 2
N_SAMPLE_VOXELS = 8192
N_SAMPLE_PIXELS = 20000


@pytest.fixture(scope="module")
def room():
    require_gpu()
    sc = scenes.scene_room()
    g, rp = sc.grid, sc.refine
    # GPU: exactly the benchmark's frame sequence (frame f accumulates for f > 0)
    verts, tris = to_dev(sc.verts), to_dev(sc.tris)
    P = rt.Pipeline(g, len(sc.verts), len(sc.tris))
    P.voxelize(verts, tris)
    seed = P.buf_a.cpu().numpy().copy()
    rep = P.rep_tri.cpu().numpy().copy()
    P.build_bvh(verts, tris)
    P.jfa(sc.jfa_steps)
    nearest = P.nearest.cpu().numpy().copy()
    for f in range(FRAMES):
        P.refine(verts, tris, rt.make_refine_params(dataclasses.replace(rp, frame_index=f, accumulate=f > 0)))
    torch.cuda.synchronize()
    got = dict(seed=seed, rep_tri=rep, nearest=nearest,
               dist_bits=P.dist_bits.cpu().numpy().view(np.uint32).ravel(),
               front=P.front.cpu().numpy().view(np.uint32).ravel(),
               back=P.back.cpu().numpy().view(np.uint32).ravel(),
               sdf=P.sdf.cpu().numpy(), counters=rt.counters_dict(P.counters))
    # oracle: full voxelize / flood / resolve, ray sampling on a seeded sample
    vv = oracle.to_voxel(sc.verts, g)
    o_seed, o_rep, _ = oracle.voxelize(vv, sc.tris, g)
    o_near = oracle.jfa(g, o_seed, sc.jfa_steps)
    u_c, mask = oracle.resolve(g, vv, sc.tris, o_near, o_rep, rp.mask_vox)
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    rng = np.random.default_rng(2210)
    sample = np.sort(rng.choice(masked, N_SAMPLE_VOXELS, replace=False)).astype(np.int32)
    state = None
    for f in range(FRAMES):
        state = oracle.init_refine_state(u_c, mask, state, accumulate=f > 0)
        d, fr, bk, wr, wt = (a.ravel() for a in state)
        oracle.refine_voxels(g, vv, sc.tris, sample, dataclasses.replace(rp, frame_index=f), f, d, fr, bk, wr, wt)
        state = tuple(a.reshape(g.shape_zyx) for a in (d, fr, bk, wr, wt))
    d, fr, bk = state[:3]
    sdf = oracle.finalize(g, vv, sc.tris, o_near, o_rep, mask, u_c, d, fr, bk, rp)
    ref = dict(seed=o_seed, rep_tri=o_rep, nearest=o_near, mask=mask, u_c=u_c, sample=sample,
               dist_bits=d.ravel(), front=fr.ravel(), back=bk.ravel(), sdf=sdf)
    return sc, got, ref


def test_room_seeds_and_flood_bit_exact(room):
    _, got, ref = room
    np.testing.assert_array_equal(got["seed"], ref["seed"])
    np.testing.assert_array_equal(got["rep_tri"], ref["rep_tri"])
    np.testing.assert_array_equal(got["nearest"], ref["nearest"])


def test_room_unmasked_field_and_mask(room):
    sc, got, ref = room
    m = ref["mask"].astype(bool)
    want = ref["u_c"][~m] - np.float32(sc.refine.beta_vox)
    assert np.abs(got["sdf"][~m].astype(np.float64) - want).max() <= 1e-5
    assert got["counters"]["masked_voxels"] == FRAMES * int(m.sum())
    assert got["counters"]["rays_failed"] == 0 and got["counters"]["stack_overflow"] == 0


@pytest.mark.slow
def test_room_sampled_refinement_bit_exact(room):
    _, got, ref = room
    s = ref["sample"]
    for k in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(got[k][s], ref[k][s], err_msg=k)
    assert np.abs(got["sdf"].ravel()[s].astype(np.float64) - ref["sdf"].ravel()[s]).max() <= 1e-5
    # the sample really exercised hits of both orientations
    assert ref["front"][s].sum() > 0 and ref["back"][s].sum() > 0


def test_room_shadow_sampled_pixels(room):
    sc, _, ref = room
    field = (ref["u_c"] - np.float32(sc.refine.beta_vox)).astype(np.float32)
    rng = np.random.default_rng(7)
    pick = rng.choice(len(sc.recv_pos), N_SAMPLE_PIXELS, replace=False)
    pos, nrm = sc.recv_pos[pick], sc.recv_nrm[pick]
    want = oracle.shadow(sc.grid, field, pos, nrm, sc.shadow)
    got = gpu_shadow(sc.grid, field, pos, nrm, sc.shadow)
    assert np.abs(got - want).max() <= 1e-4
    assert 0.0 < want.mean() < 1.0


def test_room_shadow_on_the_refined_field(room):
    """The 1920x1080 receivers' raymarch over the field the GPU refined (two frames of
    8 rays): both sides march that same field."""
    sc, got, _ = room
    field = got["sdf"].astype(np.float32)
    rng = np.random.default_rng(8)
    pick = rng.choice(len(sc.recv_pos), N_SAMPLE_PIXELS, replace=False)
    pos, nrm = sc.recv_pos[pick], sc.recv_nrm[pick]
    want = oracle.shadow(sc.grid, field, pos, nrm, sc.shadow)
    got_vis = gpu_shadow(sc.grid, field, pos, nrm, sc.shadow)
    assert np.abs(got_vis - want).max() <= 1e-4
    assert 0.0 < want.mean() < 1.0 and (want < 0.5).mean() > 0.01
