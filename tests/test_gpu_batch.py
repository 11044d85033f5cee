"""The batched rebuild (rtsdf_batch_*) through the C-ABI.

Every scene of a batch must be bit-identical to its own single-scene build with
the same parameters (same Philox key and scene id): representative triangles,
flooded seeds, signed field everywhere; refine state (distance bits, front/back
votes) at masked voxels.  (The voxelizer's seeds are not compared directly: as
with rtsdf_jfa, the seed buffer is the first JFA ping-pong buffer and holds
flooding data after the rebuild; the flooded result pins them.)  The small batch is also checked against the
oracle scene by scene; every tuning (brick shape x warps per CTA, JFA graph on or
off) gives the same bits; the 48-scene workload of uneven sizes is compared with
48 single-scene builds.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import gpu_rebuild, require_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4), (8, 4, 2), (16, 2, 2)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _mask_from_nearest(g, nearest, mask_vox):
    """Integer ray mask from the flooded seeds (|v - s|^2 <= D^2, no seed: unmasked)."""
    k, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
    s = nearest.astype(np.int64)
    si, sj, sk = s & 1023, (s >> 10) & 1023, (s >> 20) & 1023
    d2 = (i - si) ** 2 + (j - sj) ** 2 + (k - sk) ** 2
    return (nearest != -1) & (d2.astype(np.float32) <= np.float32(mask_vox) ** 2)


def _batch_scene_arrays(B: rt.Batch, i: int) -> dict:
    out = {n: B.view(i, n).cpu().numpy().copy()
           for n in ("rep_tri", "nearest", "dist_bits", "front", "back", "sdf")}
    for n in ("dist_bits", "front", "back"):
        out[n] = out[n].view(np.uint32)
    return out


def _assert_same(a: dict, b: dict, mask: np.ndarray, what: str, sdf_tol: float = 0.0):
    for n in ("rep_tri", "nearest"):
        np.testing.assert_array_equal(a[n], b[n], err_msg=f"{what}: {n}")
    if sdf_tol == 0.0:
        np.testing.assert_array_equal(a["sdf"], b["sdf"], err_msg=f"{what}: sdf")
    else:
        assert np.abs(a["sdf"].astype(np.float64) - b["sdf"].astype(np.float64)).max() <= sdf_tol, what
    for n in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(a[n][mask], b[n][mask], err_msg=f"{what}: {n}")


def _plain(sc, frames=1):
    got, _ = gpu_rebuild(sc, frames=frames)
    return got


def test_small_batch_matches_oracle_and_single_scene_builds():
    scs = scenes.scene_batch_small()
    B = rt.Batch(scs)
    B.rebuild(0, False)
    torch.cuda.synchronize()
    masked_total = 0
    for i, sc in enumerate(scs):
        got = _batch_scene_arrays(B, i)
        ref = oracle.rebuild(sc)
        m = ref["mask"].astype(bool)
        _assert_same(got, ref, m, sc.name + " vs oracle", sdf_tol=1e-5)
        _assert_same(got, _plain(sc), m, sc.name + " vs single-scene")
        masked_total += int(m.sum())
    c = rt.counters_dict(B.counters)
    assert c["masked_voxels"] == masked_total
    assert c["rays_failed"] == 0 and c["stack_overflow"] == 0


def test_coarse_scene_in_a_batch_matches_oracle():
    """A coarse scene (the small room on 24x12x24: most of its 1,178 triangles lie within
    reach of every brick, so each brick's walk overflows the staging list and the
    batch's per-ray launch refines it) batched with a fine one: both against the
    oracle and against their single-scene builds (whose per-ray walk counts its work
    and so opens every box, where the batch skips boxes beyond the closest hit)."""
    coarse = dataclasses.replace(scenes.scene_small_room(n=24), frames=1)
    coarse = dataclasses.replace(coarse, refine=dataclasses.replace(coarse.refine, accumulate=False))
    scs = [coarse, scenes.scene_batch_small()[3]]
    B = rt.Batch(scs)
    B.rebuild(0, False)
    torch.cuda.synchronize()
    for i, sc in enumerate(scs):
        got = _batch_scene_arrays(B, i)
        ref = oracle.rebuild(sc)
        m = ref["mask"].astype(bool)
        _assert_same(got, ref, m, sc.name + " vs oracle", sdf_tol=1e-5)
        _assert_same(got, _plain(sc), m, sc.name + " vs single-scene")
    c = rt.counters_dict(B.counters)
    assert c["rays_failed"] == 0 and c["stack_overflow"] == 0


def test_every_tuning_gives_the_same_bits():
    scs = scenes.scene_batch_small()
    B = rt.Batch(scs)
    B.rebuild(0, False)
    torch.cuda.synchronize()
    base = [_batch_scene_arrays(B, i) for i in range(len(scs))]
    masks = [_mask_from_nearest(sc.grid, base[i]["nearest"], sc.refine.mask_vox) for i, sc in enumerate(scs)]
    for shape in SHAPES:
        for warps in (1, 2, 4):
            for graph in (True, False):
                B.set_tuning(shape, warps, graph)
                B.sdf.fill_(float("nan"))
                B.rebuild(0, False)
                torch.cuda.synchronize()
                for i in range(len(scs)):
                    _assert_same(_batch_scene_arrays(B, i), base[i], masks[i], f"{shape} x{warps} graph={graph}")
    ms = B.autotune(reps=2)
    assert ms > 0
    t = B.tuning
    assert (t["brick_x"], t["brick_y"], t["brick_z"]) in SHAPES and t["warps_per_cta"] in (1, 2, 4)


def test_48_scene_batch_matches_single_scene_builds():
    scs = scenes.scene_batch()
    B = rt.Batch(scs)
    B.autotune(reps=1)
    for f in range(2):  # two accumulated frames
        B.rebuild(f, f > 0)
    torch.cuda.synchronize()
    c = rt.counters_dict(B.counters)
    assert c["rays_failed"] == 0 and c["stack_overflow"] == 0 and c["skipped_triangles"] == 0
    for i, sc in enumerate(scs):
        sc2 = dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, accumulate=True))
        plain = _plain(sc2, frames=2)
        got = _batch_scene_arrays(B, i)
        m = _mask_from_nearest(sc.grid, plain["nearest"], sc.refine.mask_vox)
        assert m.sum() > 0
        _assert_same(got, plain, m, sc.name)
        torch.cuda.empty_cache()


def test_batch_at_capacity_matches_single_scene_builds():
    """RTSDF_BATCH_MAX_SCENES (64) small scenes of ragged sizes in one plan (full scene and
    JFA pass tables): every scene bit-identical to its own single-scene build."""
    scs = []
    seed = 100
    while len(scs) < 64:
        for sc in scenes.scene_batch_small(seed=seed):
            if len(scs) < 64:
                scs.append(dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, scene_id=len(scs))))
        seed += 1
    B = rt.Batch(scs)
    B.rebuild(0, False)
    torch.cuda.synchronize()
    c = rt.counters_dict(B.counters)
    assert c["rays_failed"] == 0 and c["stack_overflow"] == 0
    for i, sc in enumerate(scs):
        got = _batch_scene_arrays(B, i)
        plain = _plain(sc)
        m = _mask_from_nearest(sc.grid, plain["nearest"], sc.refine.mask_vox)
        _assert_same(got, plain, m, f"{sc.name} #{i}")


def test_batch_decay_matches_single_scene_builds():
    """accumulate = 2 (the Eq. (1) decay with each scene's alpha) in one batch: frame 0 fresh,
    frames 1 and 2 decayed; every scene bit-identical to its own single-scene sequence."""
    scs = [dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, accumulate=2, decay_alpha=0.9))
           for sc in scenes.scene_batch_small()]
    B = rt.Batch(scs)
    for f in range(3):
        B.rebuild(f, 2 if f > 0 else 0)
    torch.cuda.synchronize()
    for i, sc in enumerate(scs):
        plain = _plain(sc, frames=3)
        got = _batch_scene_arrays(B, i)
        m = _mask_from_nearest(sc.grid, plain["nearest"], sc.refine.mask_vox)
        _assert_same(got, plain, m, sc.name + " decay")
