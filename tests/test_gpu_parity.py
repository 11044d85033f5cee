"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Bars: seeds, representative triangles, flooded seeds, hit counts and front/back
votes bit-exact; refined distances bit-exact (both sides take the same FP32
operations); signed field within 1e-5 voxel; shadow visibility within 1e-4.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import compare_rebuild, gpu_rebuild, gpu_shadow, require_gpu, to_dev

pytestmark = pytest.mark.gpu

SHADOW_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_tiny_icosphere_full_parity():
    sc = scenes.scene_tiny(shadow_res=128)
    ref = oracle.rebuild(sc)
    got, P = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    assert got["counters"]["masked_voxels"] == int(ref["mask"].sum())
    assert got["counters"]["rays_failed"] == 0 and got["counters"]["stack_overflow"] == 0
    vis_ref = oracle.shadow(sc.grid, ref["sdf"], sc.recv_pos, sc.recv_nrm, sc.shadow)
    vis = P.shadow(to_dev(sc.recv_pos), to_dev(sc.recv_nrm), rt.make_shadow_params(sc.shadow)).cpu().numpy()
    assert np.abs(vis - vis_ref).max() <= SHADOW_TOL


def test_small_room_accumulated_frames_parity():
    sc = scenes.scene_small_room()
    ref = oracle.rebuild(sc)
    got, P = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    vis_ref = oracle.shadow(sc.grid, ref["sdf"], sc.recv_pos, sc.recv_nrm, sc.shadow)
    vis = P.shadow(to_dev(sc.recv_pos), to_dev(sc.recv_nrm), rt.make_shadow_params(sc.shadow)).cpu().numpy()
    assert np.abs(vis - vis_ref).max() <= SHADOW_TOL


@pytest.mark.parametrize("count_work", [True, False])
def test_coarse_grid_parity(count_work):
    """The small room on a 24x12x24 grid: the 8-voxel rays span a third of the scene,
    so every brick has far more triangles within reach than its staging list holds
    and the refinement traces each ray through the BVH on its own (uncounted: boxes
    entered beyond the closest hit so far are skipped; counted: every box within the
    ray's length is opened); the field must still equal the oracle's, whole grid, two
    accumulated frames."""
    sc = scenes.scene_small_room(n=24)
    ref = oracle.rebuild(sc)
    got, _ = gpu_rebuild(sc, count_work=count_work)
    if count_work:
        # bricks whose walk overflowed (most of the 1,178 triangles within reach) stage
        # nothing; the others stage at most 256, so reach tests stay below 256 per voxel
        c = got["counters"]
        assert 0 < c["reach_tests"] <= 256 * c["masked_voxels"] or c["reach_tests"] == 0, c
        assert c["exact_tests"] > 0, c
    else:
        del got["counters"]  # the uncounted kernels count no near-edge hits
    compare_rebuild(ref, got)


def _random_scene(seed=0, dims=(37, 21, 29), n=60, R=5):
    rng = np.random.default_rng(seed)
    g = scenes.Grid(*dims, (-0.3, 0.1, -0.2), 0.05)
    ext = np.array(dims) * g.h
    c = np.array(g.origin) + rng.uniform(-0.1, 1.1, (n, 3)) * ext  # some outside the grid
    tri = c[:, None, :] + rng.normal(0, 0.15, (n, 3, 3)) * rng.choice([0.1, 1.0, 3.0], (n, 1, 1))
    V = tri.reshape(-1, 3).astype(np.float32)
    T = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    T[5] = [0, 0, 0]            # degenerate (a point)
    T[6] = [1, 2, 2]            # degenerate (a segment)
    T[7] = [0, 1, 10_000]       # invalid index: skipped
    V[3 * 9] = np.nan           # non-finite vertex: triangle 9 skipped
    rp = scenes.RefineParams(mask_vox=2.5, rays_per_voxel=R, max_ray_vox=6.0, beta_vox=0.5, key=(11, 22))
    return scenes.Scene("random", V, T, g, rp, scenes.ShadowParams(steps=40, max_step_vox=2.0),
                        scenes.jfa_steps(g), 1, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))


@pytest.mark.parametrize("R", [5, 16])
def test_random_triangles_ragged_grid_parity(R):
    """Ragged dims, triangles partly outside, degenerate and invalid triangles, and
    a ray count that does not divide the warp (atomic merge path)."""
    sc = _random_scene(R=R)
    ref = oracle.rebuild(sc)
    got, _ = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    assert got["counters"]["skipped_triangles"] == 2 * 2  # voxelize + BVH each count both


def test_sign_fallback_off_parity():
    """sign_fallback = 0: voxels whose front and back votes tie (including no hit) take +dist
    instead of the representative plane's side; whole grids against the oracle."""
    sc = scenes.scene_small_room(seed=9, n=30)
    sc = dataclasses.replace(sc, refine=dataclasses.replace(sc.refine, sign_fallback=False))
    ref = oracle.rebuild(sc)
    got, _ = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    m = ref["mask"].astype(bool)
    tie = m & (ref["front"] == ref["back"])
    assert tie.sum() > 0 and np.all(got["sdf"][tie] >= 0.0)


def _dense_cluster_scene(R: int, n: int = 3000):
    """n small triangles packed in a ball of radius 2.5 voxels: every brick near it
    reaches far more triangles than one staging round of the refine walk holds."""
    rng = np.random.default_rng(21)
    g = scenes.Grid(24, 24, 24, (0.0, 0.0, 0.0), 1.0 / 24)
    u = rng.normal(size=(n, 3))
    c = 12.0 + u / np.linalg.norm(u, axis=1, keepdims=True) * 2.5 * rng.uniform(0, 1, (n, 1)) ** (1 / 3)
    tri = (c[:, None, :] + rng.normal(0, 0.3, (n, 3, 3))) * g.h
    V = tri.reshape(-1, 3).astype(np.float32)
    T = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    rp = scenes.RefineParams(mask_vox=3.0, rays_per_voxel=R, max_ray_vox=6.0, beta_vox=1.0, key=(7, 9))
    return scenes.Scene("cluster", V, T, g, rp, scenes.ShadowParams(steps=30, max_step_vox=2.0),
                        scenes.jfa_steps(g), 1, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))


@pytest.mark.parametrize("R", [4, 16])
def test_dense_cluster_staging_rounds_parity(R):
    """Bricks whose candidate triangles overflow the staging list (the walk resumes
    in rounds, per pass and per ray group), bit-exact against the oracle's brute force."""
    sc = _dense_cluster_scene(R)
    vv = sc.verts.astype(np.float64).reshape(-1, 3, 3) / sc.grid.h
    lo, hi = vv.min(axis=1), vv.max(axis=1)
    qlo = np.array([8.5, 8.5, 8.5])  # the brick at (2, 2, 2): voxel centres 8.5 .. 11.5
    gap = np.maximum(np.maximum(lo - (qlo + 3.0), qlo - hi), 0.0)
    assert int(((gap ** 2).sum(1) <= 36.0).sum()) > 2 * 256  # several staging rounds for that brick
    ref = oracle.rebuild(sc)
    got, _ = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    assert got["counters"]["stack_overflow"] == 0 and got["counters"]["rays_hit"] > 0


def test_voxelize_big_and_sliver_triangles_bit_exact():
    """Long triangles at random orientations, from well shaped to slivers (sine of the
    angle between edges 0.5 down to 1e-5), spanning many bricks: seeds and representative
    triangles bit-exact against the oracle (the big-triangle plane filter must keep
    every voxel the separating-axis test accepts)."""
    rng = np.random.default_rng(31)
    g = scenes.Grid(64, 48, 40, (0.0, 0.0, 0.0), 0.05)
    dims = np.array([64, 48, 40], np.float64)
    tris = []
    for sin in (0.5, 1e-2, 1e-3, 2e-4, 5e-5, 1e-5):
        for _ in range(12):
            a = rng.uniform(0.1, 0.9, 3) * dims
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            q = rng.normal(size=3)
            q -= d * (q @ d)
            q /= np.linalg.norm(q)
            L = rng.uniform(20.0, 45.0)
            b = a + d * L
            c = a + d * L * rng.uniform(0.2, 0.8) + q * L * sin
            tris.append([a, b, c])
    V = (np.array(tris).reshape(-1, 3) * g.h).astype(np.float32)
    T = np.arange(len(V), dtype=np.int32).reshape(-1, 3)
    want_seed, want_rep, _ = oracle.voxelize(oracle.to_voxel(V, g), T, g)
    gg = rt.make_grid(g)
    seed = torch.empty(g.shape_zyx, dtype=torch.int32, device="cuda")
    rep = torch.empty_like(seed)
    ws = torch.empty(rt.rtsdf_voxelize_workspace(len(T), gg), dtype=torch.uint8, device="cuda")
    rt.rtsdf_voxelize(to_dev(V), to_dev(T), gg, seed, rep, ws)
    assert int((want_seed != -1).sum()) > 1000
    np.testing.assert_array_equal(seed.cpu().numpy(), want_seed)
    np.testing.assert_array_equal(rep.cpu().numpy(), want_rep)


def test_jfa_random_seeds_and_shapes_parity():
    rng = np.random.default_rng(1)
    for dims in [(1, 1, 1), (2, 3, 1), (33, 17, 65), (1023, 2, 3), (64, 64, 64)]:
        g = scenes.Grid(*dims, (0.0, 0.0, 0.0), 1.0)
        nvox = g.nvox
        seeds = np.full(g.shape_zyx, -1, np.int32)
        for frac in (0.0, 0.001, 0.05):
            cnt = int(nvox * frac)
            flat = rng.choice(nvox, cnt, replace=False) if cnt else np.zeros(0, int)
            k, j, i = np.unravel_index(flat, g.shape_zyx)
            s = seeds.copy()
            s[k, j, i] = (k << 20) | (j << 10) | i
            steps = scenes.jfa_steps(g, extra_one=True) + [3, 7]
            want = oracle.jfa(g, s, steps)
            a, b = to_dev(s), torch.empty_like(to_dev(s))
            out = rt.rtsdf_jfa(rt.make_grid(g), a, b, steps)
            np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_jfa_lattice_and_plane_seeds_with_ties_parity():
    """Seeds on a ground plane, a wall and a coarse lattice make many voxels
    equidistant from several seeds, so the lower-packed-seed rule decides often;
    widths that are not multiples of twice the offset leave ragged column pairs."""
    for dims in [(100, 50, 100), (37, 29, 41), (257, 9, 6)]:
        g = scenes.Grid(*dims, (0.0, 0.0, 0.0), 1.0)
        k, j, i = np.meshgrid(np.arange(g.nz), np.arange(g.ny), np.arange(g.nx), indexing="ij")
        on = (j == min(3, g.ny - 1)) | (i == g.nx // 3) | ((i % 7 == 0) & (j % 5 == 0) & (k % 9 == 0))
        s = np.where(on, (k << 20) | (j << 10) | i, -1).astype(np.int32)
        steps = scenes.jfa_steps(g, extra_one=True)
        want = oracle.jfa(g, s, steps)
        a, b = to_dev(s), torch.empty_like(to_dev(s))
        out = rt.rtsdf_jfa(rt.make_grid(g), a, b, steps)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        # one pass at a time as well, so a mistake in any single offset shows up
        cur = s
        for kk in steps:
            want1 = oracle.jfa_pass(g, cur, kk)
            a, b = to_dev(cur), torch.empty_like(to_dev(cur))
            got1 = rt.rtsdf_jfa(rt.make_grid(g), a, b, [kk]).cpu().numpy()
            np.testing.assert_array_equal(got1, want1, err_msg=f"dims {dims} offset {kk}")
            cur = want1


def test_empty_mesh_gives_empty_field_and_full_light():
    g = scenes.Grid(16, 12, 10, (0.0, 0.0, 0.0), 0.1)
    sc = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), g,
                      scenes.RefineParams(rays_per_voxel=4), scenes.ShadowParams(steps=20, max_step_vox=2.0),
                      scenes.jfa_steps(g), 1, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    ref = oracle.rebuild(sc)
    got, P = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    assert np.all(got["nearest"] == -1)
    assert np.all(got["sdf"] == np.float32(16 + 12 + 10) - np.float32(1.0))
    pos, nrm = scenes.receivers_plane(0.1, 0.0, 1.6, 0.0, 1.0, 8, 8)
    vis = P.shadow(to_dev(pos), to_dev(nrm), rt.make_shadow_params(sc.shadow)).cpu().numpy()
    assert np.all(vis == 1.0)


def test_single_triangle_and_bvh_of_one_leaf():
    g = scenes.Grid(20, 20, 20, (0.0, 0.0, 0.0), 0.05)
    V = np.array([[0.2, 0.5, 0.2], [0.8, 0.5, 0.3], [0.4, 0.5, 0.9]], np.float32)
    T = np.array([[0, 2, 1]], np.int32)
    sc = scenes.Scene("one", V, T, g, scenes.RefineParams(mask_vox=3.0, rays_per_voxel=8, key=(5, 6)),
                      scenes.ShadowParams(steps=30, max_step_vox=1.0), scenes.jfa_steps(g), 1,
                      np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    ref = oracle.rebuild(sc)
    got, _ = gpu_rebuild(sc)
    compare_rebuild(ref, got)
    assert got["counters"]["rays_hit"] > 0


def test_results_are_deterministic():
    sc = scenes.scene_small_room(seed=3, n=40)
    a, _ = gpu_rebuild(sc)
    for _ in range(2):
        b, _ = gpu_rebuild(sc)
        for k in ("seed", "rep_tri", "nearest", "dist_bits", "front", "back"):
            np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a["sdf"].view(np.uint32), b["sdf"].view(np.uint32))


def test_shadow_parity_on_analytic_field():
    """Shadow kernel alone on a seeded analytic field (sphere + floor), ragged grid,
    bias and hit epsilon set, receivers with tilted normals."""
    g = scenes.Grid(50, 40, 30, (0.0, 0.0, 0.0), 0.04)
    k, j, i = np.meshgrid(*(np.arange(n) + 0.5 for n in (30, 40, 50)), indexing="ij")
    f = np.minimum(np.sqrt((i - 25) ** 2 + (j - 25) ** 2 + (k - 15) ** 2) - 7.0, j - 3.0).astype(np.float32)
    rng = np.random.default_rng(4)
    pos = np.stack([rng.uniform(0, 2.0, 5000), np.full(5000, 0.13), rng.uniform(0, 1.2, 5000)], 1).astype(np.float32)
    nrm = rng.normal(0, 0.2, (5000, 3)) + [0, 1, 0]
    nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
    for sp in (scenes.ShadowParams(light_dir=(0.3, 1.0, 0.2), k=8.0, steps=96, max_step_vox=1.25),
               scenes.ShadowParams(light_dir=(-0.5, 0.7, 0.1), k=3.0, steps=64, max_step_vox=4.0,
                                   bias_vox=0.25, hit_eps_vox=0.05, start_offset_vox=0.5),
               scenes.ShadowParams(light_dir=(0.3, 1.0, 0.2), k=8.0, steps=96, max_step_vox=1.25, jitter_vox=1.25,
                                   frame_index=7)):
        want = oracle.shadow(g, f, pos, nrm, sp)
        got = gpu_shadow(g, f, pos, nrm, sp)
        assert np.abs(got - want).max() <= SHADOW_TOL


def test_coherent_shadow_equals_plain_shadow():
    """The regrouped raymarch gives the plain raymarch's visibilities bit for bit,
    whatever the march lengths it regroups by (zeroes, the previous call's, random
    bytes), on receiver counts below, at and above the 512-receiver block; and the
    lengths it writes are the plain march's stopping steps."""
    g = scenes.Grid(50, 40, 30, (0.0, 0.0, 0.0), 0.04)
    k, j, i = np.meshgrid(*(np.arange(n) + 0.5 for n in (30, 40, 50)), indexing="ij")
    f = np.minimum(np.sqrt((i - 25) ** 2 + (j - 25) ** 2 + (k - 15) ** 2) - 7.0, j - 3.0).astype(np.float32)
    rng = np.random.default_rng(9)
    sp = scenes.ShadowParams(light_dir=(0.3, 1.0, 0.2), k=8.0, steps=96, max_step_vox=1.25, jitter_vox=0.5,
                             frame_index=3)
    for P in (1, 300, 512, 5000, 12345):
        pos = np.stack([rng.uniform(0, 2.0, P), np.full(P, 0.13), rng.uniform(0, 1.2, P)], 1).astype(np.float32)
        nrm = np.tile(np.array([[0.0, 1.0, 0.0]], np.float32), (P, 1))
        want = oracle.shadow(g, f, pos, nrm, sp)
        plain = gpu_shadow(g, f, pos, nrm, sp)
        dpos, dnrm, dsdf = to_dev(pos), to_dev(nrm), to_dev(f)
        steps = torch.zeros(P, dtype=torch.uint8, device="cuda")
        vis = torch.empty(P, dtype=torch.float32, device="cuda")
        gg, spp = rt.make_grid(g), rt.make_shadow_params(sp)
        for init in ("zeros", "previous", "random"):
            if init == "random":
                steps.copy_(torch.from_numpy(rng.integers(0, 256, P).astype(np.uint8)))
            rt.rtsdf_shadow_coherent(gg, dsdf, dpos, dnrm, spp, vis, steps)
            np.testing.assert_array_equal(vis.cpu().numpy(), plain, err_msg=f"P={P} {init}")
        assert np.abs(plain - want).max() <= SHADOW_TOL
        st = steps.cpu().numpy().astype(int)
        assert st.max() <= sp.steps and st.max() > 0
        if P >= 5000:
            assert len(np.unique(st)) > 5  # marches of many lengths were regrouped


def test_accumulation_is_monotone_and_resumable():
    """Frames 0..3 in one run equal frames 0..1 then 2..3 resumed from the saved
    state (counter-based directions make the state a complete checkpoint)."""
    sc = scenes.scene_small_room(seed=5, n=40)
    full, P = gpu_rebuild(sc, frames=4)
    verts, tris = to_dev(sc.verts), to_dev(sc.tris)
    part, P2 = gpu_rebuild(sc, frames=2)
    for f in (2, 3):
        rp = dataclasses.replace(sc.refine, frame_index=f, accumulate=True)
        P2.refine(verts, tris, rt.make_refine_params(rp))
    for k in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(getattr(P2, k).cpu().numpy(), getattr(P, k).cpu().numpy())
    m = full["front"] + full["back"] >= part["front"] + part["back"]
    assert np.all(m)
