"""The adjoint through the C-ABI against the FP64 oracle.

- rtsdf_refine_tracked: the winner record (ray id, triangle) bit-exact against the
  oracle's refinement, and the tracked call leaves dist/front/back/sdf as the
  untracked one does;
- rtsdf_sample: bit-exact trilinear samples;
- rtsdf_backward behind the autograd Function: dLoss/d(vertices) and
  dLoss/d(light direction) for L = sum (samples - s*)^2 + sum (vis - v*)^2 against
  the oracle's FP64 gradient of the same frozen function (its own forward on the
  same seeded scene; targets from the oracle's forward of the Gaussian-perturbed
  copy), on a miniature and on the 128^3 differentiation workload.

Tolerances: the GPU accumulates FP32 terms with atomics while the oracle sums in
FP64, so gradients agree to a relative 1e-3 of the largest entry (per entry) and
of the norm; the forward outputs keep the forward's bars (samples bit-exact,
visibility 1e-4).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes
from tests.gpu_helpers import require_gpu, to_dev

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _tracked_rebuild(sc, frames):
    verts, tris = to_dev(sc.verts), to_dev(sc.tris)
    out = {}
    for track in (False, True):
        P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris), track=track)
        P.voxelize(verts, tris)
        P.build_bvh(verts, tris)
        P.jfa(sc.jfa_steps)
        for f in range(frames):
            rp = dataclasses.replace(sc.refine, frame_index=f, accumulate=int(sc.refine.accumulate) if f > 0 else 0)
            P.refine(verts, tris, rt.make_refine_params(rp))
        torch.cuda.synchronize()
        out[track] = dict(dist_bits=P.dist_bits.cpu().numpy().view(np.uint32), front=P.front.cpu().numpy(),
                          back=P.back.cpu().numpy(), sdf=P.sdf.cpu().numpy())
        if track:
            out[track].update(win_ray=P.win_ray.cpu().numpy().view(np.uint32), win_tri=P.win_tri.cpu().numpy())
    return out


@pytest.mark.parametrize("which", ["tiny", "small_room"])
def test_winner_record_bit_exact(which):
    sc = scenes.scene_tiny(shadow_res=16) if which == "tiny" else scenes.scene_small_room()
    ref = oracle.rebuild(sc)
    got = _tracked_rebuild(sc, sc.frames)
    m = ref["mask"].astype(bool)
    for k in ("dist_bits", "front", "back"):
        np.testing.assert_array_equal(got[True][k][m], got[False][k][m], err_msg=k)
    np.testing.assert_array_equal(got[True]["sdf"], got[False]["sdf"])
    # everywhere: unmasked voxels hold the coarse record
    np.testing.assert_array_equal(got[True]["win_ray"], ref["win_ray"])
    np.testing.assert_array_equal(got[True]["win_tri"], ref["win_tri"])
    assert (ref["win_ray"][m] != 0xFFFFFFFF).sum() > 100 and (ref["win_ray"][m] == 0xFFFFFFFF).sum() > 0


def test_sample_bit_exact():
    sc = scenes.scene_small_room()
    ref = oracle.rebuild(sc, frames=1)
    rng = np.random.default_rng(4)
    lo = np.array(sc.grid.origin) - 0.1
    hi = np.array(sc.grid.origin) + np.array([sc.grid.nx, sc.grid.ny, sc.grid.nz]) * sc.grid.h + 0.1
    pts = rng.uniform(lo, hi, (5000, 3)).astype(np.float32)   # some outside: clamp to edge
    pts[:8] = [[0.0, 0.0, 0.0], [2.0, 1.0, 2.0], [1.0, 0.5, 1.0], [0.5 * sc.grid.h] * 3,
               [sc.grid.h, sc.grid.h, sc.grid.h], [1.5 * sc.grid.h] * 3, [-5.0, 0.3, 9.0], [1.0, 1.0, 1.0]]
    want = oracle.sample(sc.grid, ref["sdf"], pts)
    out = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    rt.rtsdf_sample(rt.make_grid(sc.grid), to_dev(ref["sdf"]), to_dev(pts), out)
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    empty = torch.empty(0, dtype=torch.float32, device="cuda")
    rt.rtsdf_sample(rt.make_grid(sc.grid), to_dev(ref["sdf"]), empty.view(0, 3), empty)


def _oracle_side(ds, light):
    """Oracle forward, targets from the perturbed copy, FP64 frozen gradient."""
    sc = ds.scene
    g, rp, sp = sc.grid, sc.refine, sc.shadow
    r = oracle.rebuild(sc)
    rt_ = oracle.rebuild(dataclasses.replace(sc, verts=ds.verts_target))
    s_tgt = oracle.sample(g, rt_["sdf"], ds.pts)
    v_tgt = oracle.shadow(g, rt_["sdf"], sc.recv_pos, sc.recv_nrm, dataclasses.replace(sp, light_dir=tuple(light)))
    src = oracle.frozen_sources(g, r["vv"], sc.tris, r["nearest"], r["rep_tri"], r["mask"], r["front"], r["back"],
                                r["win_ray"], r["win_tri"], rp)
    V64 = sc.verts.astype(np.float64)
    f64 = oracle.frozen_sdf_f64(g, V64, sc.tris, src, rp.beta_vox)
    gsdf = np.zeros(g.nvox)
    gl = np.zeros(3)
    sp_l = dataclasses.replace(sp, light_dir=tuple(light))
    loss = oracle.sample_loss_f64(g, f64, ds.pts, s_tgt, gsdf)
    loss += oracle.shadow_loss_f64(g, r["sdf"], f64, sc.recv_pos, sc.recv_nrm, np.array(light, np.float64), sp_l,
                                   v_tgt, gsdf, gl)
    gV = oracle.frozen_sdf_backward_f64(g, V64, sc.tris, src, rp.beta_vox, gsdf)
    samples = oracle.sample(g, r["sdf"], ds.pts)
    vis = oracle.shadow(g, r["sdf"], sc.recv_pos, sc.recv_nrm, sp_l)
    return dict(r=r, src=src, s_tgt=s_tgt, v_tgt=v_tgt, loss=loss, gV=gV, gl=gl, samples=samples, vis=vis)


def _gpu_side(ds, light, s_tgt, v_tgt, light_on_gpu=False):
    sc = ds.scene
    verts = to_dev(sc.verts).requires_grad_(True)
    L = torch.tensor(light, dtype=torch.float32, device="cuda" if light_on_gpu else "cpu", requires_grad=True)
    P = rt.Pipeline(sc.grid, len(sc.verts), len(sc.tris), track=True)
    frames = [dataclasses.replace(sc.refine, frame_index=f, accumulate=int(sc.refine.accumulate) if f > 0 else 0)
              for f in range(sc.frames)]
    samples, vis = rt.sdf_shadow(verts, L, P, to_dev(sc.tris), sc.jfa_steps, frames, to_dev(ds.pts),
                                 to_dev(sc.recv_pos), to_dev(sc.recv_nrm), sc.shadow)
    loss = ((samples - to_dev(s_tgt)) ** 2).sum() + ((vis - to_dev(v_tgt)) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return dict(samples=samples.detach().cpu().numpy(), vis=vis.detach().cpu().numpy(), loss=float(loss.detach()),
                gV=verts.grad.cpu().numpy().astype(np.float64), gl=L.grad.cpu().numpy().astype(np.float64),
                gl_device=L.grad.device.type)


def _compare(ds, light, light_on_gpu=False):
    o = _oracle_side(ds, light)
    g = _gpu_side(ds, light, o["s_tgt"], o["v_tgt"], light_on_gpu)
    np.testing.assert_array_equal(g["samples"], o["samples"])
    assert np.abs(g["vis"] - o["vis"]).max() <= 1e-4
    assert abs(g["loss"] - o["loss"]) <= 1e-4 * abs(o["loss"])
    gV, rV = g["gV"], o["gV"]
    scale = np.abs(rV).max()
    assert scale > 0
    err = np.abs(gV - rV)
    assert err.max() <= GRAD_RTOL * scale, (err.max(), scale, np.unravel_index(err.argmax(), err.shape))
    assert np.linalg.norm(gV - rV) <= GRAD_RTOL * np.linalg.norm(rV)
    assert np.abs(g["gl"] - o["gl"]).max() <= GRAD_RTOL * max(np.abs(o["gl"]).max(), 1e-6), (g["gl"], o["gl"])
    # the gradient reaches vertices of every object and the light
    assert (np.abs(rV).sum(1) > 0).mean() > 0.5 and np.abs(o["gl"]).max() > 0
    return o, g


@pytest.mark.parametrize("jitter", [0.0, 1.5])
def test_adjoint_matches_fp64_oracle_miniature(jitter):
    ds = scenes.scene_diff(48, 2, 4, 1, n_samples=4096, shadow_res=64)
    sc = dataclasses.replace(ds.scene, shadow=dataclasses.replace(ds.scene.shadow, jitter_vox=jitter, frame_index=3))
    _compare(dataclasses.replace(ds, scene=sc), (0.3, 1.0, 0.2))


def test_light_on_the_gpu_reads_the_same_direction():
    """A light tensor on the GPU is read by the kernels where it lives (the C-ABI's
    light_dir_device): the visibilities are bit-identical to those of the same light
    given by value, the gradient meets the same FP64 bars and stays on the GPU."""
    ds = scenes.scene_diff(48, 2, 4, 1, n_samples=4096, shadow_res=64)
    light = (0.3, 1.0, 0.2)
    o, g = _compare(ds, light, light_on_gpu=True)
    assert g["gl_device"] == "cuda"
    h = _gpu_side(ds, light, o["s_tgt"], o["v_tgt"], light_on_gpu=False)
    np.testing.assert_array_equal(g["vis"], h["vis"])
    np.testing.assert_array_equal(g["samples"], h["samples"])
    assert np.abs(g["gl"] - h["gl"]).max() <= 1e-5 * max(np.abs(h["gl"]).max(), 1e-6)


def test_adjoint_matches_fp64_oracle_128cube():
    """The 128^3 differentiation workload: 8 icospheres (subdiv 3) + 2 boxes,
    65,536 samples, 512^2 shadow; plus central differences of the oracle's frozen
    FP64 loss on random vertices against the GPU gradient (h = 1e-5 world: at
    1e-3, 0.13 voxel here, the quotient's own truncation error dominates near
    surfaces)."""
    ds = scenes.scene_diff()
    light = (0.3, 1.0, 0.2)
    o, g = _compare(ds, light)
    sc = ds.scene
    rng = np.random.default_rng(5)
    V64 = sc.verts.astype(np.float64)
    L64 = np.array(light, np.float64)

    def frozen_loss(V):
        f = oracle.frozen_sdf_f64(sc.grid, V, sc.tris, o["src"], sc.refine.beta_vox)
        return (oracle.sample_loss_f64(sc.grid, f, ds.pts, o["s_tgt"])
                + oracle.shadow_loss_f64(sc.grid, o["r"]["sdf"], f, sc.recv_pos, sc.recv_nrm, L64, sc.shadow,
                                         o["v_tgt"], light_decide=light))

    scale = np.abs(o["gV"]).max()
    cand = np.flatnonzero(np.abs(o["gV"]).sum(1) > 1e-3 * scale)
    h = 1e-5
    for v in rng.choice(cand, 16, replace=False):
        a = int(np.argmax(np.abs(o["gV"][v])))
        Vp, Vm = V64.copy(), V64.copy()
        Vp[v, a] += h
        Vm[v, a] -= h
        fd = (frozen_loss(Vp) - frozen_loss(Vm)) / (2 * h)
        assert abs(fd - g["gV"][v, a]) <= GRAD_RTOL * max(abs(fd), 1e-2 * scale), (v, a, fd, g["gV"][v, a])
