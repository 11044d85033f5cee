"""Python face of the CPU oracle (`rtsdf_oracle.c`).

TEST INFRASTRUCTURE ONLY: imported by `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py`, never by the library.  It compiles the plain C
oracle with gcc on first use and wraps each step with numpy arrays.  The step
functions follow the paper's order: voxelize (Sec. 2.2) -> jump flood (Sec. 2.2)
-> coarse distance and ray mask (Sec. 2.2-2.3) -> ray-sampled refinement
(Sec. 2.1) -> signed field -> soft-shadow raymarch (Sec. 2.4, 2.5.2-2.5.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_DIR, "rtsdf_oracle.c"), os.path.join(_DIR, "rtsdf_oracle_adjoint.c")]
_LIB = os.path.join(_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

EMPTY = -1


def build(force: bool = False) -> str:
    """Compile the oracle (FP32 without contraction, OpenMP over independent voxels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            [os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(os.path.join(_DIR, "rtsdf_oracle.h"))]):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-std=c11", "-shared", "-fPIC", "-o", tmp] + _SRCS + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("ox", C.c_float), ("oy", C.c_float), ("oz", C.c_float), ("h", C.c_float)]


def _g(grid) -> _Grid:
    return _Grid(grid.nx, grid.ny, grid.nz, *[float(v) for v in grid.origin], float(grid.h))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            f32, i32, i64, u32 = C.c_float, C.c_int32, C.c_int64, C.c_uint32
            G = C.POINTER(_Grid)
            sig = {
                "or_to_voxel": (None, [P, i32, G, P]),
                "or_tri_box_overlap": (C.c_int, [P, P, P, f32, f32, f32, f32]),
                "or_closest_d2": (f32, [P, P, P, P]),
                "or_voxelize": (i32, [P, i32, P, i32, G, P, P]),
                "or_jfa_pass": (None, [G, P, i32, P]),
                "or_resolve": (None, [G, P, P, P, P, f32, f32, P, P]),
                "or_philox4x32_10": (None, [P, P, P]),
                "or_sphere_dir": (C.c_int, [u32, u32, u32, P, P]),
                "or_ray_tri": (C.c_int, [P, P, P, P, P, f32, P, P, P]),
                "or_refine_voxels": (i64, [G, P, i32, P, i32, P, i64, i32, f32, P, u32, u32, P, P, P, P, P, P]),
                "or_vote_sign": (C.c_int, [u32, u32, P, P, P, P, C.c_int]),
                "or_finalize": (None, [G, P, P, P, P, P, P, P, P, P, f32, C.c_int, P]),
                "or_trilinear": (f32, [G, P, f32, f32, f32]),
                "or_resolve_2res": (None, [G, G, i32, P, P, P, P, f32, f32, P, P]),
                "or_fine_rep_2res": (None, [G, G, i32, P, P, P]),
                "or_sample": (None, [G, P, P, i32, P]),
                "or_shadow": (None, [G, P, P, P, i32, P, f32, i32, f32, f32, f32, f32, f32, P, P]),
                "or_jitter_starts": (None, [i32, f32, f32, u32, P]),
                "or_num_threads": (C.c_int, []),
                "or_set_num_threads": (None, [C.c_int]),
                "or_frozen_sources": (None, [G, P, P, P, P, P, P, P, P, P, P, u32, C.c_int, P]),
                "or_frozen_sdf_f64": (None, [G, P, P, P, C.c_double, P]),
                "or_frozen_sdf_backward_f64": (None, [G, P, P, P, C.c_double, P, P]),
                "or_sample_loss_f64": (C.c_double, [G, P, P, i32, P, P]),
                "or_shadow_loss_f64": (C.c_double, [G, P, P, P, P, i32, P, P, f32, i32, f32, f32, f32, f32, f32,
                                                    P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


def empty_dist(grid) -> float:
    """Coarse distance given to voxels that no seed reaches: nx + ny + nz voxels."""
    return float(grid.nx + grid.ny + grid.nz)


# ------------------------------------------------------------------ primitives

def to_voxel(verts, grid) -> np.ndarray:
    v = _f32(verts)
    out = np.empty_like(v)
    lib().or_to_voxel(_p(v), len(v), C.byref(_g(grid)), _p(out))
    return out


def tri_box_overlap(a, b, c, centre, hs: float) -> bool:
    a, b, c = _f32(a), _f32(b), _f32(c)
    return bool(lib().or_tri_box_overlap(_p(a), _p(b), _p(c), float(centre[0]), float(centre[1]),
                                         float(centre[2]), float(hs)))


def closest_d2(p, a, b, c) -> float:
    p, a, b, c = _f32(p), _f32(a), _f32(b), _f32(c)
    return float(lib().or_closest_d2(_p(p), _p(a), _p(b), _p(c)))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def sphere_dir(voxel: int, ray: int, scene: int, key) -> tuple[np.ndarray, int]:
    k = np.ascontiguousarray(key, dtype=np.uint32)
    d = np.zeros(3, dtype=np.float32)
    att = lib().or_sphere_dir(voxel & 0xFFFFFFFF, ray & 0xFFFFFFFF, scene & 0xFFFFFFFF, _p(k), _p(d))
    return d, att


def ray_tri(o, d, a, b, c, tmax: float, with_margin: bool = False):
    """(hit, t, front), plus the hit's smallest barycentric coordinate with_margin."""
    o, d, a, b, c = _f32(o), _f32(d), _f32(a), _f32(b), _f32(c)
    t = np.zeros(1, dtype=np.float32)
    f = np.zeros(1, dtype=np.int32)
    m = np.zeros(1, dtype=np.float32)
    hit = lib().or_ray_tri(_p(o), _p(d), _p(a), _p(b), _p(c), float(tmax), _p(t), _p(f), _p(m))
    out = (bool(hit), float(t[0]), bool(f[0])) if hit else (False, None, None)
    return out + ((float(m[0]) if hit else None),) if with_margin else out


def sample(grid, sdf, pts) -> np.ndarray:
    """The FP32 field at world points (trilinear, clamp to edge)."""
    s, pts = _f32(sdf), _f32(pts)
    out = np.empty(len(pts), dtype=np.float32)
    lib().or_sample(C.byref(_g(grid)), _p(s), _p(pts), len(pts), _p(out))
    return out


def trilinear(grid, sdf, q) -> float:
    s = _f32(sdf)
    return float(lib().or_trilinear(C.byref(_g(grid)), _p(s), float(q[0]), float(q[1]), float(q[2])))


# ------------------------------------------------------------------ the steps

def voxelize(vv, tris, grid):
    """Sec. 2.2 seeds from voxel-space vertices: (seed grid, rep-tri grid, skipped count)."""
    vv, t = _f32(vv), _i32(tris)
    seed = np.empty(grid.shape_zyx, dtype=np.int32)
    rep = np.empty(grid.shape_zyx, dtype=np.int32)
    sk = lib().or_voxelize(_p(vv), len(vv), _p(t), len(t), C.byref(_g(grid)), _p(seed), _p(rep))
    return seed, rep, int(sk)


def jfa_pass(grid, seeds, k: int) -> np.ndarray:
    a = _i32(seeds)
    out = np.empty_like(a)
    lib().or_jfa_pass(C.byref(_g(grid)), _p(a), int(k), _p(out))
    return out


def jfa(grid, seeds, steps) -> np.ndarray:
    a = _i32(seeds).copy()
    for k in steps:
        a = jfa_pass(grid, a, k)
    return a


def resolve(grid, vv, tris, nearest, rep_tri, mask_vox: float):
    vv, t, n, r = _f32(vv), _i32(tris), _i32(nearest), _i32(rep_tri)
    u_c = np.empty(grid.shape_zyx, dtype=np.float32)
    mask = np.empty(grid.shape_zyx, dtype=np.uint8)
    lib().or_resolve(C.byref(_g(grid)), _p(vv), _p(t), _p(n), _p(r), float(mask_vox),
                     empty_dist(grid), _p(u_c), _p(mask))
    return u_c, mask


def refine_voxels(grid, vv, tris, vox, rp, frame: int, dist_bits, front, back, win_ray=None, win_tri=None,
                  near_edge=None) -> int:
    """Sec. 2.1 on the listed voxels; dist_bits/front/back (and the winner record
    win_ray/win_tri when given) are updated in place.  near_edge (an int64 array of
    one element, optional) receives the number of ray/triangle hits within 1e-6
    (barycentric) of an edge.  Returns the rays whose direction could not be drawn."""
    vv, t, vox = _f32(vv), _i32(tris), _i32(vox)
    key = np.array(rp.key, dtype=np.uint32)
    for a in (dist_bits, front, back):
        assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    wr = None if win_ray is None else _p(win_ray)
    wt = None if win_tri is None else _p(win_tri)
    return int(lib().or_refine_voxels(C.byref(_g(grid)), _p(vv), len(vv), _p(t), len(t), _p(vox),
                                      len(vox), int(rp.rays_per_voxel), float(rp.max_ray_vox),
                                      _p(key), frame & 0xFFFFFFFF, rp.scene_id & 0xFFFFFFFF,
                                      _p(dist_bits), _p(front), _p(back), wr, wt,
                                      None if near_edge is None else _p(near_edge)))


def finalize(grid, vv, tris, nearest, rep_tri, mask, u_c, dist_bits, front, back, rp) -> np.ndarray:
    sdf = np.empty(grid.shape_zyx, dtype=np.float32)
    arrs = [_f32(vv), _i32(tris), _i32(nearest), _i32(rep_tri),
            np.ascontiguousarray(mask, dtype=np.uint8), _f32(u_c),
            np.ascontiguousarray(dist_bits, dtype=np.uint32),
            np.ascontiguousarray(front, dtype=np.uint32), np.ascontiguousarray(back, dtype=np.uint32)]
    lib().or_finalize(C.byref(_g(grid)), *[_p(a) for a in arrs], float(rp.beta_vox),
                      int(bool(rp.sign_fallback)), _p(sdf))
    return sdf


def resolve_2res(grid_f, grid_c, ratio, vv_f, tris, nearest_c, rep_c, mask_vox):
    """Sec. 2.5.1 two resolutions: (u_c, mask) on the fine grid from the coarse seeds."""
    u_c = np.empty(grid_f.shape_zyx, dtype=np.float32)
    mask = np.empty(grid_f.shape_zyx, dtype=np.uint8)
    lib().or_resolve_2res(C.byref(_g(grid_f)), C.byref(_g(grid_c)), int(ratio), _p(_f32(vv_f)), _p(_i32(tris)),
                          _p(_i32(nearest_c)), _p(_i32(rep_c)), float(mask_vox),
                          float(grid_f.nx + grid_f.ny + grid_f.nz), _p(u_c), _p(mask))
    return u_c, mask


def rebuild_2res(scene, grid_c, steps_c, frames: int = 1, frame0: int = 0, voxel_subset=None):
    """Two-resolution rebuild (Sec. 2.5.1): voxelize and flood on the coarse grid
    grid_c, resolve and refine on the scene's (fine) grid; scene.refine.mask_vox is in
    coarse voxels."""
    gf, rp = scene.grid, scene.refine
    ratio = int(round(grid_c.h / gf.h))
    vv_c = to_voxel(scene.verts, grid_c)
    seed_c, rep_c, _ = voxelize(vv_c, scene.tris, grid_c)
    near_c = jfa(grid_c, seed_c, steps_c)
    vv = to_voxel(scene.verts, gf)
    u_c, mask = resolve_2res(gf, grid_c, ratio, vv, scene.tris, near_c, rep_c, rp.mask_vox)
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    todo = masked if voxel_subset is None else np.intersect1d(masked, voxel_subset).astype(np.int32)
    state = None
    for f in range(frames):
        state = init_refine_state(u_c, mask, state, accumulate=rp.accumulate, alpha=rp.decay_alpha)
        d, fr, bk = (a.ravel().copy() for a in state[:3])
        refine_voxels(gf, vv, scene.tris, todo, rp, frame0 + f, d, fr, bk)
        state = (d.reshape(gf.shape_zyx), fr.reshape(gf.shape_zyx), bk.reshape(gf.shape_zyx)) + tuple(state[3:])
    rep_f = np.empty(gf.shape_zyx, dtype=np.int32)
    lib().or_fine_rep_2res(C.byref(_g(gf)), C.byref(_g(grid_c)), ratio, _p(_i32(near_c)), _p(_i32(rep_c)),
                           _p(rep_f))
    k, j, i = np.meshgrid(np.arange(gf.nz), np.arange(gf.ny), np.arange(gf.nx), indexing="ij")
    self_seed = ((k << 20) | (j << 10) | i).astype(np.int32)   # each voxel its own seed: rep_f per voxel
    sdf = finalize(gf, vv, scene.tris, self_seed, rep_f, mask, u_c, *state[:3], rp)
    return dict(seed_c=seed_c, rep_c=rep_c, nearest_c=near_c, u_c=u_c, mask=mask, masked=masked,
                dist_bits=state[0], front=state[1], back=state[2], sdf=sdf)


def jitter_starts(P: int, sp) -> np.ndarray:
    """First-sample distance of every receiver (Sec. 2.5.2 jitter; start_offset when 0)."""
    out = np.empty(max(P, 1), dtype=np.float32)
    lib().or_jitter_starts(int(P), float(sp.start_offset_vox), float(getattr(sp, "jitter_vox", 0.0)),
                           int(getattr(sp, "frame_index", 0)) & 0xFFFFFFFF, _p(out))
    return out


def shadow(grid, sdf, pos, nrm, sp) -> np.ndarray:
    s, pos, nrm = _f32(sdf), _f32(pos), _f32(nrm)
    L = np.array(sp.light_dir, dtype=np.float32)
    vis = np.empty(len(pos), dtype=np.float32)
    t0 = jitter_starts(len(pos), sp)
    lib().or_shadow(C.byref(_g(grid)), _p(s), _p(pos), _p(nrm), len(pos), _p(L), float(sp.k),
                    int(sp.steps), float(sp.max_step_vox), float(sp.start_offset_vox),
                    float(sp.normal_offset_vox), float(sp.hit_eps_vox), float(sp.bias_vox), _p(t0), _p(vis))
    return vis


def init_refine_state(u_c, mask, state=None, accumulate=0, alpha=0.95):
    """Refinement state before a frame's rays: masked voxels start from the coarse
    distance (or the smaller of it and the accumulated distance), counts from zero
    (or the accumulated counts); unmasked voxels hold the coarse distance, no votes.
    With a 5-tuple state (dist, front, back, win_ray, win_tri) the winner record
    follows: the coarse source wins when it sets the distance.

    accumulate = 2 is the decayed accumulation of Sec. 2.5.1, Eq. (1): masked voxels
    start from alpha * f_{t-1} + (1 - alpha) * c_t (FP32, products then sum; c_t the
    coarse distance), which this frame's hits then lower (the minimum with r_t);
    votes are this frame's only; unmasked voxels take c_t."""
    d0 = u_c.view(np.uint32).copy()
    none_ray = np.full_like(d0, 0xFFFFFFFF)
    none_tri = np.full(d0.shape, -1, dtype=np.int32)
    if state is None or not accumulate:
        return d0, np.zeros_like(d0), np.zeros_like(d0), none_ray, none_tri
    if int(accumulate) == 2:
        m = mask.astype(bool)
        a = np.float32(alpha)
        f_prev = np.ascontiguousarray(state[0], dtype=np.uint32).view(np.float32)
        blend = (a * f_prev + (np.float32(1.0) - a) * u_c.astype(np.float32)).astype(np.float32)
        dist = np.where(m, blend.view(np.uint32), d0).astype(np.uint32)
        zeros = np.zeros_like(d0)
        return np.ascontiguousarray(dist), zeros, zeros.copy(), none_ray, none_tri
    dist, fr, bk = state[:3]
    wr = state[3] if len(state) > 3 else none_ray
    wt = state[4] if len(state) > 4 else none_tri
    m = mask.astype(bool)
    coarse_wins = m & (d0 < dist)
    dist = np.where(m, np.minimum(dist, d0), d0)
    wr = np.where(coarse_wins | ~m, 0xFFFFFFFF, wr).astype(np.uint32)
    wt = np.where(coarse_wins | ~m, -1, wt).astype(np.int32)
    return (np.ascontiguousarray(dist, dtype=np.uint32), np.where(m, fr, 0).astype(np.uint32),
            np.where(m, bk, 0).astype(np.uint32), np.ascontiguousarray(wr), np.ascontiguousarray(wt))


def rebuild(scene, frames: int | None = None, frame0: int = 0, voxel_subset=None):
    """Full oracle rebuild of a scene: every intermediate of the hot path.

    `voxel_subset` (linear indices) restricts ray sampling to those masked voxels
    (for large grids); the returned refine arrays are then only meaningful there.
    """
    g, rp = scene.grid, scene.refine
    vv = to_voxel(scene.verts, g)
    seed, rep, skipped = voxelize(vv, scene.tris, g)
    nearest = jfa(g, seed, scene.jfa_steps)
    u_c, mask = resolve(g, vv, scene.tris, nearest, rep, rp.mask_vox)
    masked = np.flatnonzero(mask.ravel()).astype(np.int32)
    todo = masked if voxel_subset is None else np.intersect1d(masked, voxel_subset).astype(np.int32)
    state = None
    nf = scene.frames if frames is None else frames
    near = np.zeros(1, dtype=np.int64)
    near_total = 0
    for f in range(nf):
        state = init_refine_state(u_c, mask, state, accumulate=rp.accumulate, alpha=rp.decay_alpha)
        dist, fr, bk, wr, wt = (a.ravel() for a in state)
        refine_voxels(g, vv, scene.tris, todo, rp, frame0 + f, dist, fr, bk, wr, wt, near_edge=near)
        near_total += int(near[0])
        state = tuple(a.reshape(g.shape_zyx) for a in (dist, fr, bk, wr, wt))
    dist, fr, bk, wr, wt = state
    sdf = finalize(g, vv, scene.tris, nearest, rep, mask, u_c, dist, fr, bk, rp)
    return dict(vv=vv, seed=seed, rep_tri=rep, skipped=skipped, nearest=nearest, u_c=u_c,
                mask=mask, masked=masked, refined=todo, dist_bits=dist, front=fr, back=bk,
                win_ray=wr, win_tri=wt, sdf=sdf, near_edge=near_total)


# ------------------------------------------------------------------ adjoint (FP64)

SRC_DTYPE = np.dtype([("kind", np.int32), ("tri", np.int32), ("sign", np.float32), ("dir", np.float32, (3,))])


def frozen_sources(grid, vv, tris, nearest, rep_tri, mask, front, back, win_ray, win_tri, rp) -> np.ndarray:
    """Every discrete choice of the forward, per voxel (kind, triangle, sign, ray dir)."""
    out = np.zeros(grid.nvox, dtype=SRC_DTYPE)
    key = np.array(rp.key, dtype=np.uint32)
    arrs = [_f32(vv), _i32(tris), _i32(nearest), _i32(rep_tri), np.ascontiguousarray(mask, dtype=np.uint8),
            np.ascontiguousarray(front, dtype=np.uint32), np.ascontiguousarray(back, dtype=np.uint32),
            np.ascontiguousarray(win_ray, dtype=np.uint32), _i32(win_tri)]
    lib().or_frozen_sources(C.byref(_g(grid)), *[_p(a) for a in arrs], _p(key), rp.scene_id & 0xFFFFFFFF,
                            int(bool(rp.sign_fallback)), _p(out))
    return out


def frozen_sdf_f64(grid, verts64, tris, src, beta: float) -> np.ndarray:
    v = np.ascontiguousarray(verts64, dtype=np.float64)
    out = np.empty(grid.nvox, dtype=np.float64)
    lib().or_frozen_sdf_f64(C.byref(_g(grid)), _p(v), _p(_i32(tris)), _p(src), float(beta), _p(out))
    return out


def frozen_sdf_backward_f64(grid, verts64, tris, src, beta: float, gsdf) -> np.ndarray:
    v = np.ascontiguousarray(verts64, dtype=np.float64)
    g = np.ascontiguousarray(gsdf, dtype=np.float64).ravel()
    out = np.zeros_like(v)
    lib().or_frozen_sdf_backward_f64(C.byref(_g(grid)), _p(v), _p(_i32(tris)), _p(src), float(beta), _p(g),
                                     _p(out))
    return out


def sample_loss_f64(grid, sdf64, pts, target, gsdf=None) -> float:
    s = np.ascontiguousarray(sdf64, dtype=np.float64).ravel()
    pts, target = _f32(pts), _f32(target)
    return float(lib().or_sample_loss_f64(C.byref(_g(grid)), _p(s), _p(pts), len(pts), _p(target),
                                          None if gsdf is None else _p(gsdf)))


def shadow_loss_f64(grid, sdf32, sdf64, pos, nrm, light, sp, target, gsdf=None, gl=None,
                    light_decide=None) -> float:
    """The frozen-control shadow loss; the control flow is that of the FP32 march
    toward `light_decide` (default: `light` in FP32)."""
    s32 = _f32(sdf32).ravel()
    s64 = np.ascontiguousarray(sdf64, dtype=np.float64).ravel()
    pos, nrm, target = _f32(pos), _f32(nrm), _f32(target)
    l = np.ascontiguousarray(light, dtype=np.float64)
    ld = _f32(light if light_decide is None else light_decide)
    return float(lib().or_shadow_loss_f64(
        C.byref(_g(grid)), _p(s32), _p(s64), _p(pos), _p(nrm), len(pos), _p(ld), _p(l), float(sp.k), int(sp.steps),
        float(sp.max_step_vox), float(sp.start_offset_vox), float(sp.normal_offset_vox), float(sp.hit_eps_vox),
        float(sp.bias_vox), _p(jitter_starts(len(pos), sp)), _p(target), None if gsdf is None else _p(gsdf),
        None if gl is None else _p(gl)))
