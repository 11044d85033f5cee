"""Seeded synthetic scenes, receiver buffers and workload descriptions.

This module only *generates inputs*: tessellated meshes, their seeded placement,
receiver points for the shadow pass and the parameter sets of the workloads.  It
holds none of the method's arithmetic (no voxelization, flooding, ray sampling
or raymarching), so both the CPU oracle and the CUDA path may consume it.

The paper evaluates on a living-room scene with dynamic objects (Sec. 3); that
scene is not available, so the workloads below stand in for it with seeded
scenes of the same kind: a ground quad plus tessellated spheres, boxes and tori
inside a room-sized box, at the 400x200x400 texture size the paper quotes for
its fine SDF (Sec. 2.1).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

# ----------------------------------------------------------------------------
# meshes (float64 geometry, int32 indices, counter-clockwise seen from outside)
# ----------------------------------------------------------------------------


def _orient_outward(verts: np.ndarray, tris: np.ndarray, inside_pts: np.ndarray) -> np.ndarray:
    """Flip every triangle whose geometric normal points toward its `inside_pts` row."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", n, cen - inside_pts) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def icosphere(subdiv: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere: 20 * 4**subdiv triangles, 10 * 4**subdiv + 2 vertices."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1, s2 in itertools.product((-1.0, 1.0), repeat=2):
        v += [(s1, s2 * g, 0.0), (0.0, s1, s2 * g), (s2 * g, 0.0, s1)]
    v = np.array(v)
    # faces = triples of mutually adjacent vertices (edge length 2)
    d = np.linalg.norm(v[:, None] - v[None], axis=-1)
    adj = np.abs(d - 2.0) < 1e-9
    faces = [(i, j, k) for i, j, k in itertools.combinations(range(12), 3)
             if adj[i, j] and adj[j, k] and adj[i, k]]
    assert len(faces) == 20
    verts = [tuple(p / np.linalg.norm(p)) for p in v]
    tris = faces
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in cache:
                p = (np.array(verts[i]) + np.array(verts[j])) * 0.5
                verts.append(tuple(p / np.linalg.norm(p)))
                cache[key] = len(verts) - 1
            return cache[key]

        nt = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nt += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = nt
    V = np.array(verts, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    T = _orient_outward(V, T, np.zeros((len(T), 3)))
    return V, T


def box_mesh() -> tuple[np.ndarray, np.ndarray]:
    """Axis-aligned cube with half-extent 1: 8 vertices, 12 triangles."""
    V = np.array(list(itertools.product((-1.0, 1.0), repeat=3)), dtype=np.float64)
    faces = []
    for axis in range(3):
        for side in (-1.0, 1.0):
            idx = [i for i in range(8) if V[i, axis] == side]
            # order the 4 face corners around the face
            o = [a for a in range(3) if a != axis]
            idx.sort(key=lambda i: math.atan2(V[i, o[1]], V[i, o[0]]))
            faces += [(idx[0], idx[1], idx[2]), (idx[0], idx[2], idx[3])]
    T = np.array(faces, dtype=np.int32)
    T = _orient_outward(V, T, np.zeros((len(T), 3)))
    return V, T


def torus_mesh(nu: int = 64, nv: int = 32, minor: float = 0.3) -> tuple[np.ndarray, np.ndarray]:
    """Torus of major radius 1 around the y axis: nu*nv vertices, 2*nu*nv triangles."""
    u = np.arange(nu) * (2 * math.pi / nu)
    w = np.arange(nv) * (2 * math.pi / nv)
    uu, ww = np.meshgrid(u, w, indexing="ij")
    r = 1.0 + minor * np.cos(ww)
    V = np.stack([r * np.cos(uu), minor * np.sin(ww), r * np.sin(uu)], -1).reshape(-1, 3)
    faces = []
    for i in range(nu):
        for j in range(nv):
            a = i * nv + j
            b = ((i + 1) % nu) * nv + j
            c = ((i + 1) % nu) * nv + (j + 1) % nv
            d = i * nv + (j + 1) % nv
            faces += [(a, b, c), (a, c, d)]
    T = np.array(faces, dtype=np.int32)
    # inside reference point of each face: the point of the tube's centre circle under it
    cen = V[T].mean(axis=1)
    ang = np.arctan2(cen[:, 2], cen[:, 0])
    inside = np.stack([np.cos(ang), np.zeros_like(ang), np.sin(ang)], -1)
    T = _orient_outward(V, T, inside)
    return V, T


def quad_mesh(y: float, x0: float, x1: float, z0: float, z1: float) -> tuple[np.ndarray, np.ndarray]:
    """Horizontal quad at height y facing +y: 4 vertices, 2 triangles."""
    V = np.array([[x0, y, z0], [x1, y, z0], [x1, y, z1], [x0, y, z1]], dtype=np.float64)
    T = np.array([[0, 2, 1], [0, 3, 2]], dtype=np.int32)
    T = _orient_outward(V, T, V[T].mean(axis=1) - np.array([0.0, 1.0, 0.0]))
    return V, T


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def merge(parts: list[tuple[np.ndarray, np.ndarray]]) -> tuple[np.ndarray, np.ndarray]:
    vs, ts, off = [], [], 0
    for V, T in parts:
        vs.append(V)
        ts.append(T + off)
        off += len(V)
    return np.concatenate(vs), np.concatenate(ts).astype(np.int32)


# ----------------------------------------------------------------------------
# grids, receivers, parameter sets
# ----------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Grid:
    """Uniform voxel grid: nx*ny*nz cells of edge h, min corner origin; x fastest."""
    nx: int
    ny: int
    nz: int
    origin: tuple[float, float, float]
    h: float

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape_zyx(self) -> tuple[int, int, int]:
        return (self.nz, self.ny, self.nx)


@dataclasses.dataclass(frozen=True)
class RefineParams:
    """Ray-sampling refinement settings (distances in voxel units)."""
    mask_vox: float = 3.0          # ray mask: refine where the flooded seed is within this distance
    rays_per_voxel: int = 16
    max_ray_vox: float = 8.0
    beta_vox: float = 1.0          # coarse SDF thickening subtracted outside the mask
    key: tuple[int, int] = (0, 0)  # counter-based generator key
    frame_index: int = 0
    scene_id: int = 0
    accumulate: int = 0            # 0 fresh, 1 min-accumulate (bool True), 2 decay of Eq. (1)
    sign_fallback: bool = True
    decay_alpha: float = 0.95      # Eq. (1) alpha (Sec. 2.5.1)


@dataclasses.dataclass(frozen=True)
class ShadowParams:
    """Soft-shadow raymarch settings (distances in voxel units)."""
    light_dir: tuple[float, float, float] = (0.3, 1.0, 0.2)
    k: float = 8.0
    steps: int = 64
    max_step_vox: float = 3.2
    start_offset_vox: float = 1.0
    normal_offset_vox: float = 1.0
    hit_eps_vox: float = 0.0
    bias_vox: float = 0.0
    jitter_vox: float = 0.0        # Sec. 2.5.2 jitter of the first sample along the light
    frame_index: int = 0


def jfa_steps(grid: Grid, extra_one: bool = False) -> list[int]:
    """Offsets n/2, n/4, ..., 1 with n the next power of two of the largest dimension."""
    n = max(grid.nx, grid.ny, grid.nz)
    top = 1
    while top * 2 < n:
        top *= 2
    steps = []
    k = top
    while k >= 1:
        steps.append(k)
        k //= 2
    if extra_one:
        steps.append(1)
    return steps


def receivers_plane(y: float, x0: float, x1: float, z0: float, z1: float,
                    w: int, hgt: int) -> tuple[np.ndarray, np.ndarray]:
    """Pixel-centre receiver points on a horizontal plane, normal +y (the headless G-buffer)."""
    xs = x0 + (np.arange(w) + 0.5) * ((x1 - x0) / w)
    zs = z0 + (np.arange(hgt) + 0.5) * ((z1 - z0) / hgt)
    zz, xx = np.meshgrid(zs, xs, indexing="ij")
    pos = np.stack([xx, np.full_like(xx, y), zz], -1).reshape(-1, 3).astype(np.float32)
    nrm = np.zeros_like(pos)
    nrm[:, 1] = 1.0
    return pos, nrm


@dataclasses.dataclass
class Scene:
    name: str
    verts: np.ndarray      # float32 [V,3] world
    tris: np.ndarray       # int32 [T,3]
    grid: Grid
    refine: RefineParams
    shadow: ShadowParams
    jfa_steps: list[int]
    frames: int            # frames of ray accumulation
    recv_pos: np.ndarray   # float32 [P,3]
    recv_nrm: np.ndarray   # float32 [P,3]


def scene_tiny(shadow_res: int = 256) -> Scene:
    """One icosphere (subdiv 3, 1280 triangles, centre 0.5, radius 0.3) in a 64^3 unit cube."""
    V, T = icosphere(3)
    V = V * 0.3 + 0.5
    g = Grid(64, 64, 64, (0.0, 0.0, 0.0), 1.0 / 64.0)
    pos, nrm = receivers_plane(0.1, 0.0, 1.0, 0.0, 1.0, shadow_res, shadow_res)
    return Scene("icosphere-64^3", V.astype(np.float32), T, g,
                 RefineParams(mask_vox=3.0, rays_per_voxel=16, max_ray_vox=8.0, beta_vox=1.0),
                 ShadowParams(steps=64, max_step_vox=0.05 / g.h),
                 jfa_steps(g), 1, pos, nrm)


_PRIMS: dict[str, tuple[np.ndarray, np.ndarray]] = {}


def _prim(kind: str) -> tuple[np.ndarray, np.ndarray]:
    if kind not in _PRIMS:
        _PRIMS[kind] = {"sphere": lambda: icosphere(4), "box": box_mesh,
                        "torus": lambda: torus_mesh(64, 32, 0.3)}[kind]()
    return _PRIMS[kind]


def room_primitives(rng: np.random.Generator, count: int, box: tuple[float, float, float],
                    target_tris: int | None, tol: float = 0.10,
                    scale=(0.05, 0.3), poses: list | None = None) -> list[tuple[np.ndarray, np.ndarray]]:
    """`count` seeded primitives (icosphere s4 / box / torus 64x32) with random pose and scale.

    When `target_tris` is given, primitive types are redrawn until the total is within `tol`.
    When `poses` is a list, (unit mesh V, T, centre, scale, rotation) of every primitive
    is appended to it.
    """
    kinds = ("sphere", "box", "torus")
    sizes = {k: len(_prim(k)[1]) for k in kinds}
    while True:
        types = rng.integers(0, 3, size=count)
        total = sum(sizes[kinds[t]] for t in types)
        if target_tris is None or abs(total - target_tris) <= tol * target_tris:
            break
    parts = []
    for t in types:
        V, T = _prim(kinds[t])
        c = np.array([rng.uniform(0.1, box[0] - 0.1), rng.uniform(0.1, box[1] - 0.1),
                      rng.uniform(0.1, box[2] - 0.1)])
        s = rng.uniform(*scale)
        R = random_rotation(rng)
        parts.append(((V * s) @ R.T + c, T))
        if poses is not None:
            poses.append((V, T, c, s, R))
    return parts


def scene_room(seed: int = 2210, nx: int = 400, ny: int = 200, nz: int = 400,
               n_prims: int = 40, target_tris: int = 100_000,
               shadow_w: int = 1920, shadow_h: int = 1080) -> Scene:
    """Paper-shaped static scene: ground quad + 40 primitives in a 2x1x2 box, ~100k triangles."""
    rng = np.random.default_rng(seed)
    box = (2.0, 1.0, 2.0)
    h = box[0] / nx
    parts = [quad_mesh(0.05, 0.0, 2.0, 0.0, 2.0)]
    parts += room_primitives(rng, n_prims, box, target_tris)
    V, T = merge(parts)
    g = Grid(nx, ny, nz, (0.0, 0.0, 0.0), h)
    pos, nrm = receivers_plane(0.05, 0.0, 2.0, 0.0, 2.0, shadow_w, shadow_h)
    return Scene(f"room-{nx}x{ny}x{nz}", V.astype(np.float32), T, g,
                 RefineParams(mask_vox=4.0, rays_per_voxel=8, max_ray_vox=8.0, beta_vox=1.0,
                              accumulate=True),
                 ShadowParams(steps=96, max_step_vox=0.05 / h),
                 jfa_steps(g, extra_one=True), 16, pos, nrm)


def scene_small_room(seed: int = 7, n: int = 48, n_prims: int = 6) -> Scene:
    """A scaled-down room (ground + a few primitives) whose oracle finishes quickly."""
    rng = np.random.default_rng(seed)
    box = (2.0, 1.0, 2.0)
    nx, ny, nz = n, n // 2, n
    h = box[0] / nx
    parts = [quad_mesh(0.05, 0.0, 2.0, 0.0, 2.0)]
    kinds = ("sphere", "box", "torus")
    for i in range(n_prims):
        Vp, Tp = {"sphere": lambda: icosphere(2), "box": box_mesh,
                  "torus": lambda: torus_mesh(16, 8, 0.3)}[kinds[i % 3]]()
        c = np.array([rng.uniform(0.2, 1.8), rng.uniform(0.2, 0.8), rng.uniform(0.2, 1.8)])
        s = rng.uniform(0.08, 0.3)
        R = random_rotation(rng)
        parts.append(((Vp * s) @ R.T + c, Tp))
    V, T = merge(parts)
    g = Grid(nx, ny, nz, (0.0, 0.0, 0.0), h)
    pos, nrm = receivers_plane(0.05, 0.0, 2.0, 0.0, 2.0, 96, 54)
    return Scene(f"small-room-{nx}x{ny}x{nz}", V.astype(np.float32), T, g,
                 RefineParams(mask_vox=4.0, rays_per_voxel=8, max_ray_vox=8.0, beta_vox=1.0,
                              accumulate=True, key=(0x12345678, 0x9abcdef0)),
                 ShadowParams(steps=96, max_step_vox=0.05 / h),
                 jfa_steps(g, extra_one=True), 2, pos, nrm)


@dataclasses.dataclass
class DiffScene:
    """A scene for the adjoint: the forward's inputs plus the loss's sample points
    and the vertices of the target copy (Gaussian-perturbed)."""
    scene: Scene
    pts: np.ndarray           # float32 [M,3] world sample points
    verts_target: np.ndarray  # float32 [V,3]


def scene_diff(n: int = 128, subdiv: int = 3, n_spheres: int = 8, n_boxes: int = 2, seed: int = 1010,
               n_samples: int = 65_536, shadow_res: int = 512, noise: float = 0.01) -> DiffScene:
    """Unit cube, n^3 grid; icospheres (radius 0.08-0.15) and boxes (half-extent
    0.05-0.12, random rotation) at seeded positions; uniform sample points; a
    receiver plane at y = 0.05 under them; the target copy has every vertex moved
    by N(0, noise^2) per coordinate."""
    rng = np.random.default_rng(seed)
    Vs, Ts = icosphere(subdiv)
    parts = []
    for _ in range(n_spheres):
        c = rng.uniform(0.2, 0.8, size=3)
        parts.append((Vs * rng.uniform(0.08, 0.15) + c, Ts))
    Vb, Tb = box_mesh()
    for _ in range(n_boxes):
        c = rng.uniform(0.25, 0.75, size=3)
        parts.append(((Vb * rng.uniform(0.05, 0.12)) @ random_rotation(rng).T + c, Tb))
    V, T = merge(parts)
    V = V.astype(np.float32)
    g = Grid(n, n, n, (0.0, 0.0, 0.0), 1.0 / n)
    pos, nrm = receivers_plane(0.05, 0.0, 1.0, 0.0, 1.0, shadow_res, shadow_res)
    sc = Scene(f"diff-{n}^3", V, T, g,
               RefineParams(mask_vox=3.0, rays_per_voxel=8, max_ray_vox=8.0, beta_vox=1.0, key=(0x2210, 0x6160)),
               ShadowParams(steps=64, max_step_vox=0.05 / g.h),
               jfa_steps(g), 1, pos, nrm)
    pts = rng.uniform(0.0, 1.0, size=(n_samples, 3)).astype(np.float32)
    vt = (V + rng.normal(0.0, noise, size=V.shape)).astype(np.float32)
    return DiffScene(sc, pts, vt)


BATCH_DIMS = ((32, 32, 32), (64, 64, 64), (128, 128, 128), (96, 48, 96), (200, 100, 200), (256, 128, 256))


def scene_batch(n: int = 48, seed: int = 4848, dims_choices=BATCH_DIMS, tri_range=(500, 60_000),
                rays: int = 8, shadow_res: int = 16) -> list[Scene]:
    """Seeded scenes of uneven sizes for the batched rebuild: grid dims drawn from
    `dims_choices` (h = 2 / largest dim, so each box is at most 2 wide), a ground
    quad plus primitives of the room mix (icospheres, boxes, tori) with random
    pose and scale 0.05-0.3 added until the scene holds a triangle count drawn
    uniformly from `tri_range`; scene i has scene id i."""
    rng = np.random.default_rng(seed)
    kinds = [("sphere2", lambda: icosphere(2)), ("sphere3", lambda: icosphere(3)), ("sphere4", lambda: icosphere(4)),
             ("box", box_mesh), ("torus32", lambda: torus_mesh(32, 16, 0.3)), ("torus64", lambda: torus_mesh(64, 32, 0.3))]
    cache = {}
    out = []
    for i in range(n):
        nx, ny, nz = dims_choices[int(rng.integers(len(dims_choices)))]
        h = 2.0 / max(nx, ny, nz)
        box = (nx * h, ny * h, nz * h)
        target = int(rng.integers(tri_range[0], tri_range[1] + 1))
        parts = [quad_mesh(0.05 * box[1], 0.0, box[0], 0.0, box[2])]
        total = 2
        while total < target:
            name, make = kinds[int(rng.integers(len(kinds)))]
            if name not in cache:
                cache[name] = make()
            Vp, Tp = cache[name]
            c = np.array([rng.uniform(0.1, b - 0.1) for b in box])
            s = rng.uniform(0.05, 0.3)
            parts.append(((Vp * s) @ random_rotation(rng).T + c, Tp))
            total += len(Tp)
        V, T = merge(parts)
        g = Grid(nx, ny, nz, (0.0, 0.0, 0.0), h)
        pos, nrm = receivers_plane(0.05 * box[1], 0.0, box[0], 0.0, box[2], shadow_res, shadow_res)
        out.append(Scene(f"batch{i}-{nx}x{ny}x{nz}", V.astype(np.float32), T, g,
                         RefineParams(mask_vox=4.0, rays_per_voxel=rays, max_ray_vox=8.0, beta_vox=1.0,
                                      key=(0xB47C, 0x4848), scene_id=i),
                         ShadowParams(steps=64, max_step_vox=0.05 / h), jfa_steps(g), 1, pos, nrm))
    return out


def scene_batch_small(seed: int = 77) -> list[Scene]:
    """A few small scenes of ragged sizes whose oracle rebuilds finish in seconds."""
    dims = ((32, 32, 32), (24, 16, 20), (40, 24, 32), (17, 33, 9), (8, 8, 8), (33, 20, 27))
    rng = np.random.default_rng(seed)
    out = []
    for i, (nx, ny, nz) in enumerate(dims):
        h = 1.0 / max(nx, ny, nz)
        box = (nx * h, ny * h, nz * h)
        parts = [quad_mesh(0.1 * box[1], 0.0, box[0], 0.0, box[2])]
        for _ in range(1 + i % 3):
            Vp, Tp = (icosphere(1 + i % 2) if rng.uniform() < 0.6 else box_mesh())
            c = np.array([rng.uniform(0.2, 0.8) * b for b in box])
            parts.append(((Vp * rng.uniform(0.1, 0.3) * min(box)) @ random_rotation(rng).T + c, Tp))
        V, T = merge(parts)
        g = Grid(nx, ny, nz, (0.0, 0.0, 0.0), h)
        pos, nrm = receivers_plane(0.1 * box[1], 0.0, box[0], 0.0, box[2], 8, 8)
        out.append(Scene(f"small-batch{i}", V.astype(np.float32), T, g,
                         RefineParams(mask_vox=3.0, rays_per_voxel=5 + i, max_ray_vox=6.0, beta_vox=1.0,
                                      key=(0x51, 0x7), scene_id=100 + i),
                         ShadowParams(steps=32, max_step_vox=2.0), jfa_steps(g, extra_one=bool(i % 2)), 1, pos,
                         nrm))
    return out


def _axis_angle(w: np.ndarray) -> np.ndarray:
    """Rotation matrix of the rotation vector w (Rodrigues)."""
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.eye(3)
    k = w / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * (K @ K)


def _vertex_normals(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    fn = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    vn = np.zeros_like(V)
    for m in range(3):
        np.add.at(vn, T[:, m], fn)
    return vn / np.maximum(np.linalg.norm(vn, axis=1, keepdims=True), 1e-30)


@dataclasses.dataclass
class RoomAnimation:
    """The room scene set in motion: per primitive a seeded linear velocity (|v| <= vmax
    per frame, reflected at the walls) and angular velocity (<= wmax per frame); `ndeform`
    primitives also move every vertex along its rest normal by amp * sin(2 pi f / 60 + phase)."""
    scene: Scene                 # frame 0 (geometry, grid, parameters, receivers)
    ground: np.ndarray           # ground quad vertices
    poses: list                  # (unit V, T, centre, scale, rotation) per primitive
    vel: np.ndarray
    omega: np.ndarray
    deform: dict                 # primitive index -> (rest normals, phases)
    box: tuple
    amp: float


def room_animation(seed: int = 2210, nx: int = 400, ny: int = 200, nz: int = 400, n_prims: int = 40,
                   target_tris: int = 100_000, shadow_w: int = 1920, shadow_h: int = 1080, rays: int = 4,
                   vmax: float = 0.005, wmax_deg: float = 2.0, ndeform: int = 10, amp: float = 0.02,
                   motion_seed: int = 120) -> RoomAnimation:
    """The dynamic workload: the room of scene_room (same seed, so frame 0 is that scene)
    rebuilt every frame from scratch with `rays` rays per voxel and no carry-over."""
    rng = np.random.default_rng(seed)
    box = (2.0, 1.0, 2.0)
    h = box[0] / nx
    ground = quad_mesh(0.05, 0.0, 2.0, 0.0, 2.0)
    poses: list = []
    parts = [ground] + room_primitives(rng, n_prims, box, target_tris, poses=poses)
    V, T = merge(parts)
    g = Grid(nx, ny, nz, (0.0, 0.0, 0.0), h)
    pos, nrm = receivers_plane(0.05, 0.0, 2.0, 0.0, 2.0, shadow_w, shadow_h)
    sc = Scene(f"dynamic-room-{nx}x{ny}x{nz}", V.astype(np.float32), T, g,
               RefineParams(mask_vox=4.0, rays_per_voxel=rays, max_ray_vox=8.0, beta_vox=1.0, accumulate=False),
               ShadowParams(steps=96, max_step_vox=0.05 / h), jfa_steps(g, extra_one=True), 1, pos, nrm)
    mr = np.random.default_rng(motion_seed)
    n = len(poses)
    dirs = mr.normal(size=(n, 3))
    vel = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * mr.uniform(0, vmax, (n, 1))
    axes = mr.normal(size=(n, 3))
    omega = axes / np.linalg.norm(axes, axis=1, keepdims=True) * np.radians(mr.uniform(0, wmax_deg, (n, 1)))
    deform = {}
    for i in sorted(mr.choice(n, min(ndeform, n), replace=False).tolist()):
        Vu, Tu = poses[i][0], poses[i][1]
        deform[i] = (_vertex_normals(Vu, Tu), mr.uniform(0, 2 * math.pi, len(Vu)))
    return RoomAnimation(sc, ground[0], poses, vel, omega, deform, box, amp)


def _reflect(x: np.ndarray, lo: float, hi: float) -> np.ndarray:
    span = hi - lo
    y = np.mod(x - lo, 2 * span)
    return lo + np.where(y > span, 2 * span - y, y)


def room_frame(anim: RoomAnimation, f: int) -> np.ndarray:
    """World vertices of frame f (same triangles as anim.scene)."""
    out = [anim.ground]
    for i, (Vu, Tu, c, s, R) in enumerate(anim.poses):
        Vl = Vu
        if i in anim.deform:
            vn, ph = anim.deform[i]
            Vl = Vu + (anim.amp / s) * np.sin(2 * math.pi * f / 60.0 + ph)[:, None] * vn
        Rf = _axis_angle(anim.omega[i] * f) @ R
        cf = np.array([_reflect(np.array(c[a] + anim.vel[i, a] * f), 0.1, anim.box[a] - 0.1) for a in range(3)])
        out.append((Vl * s) @ Rf.T + cf)
    return np.concatenate(out).astype(np.float32)
