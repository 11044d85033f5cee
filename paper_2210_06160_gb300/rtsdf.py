"""Thin Python binding of librtsdf (include/rtsdf.h).

The functions carry the C-ABI names and only marshal arguments: torch CUDA
tensors are passed as device pointers on the current torch stream, every step of
the computation runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  There is no fallback: if the compiled library is missing or
no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librtsdf.so")

EMPTY = -1
MAX_DIM = 1023

_lock = threading.Lock()
_lib = None


class RtsdfError(RuntimeError):
    pass


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("origin", C.c_float * 3), ("h", C.c_float)]


class RefineParams(C.Structure):
    _fields_ = [("mask_vox", C.c_float), ("rays_per_voxel", C.c_int32), ("max_ray_vox", C.c_float),
                ("beta_vox", C.c_float), ("key", C.c_uint32 * 2), ("frame_index", C.c_uint32),
                ("scene_id", C.c_uint32), ("accumulate", C.c_int32), ("sign_fallback", C.c_int32),
                ("decay_alpha", C.c_float), ("count_work", C.c_int32)]


class ShadowParams(C.Structure):
    _fields_ = [("light_dir", C.c_float * 3), ("k", C.c_float), ("steps", C.c_int32),
                ("max_step_vox", C.c_float), ("start_offset_vox", C.c_float),
                ("normal_offset_vox", C.c_float), ("hit_eps_vox", C.c_float), ("bias_vox", C.c_float),
                ("jitter_vox", C.c_float), ("frame_index", C.c_uint32), ("light_dir_device", C.c_void_p)]


class Counters(C.Structure):
    _fields_ = [("skipped_triangles", C.c_uint32), ("masked_voxels", C.c_uint32),
                ("rays_hit", C.c_uint32), ("rays_failed", C.c_uint32),
                ("stack_overflow", C.c_uint32), ("near_edge_hits", C.c_uint32), ("reserved", C.c_uint32 * 2),
                ("node_tests", C.c_uint64), ("reach_tests", C.c_uint64), ("filter_pairs", C.c_uint64),
                ("exact_tests", C.c_uint64)]


COUNTER_FIELDS = [f for f, _ in Counters._fields_ if f != "reserved"]
COUNTER_WORDS = C.sizeof(Counters) // 4  # int32 words of a counters tensor

BATCH_MAX_SCENES = 64
BATCH_MAX_STEPS = 16


class BatchScene(C.Structure):
    _fields_ = [("grid", Grid), ("V", C.c_int32), ("T", C.c_int32), ("nsteps", C.c_int32),
                ("steps", C.c_int32 * BATCH_MAX_STEPS), ("refine", RefineParams)]


class BatchLayout(C.Structure):
    _fields_ = [("voxel_offset", C.c_int64), ("vertex_offset", C.c_int32), ("triangle_offset", C.c_int32),
                ("bvh_offset", C.c_int64), ("flooded_in_b", C.c_int32), ("reserved", C.c_int32)]


class BatchTuning(C.Structure):
    _fields_ = [("brick_x", C.c_int32), ("brick_y", C.c_int32), ("brick_z", C.c_int32),
                ("warps_per_cta", C.c_int32), ("use_graph", C.c_int32)]


class BatchBuffers(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("tris", C.c_void_p), ("seed", C.c_void_p), ("buf_b", C.c_void_p),
                ("rep_tri", C.c_void_p), ("bvh", C.c_void_p), ("bvh_bytes", C.c_size_t),
                ("dist_bits", C.c_void_p), ("front", C.c_void_p), ("back", C.c_void_p), ("sdf", C.c_void_p),
                ("ws", C.c_void_p), ("ws_bytes", C.c_size_t)]

_P = C.c_void_p
_SIGS = {
    "rtsdf_version": (C.c_int32, []),
    "rtsdf_kernel_launches": (C.c_uint64, []),
    "rtsdf_status_string": (C.c_char_p, [C.c_int]),
    "rtsdf_voxelize_workspace": (C.c_size_t, [C.c_int32, C.POINTER(Grid)]),
    "rtsdf_voxelize": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.POINTER(Grid), _P, _P, _P, C.c_size_t, _P, _P]),
    "rtsdf_bvh_bytes": (C.c_size_t, [C.c_int32]),
    "rtsdf_bvh_workspace": (C.c_size_t, [C.c_int32]),
    "rtsdf_build_bvh": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.POINTER(Grid), _P, C.c_size_t, _P, C.c_size_t,
                                  _P, _P]),
    "rtsdf_build_bvh_noalloc": (C.c_int, [_P, C.c_int32, _P, C.c_int32, C.POINTER(Grid), _P, C.c_size_t, _P, _P]),
    "rtsdf_jfa": (C.c_int, [C.POINTER(Grid), _P, _P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_void_p), _P]),
    "rtsdf_refine_workspace": (C.c_size_t, [C.POINTER(Grid)]),
    "rtsdf_refine": (C.c_int, [C.POINTER(Grid), _P, C.c_int32, _P, C.c_int32, _P, C.c_size_t, _P, _P,
                               C.POINTER(RefineParams), _P, _P, _P, _P, _P, C.c_size_t, _P, _P]),
    "rtsdf_refine_tracked": (C.c_int, [C.POINTER(Grid), _P, C.c_int32, _P, C.c_int32, _P, C.c_size_t, _P, _P,
                                       C.POINTER(RefineParams), _P, _P, _P, _P, _P, _P, _P, C.c_size_t, _P, _P]),
    "rtsdf_refine_2res": (C.c_int, [C.POINTER(Grid), C.POINTER(Grid), _P, C.c_int32, _P, C.c_int32, _P, C.c_size_t,
                                    _P, _P, C.POINTER(RefineParams), _P, _P, _P, _P, _P, C.c_size_t, _P, _P]),
    "rtsdf_shadow": (C.c_int, [C.POINTER(Grid), _P, _P, _P, C.c_int32, C.POINTER(ShadowParams), _P, _P]),
    "rtsdf_shadow_coherent": (C.c_int, [C.POINTER(Grid), _P, _P, _P, C.c_int32, C.POINTER(ShadowParams), _P, _P,
                                        _P]),
    "rtsdf_sample": (C.c_int, [C.POINTER(Grid), _P, _P, C.c_int32, _P, _P]),
    "rtsdf_texture_create": (C.c_int, [C.POINTER(Grid), C.POINTER(C.c_void_p)]),
    "rtsdf_texture_destroy": (None, [_P]),
    "rtsdf_texture_upload": (C.c_int, [_P, _P, _P]),
    "rtsdf_shadow_tex": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(ShadowParams), _P, _P]),
    "rtsdf_backward_workspace": (C.c_size_t, [C.POINTER(Grid)]),
    "rtsdf_backward": (C.c_int, [C.POINTER(Grid), _P, C.c_int32, _P, C.c_int32, _P, _P, _P, _P, _P, _P,
                                 C.POINTER(RefineParams), _P, _P, C.c_int32, _P, _P, _P, C.c_int32,
                                 C.POINTER(ShadowParams), _P, _P, _P, _P, C.c_size_t, _P]),
    "rtsdf_batch_plan_create": (C.c_int, [C.POINTER(BatchScene), C.c_int32, C.POINTER(C.c_void_p)]),
    "rtsdf_batch_plan_destroy": (None, [_P]),
    "rtsdf_batch_layout_of": (C.c_int, [_P, C.c_int32, C.POINTER(BatchLayout)]),
    "rtsdf_batch_voxels": (C.c_size_t, [_P]),
    "rtsdf_batch_bvh_bytes": (C.c_size_t, [_P]),
    "rtsdf_batch_workspace": (C.c_size_t, [_P]),
    "rtsdf_batch_get_tuning": (C.c_int, [_P, C.POINTER(BatchTuning)]),
    "rtsdf_batch_set_tuning": (C.c_int, [_P, C.POINTER(BatchTuning)]),
    "rtsdf_batch_rebuild": (C.c_int, [_P, C.POINTER(BatchBuffers), C.c_uint32, C.c_int32, _P, _P]),
    "rtsdf_batch_autotune": (C.c_int, [_P, C.POINTER(BatchBuffers), C.c_int32, C.POINTER(C.c_float), _P]),
}

BACKWARD_MAX_STEPS = 512


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RtsdfError(f"librtsdf.so not built ({LIB_PATH}); run `python -m paper_2210_06160_gb300.build`")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, what: str) -> None:
    if status != 0:
        msg = lib().rtsdf_status_string(status).decode()
        raise RtsdfError(f"{what} failed: {msg} ({status})")


def _dev(t: torch.Tensor | None, dtype, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise RtsdfError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise RtsdfError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise RtsdfError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def make_grid(g) -> Grid:
    """From any object with nx, ny, nz, origin, h (e.g. scenes.Grid)."""
    return Grid(int(g.nx), int(g.ny), int(g.nz), (C.c_float * 3)(*[float(v) for v in g.origin]), float(g.h))


def make_refine_params(rp, count_work: bool = False) -> RefineParams:
    return RefineParams(float(rp.mask_vox), int(rp.rays_per_voxel), float(rp.max_ray_vox), float(rp.beta_vox),
                        (C.c_uint32 * 2)(*[int(k) & 0xFFFFFFFF for k in rp.key]), int(rp.frame_index) & 0xFFFFFFFF,
                        int(rp.scene_id) & 0xFFFFFFFF, int(rp.accumulate), int(bool(rp.sign_fallback)),
                        float(getattr(rp, "decay_alpha", 0.95)), int(bool(count_work)))


def make_shadow_params(sp, light_device=None) -> ShadowParams:
    """light_device: optional CUDA float32 tensor of 3 elements that the kernels read
    for the light direction instead of sp.light_dir (the caller keeps it alive until
    they have run)."""
    ptr = None
    if light_device is not None:
        _dev(light_device, torch.float32, "light_device")
        if light_device.numel() != 3:
            raise RtsdfError("light_device must hold 3 floats")
        ptr = C.c_void_p(light_device.data_ptr())
    return ShadowParams((C.c_float * 3)(*[float(v) for v in sp.light_dir]), float(sp.k), int(sp.steps),
                        float(sp.max_step_vox), float(sp.start_offset_vox), float(sp.normal_offset_vox),
                        float(sp.hit_eps_vox), float(sp.bias_vox), float(getattr(sp, "jitter_vox", 0.0)),
                        int(getattr(sp, "frame_index", 0)) & 0xFFFFFFFF, ptr)


# ------------------------------------------------------------ size queries

def rtsdf_voxelize_workspace(T: int, grid: Grid) -> int:
    return int(lib().rtsdf_voxelize_workspace(int(T), C.byref(grid)))


def rtsdf_bvh_bytes(T: int) -> int:
    return int(lib().rtsdf_bvh_bytes(int(T)))


def rtsdf_bvh_workspace(T: int) -> int:
    return int(lib().rtsdf_bvh_workspace(int(T)))


def rtsdf_refine_workspace(grid: Grid) -> int:
    return int(lib().rtsdf_refine_workspace(C.byref(grid)))


def rtsdf_backward_workspace(grid: Grid) -> int:
    return int(lib().rtsdf_backward_workspace(C.byref(grid)))


# ------------------------------------------------------------ the calls

def rtsdf_voxelize(verts, tris, grid: Grid, seed, rep_tri, ws, counters=None, stream=None) -> None:
    _check(lib().rtsdf_voxelize(_dev(verts, torch.float32, "verts"), verts.shape[0],
                                _dev(tris, torch.int32, "tris"), tris.shape[0], C.byref(grid),
                                _dev(seed, torch.int32, "seed"), _dev(rep_tri, torch.int32, "rep_tri"),
                                _dev(ws, torch.uint8, "ws"), ws.numel(),
                                _dev(counters, torch.int32, "counters"), _stream(stream)), "rtsdf_voxelize")


def rtsdf_build_bvh(verts, tris, grid: Grid, bvh, ws, counters=None, stream=None) -> None:
    _check(lib().rtsdf_build_bvh(_dev(verts, torch.float32, "verts"), verts.shape[0],
                                 _dev(tris, torch.int32, "tris"), tris.shape[0], C.byref(grid),
                                 _dev(bvh, torch.uint8, "bvh"), bvh.numel(), _dev(ws, torch.uint8, "ws"), ws.numel(),
                                 _dev(counters, torch.int32, "counters"), _stream(stream)), "rtsdf_build_bvh")


def rtsdf_build_bvh_noalloc(verts, tris, grid: Grid, bvh, counters=None, stream=None) -> None:
    """rtsdf_build_bvh with the library's fixed internal scratch (no workspace);
    at most RTSDF_NOALLOC_MAX_TRIS triangles; overlapping calls race."""
    _check(lib().rtsdf_build_bvh_noalloc(_dev(verts, torch.float32, "verts"), verts.shape[0],
                                         _dev(tris, torch.int32, "tris"), tris.shape[0], C.byref(grid),
                                         _dev(bvh, torch.uint8, "bvh"), bvh.numel(),
                                         _dev(counters, torch.int32, "counters"), _stream(stream)),
           "rtsdf_build_bvh_noalloc")


def rtsdf_jfa(grid: Grid, buf_a, buf_b, steps, stream=None):
    """Runs the passes; returns the tensor (buf_a or buf_b) that holds the result."""
    arr = (C.c_int32 * max(1, len(steps)))(*[int(k) for k in steps])
    res = C.c_void_p()
    _check(lib().rtsdf_jfa(C.byref(grid), _dev(buf_a, torch.int32, "buf_a"), _dev(buf_b, torch.int32, "buf_b"),
                           arr, len(steps), C.byref(res), _stream(stream)), "rtsdf_jfa")
    return buf_a if res.value == buf_a.data_ptr() else buf_b


def rtsdf_refine(grid: Grid, verts, tris, bvh, nearest, rep_tri, params: RefineParams, dist_bits, front, back,
                 sdf_out, ws, counters=None, stream=None) -> None:
    _check(lib().rtsdf_refine(C.byref(grid), _dev(verts, torch.float32, "verts"), verts.shape[0],
                              _dev(tris, torch.int32, "tris"), tris.shape[0], _dev(bvh, torch.uint8, "bvh"),
                              bvh.numel(), _dev(nearest, torch.int32, "nearest"),
                              _dev(rep_tri, torch.int32, "rep_tri"), C.byref(params),
                              _dev(dist_bits, torch.int32, "dist_bits"), _dev(front, torch.int32, "front"),
                              _dev(back, torch.int32, "back"), _dev(sdf_out, torch.float32, "sdf_out"),
                              _dev(ws, torch.uint8, "ws"), ws.numel(), _dev(counters, torch.int32, "counters"),
                              _stream(stream)), "rtsdf_refine")


def rtsdf_refine_tracked(grid: Grid, verts, tris, bvh, nearest, rep_tri, params: RefineParams, dist_bits, front,
                         back, sdf_out, win_ray, win_tri, ws, counters=None, stream=None) -> None:
    """rtsdf_refine that also records the winning source of every voxel's distance."""
    _check(lib().rtsdf_refine_tracked(C.byref(grid), _dev(verts, torch.float32, "verts"), verts.shape[0],
                                      _dev(tris, torch.int32, "tris"), tris.shape[0], _dev(bvh, torch.uint8, "bvh"),
                                      bvh.numel(), _dev(nearest, torch.int32, "nearest"),
                                      _dev(rep_tri, torch.int32, "rep_tri"), C.byref(params),
                                      _dev(dist_bits, torch.int32, "dist_bits"), _dev(front, torch.int32, "front"),
                                      _dev(back, torch.int32, "back"), _dev(sdf_out, torch.float32, "sdf_out"),
                                      _dev(win_ray, torch.int32, "win_ray"), _dev(win_tri, torch.int32, "win_tri"),
                                      _dev(ws, torch.uint8, "ws"), ws.numel(), _dev(counters, torch.int32, "counters"),
                                      _stream(stream)), "rtsdf_refine_tracked")


def rtsdf_refine_2res(fine: Grid, coarse: Grid, verts, tris, bvh, nearest_c, rep_tri_c, params: RefineParams,
                      dist_bits, front, back, sdf_out, ws, counters=None, stream=None) -> None:
    """rtsdf_refine on the fine grid with flooded seeds / representative triangles of the coarse grid."""
    _check(lib().rtsdf_refine_2res(C.byref(fine), C.byref(coarse), _dev(verts, torch.float32, "verts"),
                                   verts.shape[0], _dev(tris, torch.int32, "tris"), tris.shape[0],
                                   _dev(bvh, torch.uint8, "bvh"), bvh.numel(), _dev(nearest_c, torch.int32, "nearest"),
                                   _dev(rep_tri_c, torch.int32, "rep_tri"), C.byref(params),
                                   _dev(dist_bits, torch.int32, "dist_bits"), _dev(front, torch.int32, "front"),
                                   _dev(back, torch.int32, "back"), _dev(sdf_out, torch.float32, "sdf_out"),
                                   _dev(ws, torch.uint8, "ws"), ws.numel(), _dev(counters, torch.int32, "counters"),
                                   _stream(stream)), "rtsdf_refine_2res")


def rtsdf_sample(grid: Grid, sdf, pts, out, stream=None) -> None:
    _check(lib().rtsdf_sample(C.byref(grid), _dev(sdf, torch.float32, "sdf"), _dev(pts, torch.float32, "pts"),
                              pts.shape[0], _dev(out, torch.float32, "out"), _stream(stream)), "rtsdf_sample")


def rtsdf_backward(grid: Grid, verts, tris, nearest, rep_tri, front, back, win_ray, win_tri, rparams: RefineParams,
                   sdf, pts, d_samples, pos, nrm, sparams: ShadowParams, d_vis, d_verts, d_light, ws,
                   stream=None) -> None:
    M = 0 if pts is None else pts.shape[0]
    P = 0 if pos is None else pos.shape[0]
    _check(lib().rtsdf_backward(C.byref(grid), _dev(verts, torch.float32, "verts"), verts.shape[0],
                                _dev(tris, torch.int32, "tris"), tris.shape[0],
                                _dev(nearest, torch.int32, "nearest"), _dev(rep_tri, torch.int32, "rep_tri"),
                                _dev(front, torch.int32, "front"), _dev(back, torch.int32, "back"),
                                _dev(win_ray, torch.int32, "win_ray"), _dev(win_tri, torch.int32, "win_tri"),
                                C.byref(rparams), _dev(sdf, torch.float32, "sdf"),
                                _dev(pts, torch.float32, "pts"), M, _dev(d_samples, torch.float32, "d_samples"),
                                _dev(pos, torch.float32, "pos"), _dev(nrm, torch.float32, "nrm"), P,
                                C.byref(sparams), _dev(d_vis, torch.float32, "d_vis"),
                                _dev(d_verts, torch.float32, "d_verts"), _dev(d_light, torch.float32, "d_light"),
                                _dev(ws, torch.uint8, "ws"), ws.numel(), _stream(stream)), "rtsdf_backward")


def rtsdf_shadow(grid: Grid, sdf, pos, nrm, params: ShadowParams, vis, stream=None) -> None:
    _check(lib().rtsdf_shadow(C.byref(grid), _dev(sdf, torch.float32, "sdf"), _dev(pos, torch.float32, "pos"),
                              _dev(nrm, torch.float32, "nrm"), pos.shape[0], C.byref(params),
                              _dev(vis, torch.float32, "vis"), _stream(stream)), "rtsdf_shadow")


def rtsdf_shadow_coherent(grid: Grid, sdf, pos, nrm, params: ShadowParams, vis, steps, stream=None) -> None:
    _check(lib().rtsdf_shadow_coherent(C.byref(grid), _dev(sdf, torch.float32, "sdf"),
                                       _dev(pos, torch.float32, "pos"), _dev(nrm, torch.float32, "nrm"),
                                       pos.shape[0], C.byref(params), _dev(vis, torch.float32, "vis"),
                                       _dev(steps, torch.uint8, "steps"), _stream(stream)), "rtsdf_shadow_coherent")


def rtsdf_kernel_launches() -> int:
    return int(lib().rtsdf_kernel_launches())


def new_counters(device) -> torch.Tensor:
    """A zeroed device counters block (rtsdf_counters) as int32 words."""
    return torch.zeros(COUNTER_WORDS, dtype=torch.int32, device=device)


def counters_dict(counters: torch.Tensor) -> dict:
    raw = Counters.from_buffer_copy(counters.cpu().numpy().tobytes()[:C.sizeof(Counters)])
    return {f: int(getattr(raw, f)) for f in COUNTER_FIELDS}


# ------------------------------------------------------------ a frame pipeline

class Pipeline:
    """Owns the device buffers of one scene size and runs the hot path through the
    C-ABI: voxelize -> BVH -> jump flood -> refine (one frame) -> shadow.

    uint32 state (dist_bits, front, back) is held in int32 tensors of the same bits.
    """

    def __init__(self, grid, n_verts: int, n_tris: int, device="cuda", track: bool = False):
        self.g = make_grid(grid)
        self.T, self.V = int(n_tris), int(n_verts)
        dev = torch.device(device)
        shp = (grid.nz, grid.ny, grid.nx)
        i32 = dict(dtype=torch.int32, device=dev)
        self.buf_a = torch.empty(shp, **i32)
        self.buf_b = torch.empty(shp, **i32)
        self.rep_tri = torch.empty(shp, **i32)
        # refine state of "no earlier frame": distance +inf, no votes, so that the
        # first call may already accumulate
        self.dist_bits = torch.full(shp, 0x7F800000, **i32)
        self.front = torch.zeros(shp, **i32)
        self.back = torch.zeros(shp, **i32)
        self.sdf = torch.empty(shp, dtype=torch.float32, device=dev)
        self.counters = new_counters(dev)
        u8 = dict(dtype=torch.uint8, device=dev)
        self.ws_vox = torch.empty(rtsdf_voxelize_workspace(self.T, self.g), **u8)
        self.bvh = torch.empty(rtsdf_bvh_bytes(self.T), **u8)
        self.ws_bvh = torch.empty(rtsdf_bvh_workspace(self.T), **u8)
        self.ws_refine = torch.empty(rtsdf_refine_workspace(self.g), **u8)
        self.nearest = None
        # winner record for the adjoint (rtsdf_refine_tracked)
        self.track = bool(track)
        self.win_ray = torch.empty(shp, **i32) if track else None
        self.win_tri = torch.empty(shp, **i32) if track else None
        self.generation = 0  # bumped by every call that changes the field

    def voxelize(self, verts, tris, stream=None):
        rtsdf_voxelize(verts, tris, self.g, self.buf_a, self.rep_tri, self.ws_vox, self.counters, stream)
        return self.buf_a

    def build_bvh(self, verts, tris, stream=None):
        rtsdf_build_bvh(verts, tris, self.g, self.bvh, self.ws_bvh, self.counters, stream)

    def jfa(self, steps, stream=None):
        self.nearest = rtsdf_jfa(self.g, self.buf_a, self.buf_b, steps, stream)
        return self.nearest

    def refine(self, verts, tris, params: RefineParams, stream=None):
        self.generation += 1
        if self.track:
            rtsdf_refine_tracked(self.g, verts, tris, self.bvh, self.nearest, self.rep_tri, params, self.dist_bits,
                                 self.front, self.back, self.sdf, self.win_ray, self.win_tri, self.ws_refine,
                                 self.counters, stream)
        else:
            rtsdf_refine(self.g, verts, tris, self.bvh, self.nearest, self.rep_tri, params, self.dist_bits,
                         self.front, self.back, self.sdf, self.ws_refine, self.counters, stream)
        return self.sdf

    def rebuild(self, verts, tris, steps, params: RefineParams, stream=None, overlap: bool = True):
        """One frame: voxelize -> jump flood -> refine; with `overlap` the BVH is built
        on a second stream while the seeds are voxelized and flooded (the BVH's small
        kernels leave most of the GPU idle), and the refinement waits for both."""
        s = torch.cuda.current_stream(self.bvh.device) if stream is None else stream
        if not overlap:
            self.voxelize(verts, tris, s)
            self.build_bvh(verts, tris, s)
            self.jfa(steps, s)
            return self.refine(verts, tris, params, s)
        side = self.side_stream()
        ready = torch.cuda.Event()
        ready.record(s)
        side.wait_event(ready)
        self.build_bvh(verts, tris, side)
        built = torch.cuda.Event()
        built.record(side)
        self.voxelize(verts, tris, s)
        self.jfa(steps, s)
        s.wait_event(built)
        return self.refine(verts, tris, params, s)

    def side_stream(self):
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=self.bvh.device)
        return self._side

    def shadow(self, pos, nrm, params: ShadowParams, vis=None, stream=None, coherent: bool = True):
        """The raymarch of every receiver; `coherent` regroups the receivers by the
        march lengths of this pipeline's previous call (same results, fewer idle lanes)."""
        if vis is None:
            vis = torch.empty(pos.shape[0], dtype=torch.float32, device=pos.device)
        if coherent:
            steps = getattr(self, "_march_steps", None)
            if steps is None or steps.numel() != pos.shape[0] or steps.device != pos.device:
                steps = self._march_steps = torch.zeros(pos.shape[0], dtype=torch.uint8, device=pos.device)
            rtsdf_shadow_coherent(self.g, self.sdf, pos, nrm, params, vis, steps, stream)
        else:
            rtsdf_shadow(self.g, self.sdf, pos, nrm, params, vis, stream)
        return vis

    def sample(self, pts, out=None, stream=None):
        if out is None:
            out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
        rtsdf_sample(self.g, self.sdf, pts, out, stream)
        return out


class SdfTexture:
    """The field as a 3D texture with hardware trilinear filtering (rtsdf_texture_*)."""

    def __init__(self, grid):
        self.g = make_grid(grid)
        self.handle = C.c_void_p()
        _check(lib().rtsdf_texture_create(C.byref(self.g), C.byref(self.handle)), "rtsdf_texture_create")

    def upload(self, sdf, stream=None):
        _check(lib().rtsdf_texture_upload(self.handle, _dev(sdf, torch.float32, "sdf"), _stream(stream)),
               "rtsdf_texture_upload")

    def shadow(self, pos, nrm, params: ShadowParams, vis=None, stream=None):
        if vis is None:
            vis = torch.empty(pos.shape[0], dtype=torch.float32, device=pos.device)
        _check(lib().rtsdf_shadow_tex(self.handle, _dev(pos, torch.float32, "pos"), _dev(nrm, torch.float32, "nrm"),
                                      pos.shape[0], C.byref(params), _dev(vis, torch.float32, "vis"),
                                      _stream(stream)), "rtsdf_shadow_tex")
        return vis

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib().rtsdf_texture_destroy(h)
            except Exception:
                pass
            self.handle = None


class TwoResPipeline:
    """Sec. 2.5.1 two resolutions: voxelize and jump-flood on a coarse grid, resolve and
    refine on a fine grid over the same box (coarse h = r * fine h)."""

    def __init__(self, fine, coarse, n_verts: int, n_tris: int, device="cuda"):
        self.coarse = Pipeline(coarse, n_verts, n_tris, device=device)   # seeds, flooding, rep_tri
        self.fine = Pipeline(fine, n_verts, n_tris, device=device)       # BVH, state, field
        self.gf, self.gc = make_grid(fine), make_grid(coarse)

    @property
    def sdf(self):
        return self.fine.sdf

    def rebuild(self, verts, tris, coarse_steps, params: RefineParams, stream=None):
        self.coarse.voxelize(verts, tris, stream)
        self.fine.build_bvh(verts, tris, stream)
        near = self.coarse.jfa(coarse_steps, stream)
        f = self.fine
        rtsdf_refine_2res(self.gf, self.gc, verts, tris, f.bvh, near, self.coarse.rep_tri, params, f.dist_bits,
                          f.front, f.back, f.sdf, f.ws_refine, f.counters, stream)
        return f.sdf

    def shadow(self, pos, nrm, params: ShadowParams, vis=None, stream=None):
        return self.fine.shadow(pos, nrm, params, vis, stream)


# ------------------------------------------------------------ differentiation

class SDFShadow(torch.autograd.Function):
    """(samples, vis) = field samples at `pts` and soft-shadow visibility of the
    receivers, for a mesh whose field is rebuilt on `pipe` (voxelize, BVH, jump
    flood, then one tracked refine per entry of `frames`); differentiable in the
    vertices and the light direction through rtsdf_backward.

    verts: CUDA float32 [V,3] world positions; light: float32 [3] tensor.  On the
    GPU, the kernels read it where it lives (nothing is copied to the host, so a
    forward and backward enqueue without synchronising); on the CPU its value
    parameterises the launches.  The backward must run before `pipe` builds another
    field.
    """

    @staticmethod
    def forward(ctx, verts, light, pipe, tris, jfa_steps, frames, pts, pos, nrm, shadow):
        if not pipe.track:
            raise RtsdfError("SDFShadow needs a Pipeline created with track=True")
        if int(shadow.steps) > BACKWARD_MAX_STEPS:
            raise RtsdfError(f"the adjoint replays at most {BACKWARD_MAX_STEPS} raymarch steps")
        import dataclasses
        light_dev = None
        if light.is_cuda:
            light_dev = light.detach().to(torch.float32).contiguous()
            sp = shadow  # its light_dir is not read: the kernels take light_dev
        else:
            sp = dataclasses.replace(shadow, light_dir=tuple(float(v) for v in light.detach().tolist()))
        verts_c = verts.detach().contiguous()
        rparams = None
        for f, rp in enumerate(frames):
            rparams = make_refine_params(rp)
            if f == 0:
                pipe.rebuild(verts_c, tris, jfa_steps, rparams)  # BVH overlapped with voxelize + JFA
            else:
                pipe.refine(verts_c, tris, rparams)
        samples = pipe.sample(pts)
        vis = pipe.shadow(pos, nrm, make_shadow_params(sp, light_dev))
        ctx.pipe, ctx.gen = pipe, pipe.generation
        ctx.rparams, ctx.sparams = rparams, make_shadow_params(sp, light_dev)
        ctx.light_dev = light_dev  # kept alive for the backward's launches
        ctx.tris, ctx.pts, ctx.pos, ctx.nrm = tris, pts, pos, nrm
        ctx.light_device = light.device
        ctx.save_for_backward(verts_c)
        return samples, vis

    @staticmethod
    def backward(ctx, d_samples, d_vis):
        (verts,) = ctx.saved_tensors
        pipe = ctx.pipe
        if pipe.generation != ctx.gen:
            raise RtsdfError("the pipeline built another field since this forward; its adjoint is gone")
        dev = verts.device
        ds = torch.zeros(ctx.pts.shape[0], dtype=torch.float32, device=dev) if d_samples is None \
            else d_samples.to(torch.float32).contiguous()
        dv = torch.zeros(ctx.pos.shape[0], dtype=torch.float32, device=dev) if d_vis is None \
            else d_vis.to(torch.float32).contiguous()
        d_verts = torch.empty_like(verts)
        d_light = torch.empty(3, dtype=torch.float32, device=dev)
        ws = torch.empty(rtsdf_backward_workspace(pipe.g), dtype=torch.uint8, device=dev)
        rtsdf_backward(pipe.g, verts, ctx.tris, pipe.nearest, pipe.rep_tri, pipe.front, pipe.back, pipe.win_ray,
                       pipe.win_tri, ctx.rparams, pipe.sdf, ctx.pts, ds, ctx.pos, ctx.nrm, ctx.sparams, dv,
                       d_verts, d_light, ws)
        return (d_verts, d_light.to(ctx.light_device), None, None, None, None, None, None, None, None)


def sdf_shadow(verts, light, pipe, tris, jfa_steps, frames, pts, pos, nrm, shadow):
    """Differentiable field samples and shadow image (see SDFShadow)."""
    return SDFShadow.apply(verts, light, pipe, tris, jfa_steps, frames, pts, pos, nrm, shadow)


# ------------------------------------------------------------ batched rebuild

def make_batch_scene(grid, n_verts: int, n_tris: int, steps, refine) -> BatchScene:
    steps = [int(k) for k in steps]
    if len(steps) > BATCH_MAX_STEPS:
        raise RtsdfError(f"at most {BATCH_MAX_STEPS} JFA steps per scene")
    arr = (C.c_int32 * BATCH_MAX_STEPS)(*(steps + [0] * (BATCH_MAX_STEPS - len(steps))))
    return BatchScene(make_grid(grid), int(n_verts), int(n_tris), len(steps), arr, make_refine_params(refine))


def rtsdf_batch_plan_create(scenes: list) -> C.c_void_p:
    arr = (BatchScene * len(scenes))(*scenes)
    plan = C.c_void_p()
    _check(lib().rtsdf_batch_plan_create(arr, len(scenes), C.byref(plan)), "rtsdf_batch_plan_create")
    return plan


def rtsdf_batch_rebuild(plan, buffers: BatchBuffers, frame_index: int, accumulate: int, counters=None,
                        stream=None) -> None:
    """accumulate: 0 fresh, 1 (or True) minimum over frames, 2 the Eq. (1) decay with each scene's alpha."""
    _check(lib().rtsdf_batch_rebuild(plan, C.byref(buffers), int(frame_index) & 0xFFFFFFFF, int(accumulate),
                                     _dev(counters, torch.int32, "counters"), _stream(stream)), "rtsdf_batch_rebuild")


def rtsdf_batch_autotune(plan, buffers: BatchBuffers, reps: int = 3, stream=None) -> float:
    ms = C.c_float()
    _check(lib().rtsdf_batch_autotune(plan, C.byref(buffers), int(reps), C.byref(ms), _stream(stream)),
           "rtsdf_batch_autotune")
    return float(ms.value)


class Batch:
    """Device buffers and plan of a batch of scenes (rtsdf_batch_*): meshes are
    concatenated scene by scene, grids laid out at the plan's voxel offsets.

    `scenes`: objects with grid, verts [V,3], tris [T,3] (indices local to the
    scene), jfa_steps and refine (e.g. scenes.Scene); scene ids come from each
    scene's refine parameters.
    """

    def __init__(self, scenes: list, device="cuda"):
        if not 1 <= len(scenes) <= BATCH_MAX_SCENES:
            raise RtsdfError(f"a batch holds 1..{BATCH_MAX_SCENES} scenes")
        self.scenes = scenes
        self.desc = [make_batch_scene(sc.grid, len(sc.verts), len(sc.tris), sc.jfa_steps, sc.refine) for sc in scenes]
        self.plan = rtsdf_batch_plan_create(self.desc)
        L = lib()
        self.layout = []
        for i in range(len(scenes)):
            lay = BatchLayout()
            _check(L.rtsdf_batch_layout_of(self.plan, i, C.byref(lay)), "rtsdf_batch_layout_of")
            self.layout.append(lay)
        dev = torch.device(device)
        self.nvox = int(L.rtsdf_batch_voxels(self.plan))
        import numpy as np
        self.verts = torch.from_numpy(np.concatenate([np.asarray(sc.verts, np.float32) for sc in scenes])
                                      .reshape(-1, 3)).to(dev)
        self.tris = torch.from_numpy(np.concatenate([np.asarray(sc.tris, np.int32) for sc in scenes])
                                     .reshape(-1, 3)).to(dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self.seed = torch.empty(self.nvox, **i32)
        self.buf_b = torch.empty(self.nvox, **i32)
        self.rep_tri = torch.empty(self.nvox, **i32)
        self.dist_bits = torch.full((self.nvox,), 0x7F800000, **i32)
        self.front = torch.zeros(self.nvox, **i32)
        self.back = torch.zeros(self.nvox, **i32)
        self.sdf = torch.empty(self.nvox, dtype=torch.float32, device=dev)
        self.bvh = torch.empty(max(256, int(L.rtsdf_batch_bvh_bytes(self.plan))), dtype=torch.uint8, device=dev)
        self.ws = torch.empty(int(L.rtsdf_batch_workspace(self.plan)), dtype=torch.uint8, device=dev)
        self.counters = new_counters(dev)
        self.buffers = BatchBuffers(self.verts.data_ptr(), self.tris.data_ptr(), self.seed.data_ptr(),
                                    self.buf_b.data_ptr(), self.rep_tri.data_ptr(), self.bvh.data_ptr(),
                                    self.bvh.numel(), self.dist_bits.data_ptr(), self.front.data_ptr(),
                                    self.back.data_ptr(), self.sdf.data_ptr(), self.ws.data_ptr(), self.ws.numel())

    def rebuild(self, frame_index: int = 0, accumulate: int = 0, stream=None):
        rtsdf_batch_rebuild(self.plan, self.buffers, frame_index, accumulate, self.counters, stream)

    def autotune(self, reps: int = 3, stream=None) -> float:
        return rtsdf_batch_autotune(self.plan, self.buffers, reps, stream)

    @property
    def tuning(self) -> dict:
        t = BatchTuning()
        _check(lib().rtsdf_batch_get_tuning(self.plan, C.byref(t)), "rtsdf_batch_get_tuning")
        return {f: int(getattr(t, f)) for f, _ in BatchTuning._fields_}

    def set_tuning(self, brick=(4, 4, 4), warps_per_cta=2, use_graph=True):
        t = BatchTuning(int(brick[0]), int(brick[1]), int(brick[2]), int(warps_per_cta), int(bool(use_graph)))
        _check(lib().rtsdf_batch_set_tuning(self.plan, C.byref(t)), "rtsdf_batch_set_tuning")

    def view(self, i: int, name: str) -> torch.Tensor:
        """Scene i's slice of a batch grid array, shaped (nz, ny, nx); 'nearest' is
        the buffer holding its flooded seeds."""
        sc, lay = self.scenes[i], self.layout[i]
        g = sc.grid
        if name == "nearest":
            name = "buf_b" if lay.flooded_in_b else "seed"
        a = getattr(self, name)
        o = int(lay.voxel_offset)
        return a[o:o + g.nx * g.ny * g.nz].view(g.nz, g.ny, g.nx)

    def __del__(self):
        plan = getattr(self, "plan", None)
        if plan is not None and plan.value:
            try:
                lib().rtsdf_batch_plan_destroy(plan)
            except Exception:
                pass
            self.plan = None
