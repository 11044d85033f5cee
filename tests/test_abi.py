"""The C-ABI library builds, loads without a GPU, exports every entry point that
include/rtsdf.h declares, and rejects bad arguments before touching any memory
(fake device addresses are never dereferenced on these paths)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_06160_gb300 import build, rtsdf
    build.build()
    return rtsdf.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rtsdf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtsdf_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_status_strings(lib):
    assert lib.rtsdf_version() >= 100
    assert lib.rtsdf_status_string(0) == b"ok"
    assert b"invalid" in lib.rtsdf_status_string(1)


FAKE = 0x7F0000000000  # 256-byte aligned, never dereferenced


def _grid(nx=8, ny=8, nz=8, h=0.1):
    from paper_2210_06160_gb300.rtsdf import Grid
    return Grid(nx, ny, nz, (C.c_float * 3)(0, 0, 0), h)


def test_grid_validation(lib):
    from paper_2210_06160_gb300.rtsdf import Grid
    bad = [_grid(0, 8, 8), _grid(8, 1024, 8), _grid(8, 8, 8, 0.0), _grid(8, 8, 8, float("nan")),
           Grid(8, 8, 8, (C.c_float * 3)(0, float("inf"), 0), 0.1)]
    for g in bad:
        assert lib.rtsdf_voxelize_workspace(10, C.byref(g)) == 0
        assert lib.rtsdf_voxelize(C.c_void_p(FAKE), 3, C.c_void_p(FAKE), 1, C.byref(g), C.c_void_p(FAKE),
                                  C.c_void_p(FAKE), C.c_void_p(FAKE), 1 << 40, None, None) == 1
    g = _grid()
    assert lib.rtsdf_voxelize_workspace(10, C.byref(g)) > 8 * 512


def test_pointer_and_size_validation(lib):
    g = _grid()
    ws = lib.rtsdf_voxelize_workspace(4, C.byref(g))
    P = C.c_void_p
    # misaligned grid buffer
    assert lib.rtsdf_voxelize(P(FAKE), 3, P(FAKE), 1, C.byref(g), P(FAKE + 4), P(FAKE), P(FAKE), ws, None, None) == 1
    # null triangles with T > 0
    assert lib.rtsdf_voxelize(P(FAKE), 3, None, 1, C.byref(g), P(FAKE), P(FAKE), P(FAKE), ws, None, None) == 1
    # negative counts
    assert lib.rtsdf_voxelize(P(FAKE), -1, P(FAKE), 1, C.byref(g), P(FAKE), P(FAKE), P(FAKE), ws, None, None) == 1
    # workspace too small
    assert lib.rtsdf_voxelize(P(FAKE), 3, P(FAKE), 4, C.byref(g), P(FAKE), P(FAKE), P(FAKE), ws - 1, None,
                              None) == 2
    T = 100
    assert lib.rtsdf_build_bvh(P(FAKE), 3, P(FAKE), T, C.byref(g), P(FAKE), lib.rtsdf_bvh_bytes(T) - 1, P(FAKE),
                               lib.rtsdf_bvh_workspace(T), None, None) == 2


def test_bvh_buffer_holds_tree_leaves_and_triangle_table(lib):
    """The BVH buffer grows linearly in T: per triangle at least an inner node (64 B), a leaf (80 B)
    and a voxel-space triangle record (48 B), plus a fixed header."""
    sizes = [lib.rtsdf_bvh_bytes(T) for T in (1, 1000, 2000, 100_000)]
    assert sizes[0] > 0
    assert sizes[2] - sizes[1] == 1000 * (64 + 80 + 48)
    assert sizes[3] >= 100_000 * (64 + 80 + 48)
    assert lib.rtsdf_bvh_bytes(-1) == 0


def test_jfa_validation(lib):
    g = _grid()
    P = C.c_void_p
    res = C.c_void_p()
    steps = (C.c_int32 * 2)(4, 0)
    assert lib.rtsdf_jfa(C.byref(g), P(FAKE), P(FAKE + 4096), steps, 2, C.byref(res), None) == 1  # step 0
    steps = (C.c_int32 * 1)(4)
    assert lib.rtsdf_jfa(C.byref(g), P(FAKE), P(FAKE), steps, 1, C.byref(res), None) == 1  # aliased buffers
    assert lib.rtsdf_jfa(C.byref(g), P(FAKE), P(FAKE + 4096), steps, -1, C.byref(res), None) == 1
    # zero passes: nothing enqueued, result is buf_a
    assert lib.rtsdf_jfa(C.byref(g), P(FAKE), P(FAKE + 4096), steps, 0, C.byref(res), None) == 0
    assert res.value == FAKE


def test_refine_and_shadow_parameter_validation(lib):
    from paper_2210_06160_gb300.rtsdf import RefineParams, ShadowParams
    g = _grid()
    P = C.c_void_p
    ws = lib.rtsdf_refine_workspace(C.byref(g))
    bvh = lib.rtsdf_bvh_bytes(1)
    for rp in (RefineParams(3.0, 0, 8.0, 1.0), RefineParams(-1.0, 8, 8.0, 1.0), RefineParams(3.0, 8, 0.0, 1.0)):
        assert lib.rtsdf_refine(C.byref(g), P(FAKE), 3, P(FAKE), 1, P(FAKE), bvh, P(FAKE), P(FAKE), C.byref(rp),
                                P(FAKE), P(FAKE), P(FAKE), P(FAKE), P(FAKE), ws, None, None) == 1
    rp = RefineParams(3.0, 8, 8.0, 1.0)
    assert lib.rtsdf_refine(C.byref(g), P(FAKE), 3, P(FAKE), 1, P(FAKE), bvh, P(FAKE), P(FAKE), C.byref(rp),
                            P(FAKE), P(FAKE), P(FAKE), P(FAKE), P(FAKE), ws - 1, None, None) == 2
    sp = ShadowParams((C.c_float * 3)(0, 0, 0), 8.0, 10, 1.0)
    assert lib.rtsdf_shadow(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 4, C.byref(sp), P(FAKE), None) == 1
    sp = ShadowParams((C.c_float * 3)(0, 1, 0), 8.0, 10, 0.0)
    assert lib.rtsdf_shadow(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 4, C.byref(sp), P(FAKE), None) == 1
    # the regrouped march: the same checks, and its march-length buffer must be given
    ok = ShadowParams((C.c_float * 3)(0, 1, 0), 8.0, 10, 1.0)
    assert lib.rtsdf_shadow_coherent(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 4, C.byref(sp), P(FAKE), P(FAKE),
                                     None) == 1
    assert lib.rtsdf_shadow_coherent(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 4, C.byref(ok), P(FAKE), None,
                                     None) == 1
    # a light read on the device: light_dir is then not looked at, the pointer must be 4-byte aligned
    dev = ShadowParams((C.c_float * 3)(0, 0, 0), 8.0, 10, 1.0)
    dev.light_dir_device = FAKE
    assert lib.rtsdf_shadow(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 0, C.byref(dev), P(FAKE), None) == 0
    dev.light_dir_device = FAKE + 2
    assert lib.rtsdf_shadow(C.byref(g), P(FAKE), P(FAKE), P(FAKE), 0, C.byref(dev), P(FAKE), None) == 1


def test_adjoint_entry_validation(lib):
    from paper_2210_06160_gb300.rtsdf import RefineParams, ShadowParams
    g = _grid()
    P = C.c_void_p
    rp = RefineParams(3.0, 8, 8.0, 1.0)
    ws = lib.rtsdf_backward_workspace(C.byref(g))
    assert ws >= 4 * 8 * 8 * 8
    refine_ws = lib.rtsdf_refine_workspace(C.byref(g))
    bvh = lib.rtsdf_bvh_bytes(1)
    # tracked refine: the winner arrays are required
    assert lib.rtsdf_refine_tracked(C.byref(g), P(FAKE), 3, P(FAKE), 1, P(FAKE), bvh, P(FAKE), P(FAKE),
                                    C.byref(rp), P(FAKE), P(FAKE), P(FAKE), P(FAKE), None, P(FAKE), P(FAKE),
                                    refine_ws, None, None) == 1
    # samples: negative count, misaligned field
    assert lib.rtsdf_sample(C.byref(g), P(FAKE), P(FAKE), -1, P(FAKE), None) == 1
    assert lib.rtsdf_sample(C.byref(g), P(FAKE + 4), P(FAKE), 4, P(FAKE), None) == 1
    assert lib.rtsdf_sample(C.byref(g), P(FAKE), None, 0, None, None) == 0   # nothing to do

    def bwd(sp, ws_bytes, M=4, Pn=4, win=P(FAKE)):
        return lib.rtsdf_backward(C.byref(g), P(FAKE), 3, P(FAKE), 1, P(FAKE), P(FAKE), P(FAKE), P(FAKE), win,
                                  P(FAKE), C.byref(rp), P(FAKE), P(FAKE), M, P(FAKE), P(FAKE), P(FAKE), Pn,
                                  C.byref(sp), P(FAKE), P(FAKE), P(FAKE), P(FAKE), ws_bytes, None)

    long_march = ShadowParams((C.c_float * 3)(0, 1, 0), 8.0, 513, 1.0)
    assert bwd(long_march, ws) == 1
    sp = ShadowParams((C.c_float * 3)(0, 1, 0), 8.0, 512, 1.0)
    assert bwd(sp, ws - 1) == 2
    assert bwd(sp, ws, win=None) == 1
    assert bwd(sp, ws, M=-1) == 1
    assert bwd(ShadowParams((C.c_float * 3)(0, 0, 0), 8.0, 64, 1.0), ws) == 1


def test_product_path_has_no_cpu_fallback():
    """The binding raises when the compiled library is absent instead of computing
    anything itself, and nothing in the package imports the oracle."""
    import paper_2210_06160_gb300 as pkg
    pkg_dir = os.path.dirname(pkg.__file__)
    for fn in os.listdir(pkg_dir):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg_dir, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
    src = open(os.path.join(pkg_dir, "rtsdf.py")).read()
    assert "raise RtsdfError" in src


def _batch_scene(nx, ny, nz, V=10, T=4, steps=(8, 4, 2, 1)):
    from paper_2210_06160_gb300 import scenes
    from paper_2210_06160_gb300.rtsdf import make_batch_scene
    g = scenes.Grid(nx, ny, nz, (0.0, 0.0, 0.0), 0.1)
    return make_batch_scene(g, V, T, steps, scenes.RefineParams())


def test_batch_plan_layout_without_gpu(lib):
    from paper_2210_06160_gb300.rtsdf import BatchBuffers, BatchLayout, BatchScene, BatchTuning
    P = C.c_void_p
    descs = [_batch_scene(32, 32, 32, 100, 50), _batch_scene(17, 9, 33, 7, 0, (16, 8, 4, 2, 1)),
             _batch_scene(5, 5, 5, 3, 1, ())]
    arr = (BatchScene * 3)(*descs)
    plan = P()
    assert lib.rtsdf_batch_plan_create(arr, 3, C.byref(plan)) == 0 and plan.value
    try:
        nvox = lib.rtsdf_batch_voxels(plan)
        lays = []
        for i in range(3):
            L = BatchLayout()
            assert lib.rtsdf_batch_layout_of(plan, i, C.byref(L)) == 0
            lays.append(L)
        assert lib.rtsdf_batch_layout_of(plan, 3, C.byref(BatchLayout())) == 1
        assert [L.voxel_offset for L in lays] == [0, 32768, 32768 + 5056]          # multiples of 64
        assert nvox == 32768 + 5056 + 128
        assert [L.vertex_offset for L in lays] == [0, 100, 107]
        assert [L.triangle_offset for L in lays] == [0, 50, 50]
        assert all(L.bvh_offset % 256 == 0 for L in lays) and lays[1].bvh_offset > lays[0].bvh_offset
        assert [L.flooded_in_b for L in lays] == [0, 1, 0]                        # nsteps parity
        assert lib.rtsdf_batch_bvh_bytes(plan) >= lib.rtsdf_bvh_bytes(50) + lib.rtsdf_bvh_bytes(1)
        ws = lib.rtsdf_batch_workspace(plan)
        assert ws >= 8 * nvox
        t = BatchTuning()
        assert lib.rtsdf_batch_get_tuning(plan, C.byref(t)) == 0 and (t.brick_x, t.brick_y, t.brick_z) == (4, 4, 4)
        for bad in (BatchTuning(4, 4, 2, 2, 1), BatchTuning(8, 4, 2, 3, 1), BatchTuning(16, 2, 2, 2, 7)):
            assert lib.rtsdf_batch_set_tuning(plan, C.byref(bad)) == 1
        assert lib.rtsdf_batch_set_tuning(plan, C.byref(BatchTuning(16, 2, 2, 4, 0))) == 0
        # argument errors are found before anything is enqueued
        B = BatchBuffers(FAKE, FAKE, FAKE, FAKE + 4096, FAKE, FAKE, lib.rtsdf_batch_bvh_bytes(plan), FAKE, FAKE,
                         FAKE, FAKE, FAKE, ws - 1)
        assert lib.rtsdf_batch_rebuild(plan, C.byref(B), 0, 0, None, None) == 2
        B.ws_bytes = ws
        B.buf_b = FAKE
        assert lib.rtsdf_batch_rebuild(plan, C.byref(B), 0, 0, None, None) == 1    # aliased JFA buffers
        B.buf_b = FAKE + 4096
        B.sdf = FAKE + 4
        assert lib.rtsdf_batch_rebuild(plan, C.byref(B), 0, 0, None, None) == 1    # misaligned grid
        assert lib.rtsdf_batch_autotune(plan, C.byref(B), 0, None, None) == 1
    finally:
        lib.rtsdf_batch_plan_destroy(plan)


def test_batch_plan_validation(lib):
    from paper_2210_06160_gb300.rtsdf import BatchScene
    P = C.c_void_p
    plan = P()
    ok = _batch_scene(8, 8, 8)
    assert lib.rtsdf_batch_plan_create((BatchScene * 1)(ok), 0, C.byref(plan)) == 1
    assert lib.rtsdf_batch_plan_create((BatchScene * 65)(*([ok] * 65)), 65, C.byref(plan)) == 1
    for bad in (_batch_scene(0, 8, 8), _batch_scene(8, 1024, 8), _batch_scene(8, 8, 8, steps=(0,)),
                _batch_scene(8, 8, 8, V=-1)):
        assert lib.rtsdf_batch_plan_create((BatchScene * 2)(ok, bad), 2, C.byref(plan)) == 1
    b = _batch_scene(8, 8, 8)
    b.nsteps = 17
    assert lib.rtsdf_batch_plan_create((BatchScene * 1)(b), 1, C.byref(plan)) == 1
    lib.rtsdf_batch_plan_destroy(None)


def test_texture_entry_validation(lib):
    from paper_2210_06160_gb300.rtsdf import ShadowParams
    P = C.c_void_p
    h = C.c_void_p()
    assert lib.rtsdf_texture_create(C.byref(_grid(0, 8, 8)), C.byref(h)) == 1 and not h.value
    assert lib.rtsdf_texture_create(C.byref(_grid()), None) == 1
    sp = ShadowParams((C.c_float * 3)(0, 1, 0), 8.0, 10, 1.0)
    assert lib.rtsdf_shadow_tex(None, P(FAKE), P(FAKE), 4, C.byref(sp), P(FAKE), None) == 1
    assert lib.rtsdf_texture_upload(None, P(FAKE), None) == 1
    lib.rtsdf_texture_destroy(None)


def _c_layout(tmp_path, ctype: str, fields) -> list[int]:
    """sizeof and field offsets of a struct of include/rtsdf.h, as a C compiler lays it out."""
    import subprocess
    src = tmp_path / f"layout_{ctype}.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rtsdf.h"\nint main(void) {\n'
                   f'    printf("%zu", sizeof({ctype}));\n'
                   + "".join(f'    printf(" %zu", offsetof({ctype}, {f}));\n' for f in fields)
                   + "    return 0;\n}\n")
    exe = tmp_path / f"layout_{ctype}"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                           str(src), "-o", str(exe)])
    return [int(v) for v in subprocess.check_output([str(exe)]).split()]


def test_counters_layout_matches_the_header(tmp_path):
    """The binding's rtsdf_counters mirrors the C struct: size and field offsets as a
    C compiler lays out include/rtsdf.h."""
    from paper_2210_06160_gb300 import rtsdf
    fields = [f for f, _ in rtsdf.Counters._fields_]
    got = _c_layout(tmp_path, "rtsdf_counters", fields)
    want = [C.sizeof(rtsdf.Counters)] + [getattr(rtsdf.Counters, f).offset for f in fields]
    assert got == want
    assert got[0] == 64 and rtsdf.COUNTER_WORDS == 16


@pytest.mark.parametrize("name", ["ShadowParams", "RefineParams"])
def test_parameter_structs_match_the_header(tmp_path, name):
    """The binding's parameter structs mirror rtsdf_shadow_params and
    rtsdf_refine_params field by field."""
    from paper_2210_06160_gb300 import rtsdf
    cls = getattr(rtsdf, name)
    ctype = {"ShadowParams": "rtsdf_shadow_params", "RefineParams": "rtsdf_refine_params"}[name]
    fields = [f for f, _ in cls._fields_]
    got = _c_layout(tmp_path, ctype, fields)
    assert got == [C.sizeof(cls)] + [getattr(cls, f).offset for f in fields]
