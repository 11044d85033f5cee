"""rtsdf_build_bvh_noalloc: the BVH build for hosts that cannot allocate device
memory for the library (an engine's memory manager owns the GPU and forbids
cudaMalloc in its frame loop).  It must produce the same BVH as rtsdf_build_bvh
with a caller workspace, on consecutive calls that reuse its fixed internal
scratch.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2210_06160_gb300 import rtsdf as rt
from paper_2210_06160_gb300 import scenes

pytestmark = pytest.mark.gpu


def _workspace_build(sc, verts, tris):
    g = rt.make_grid(sc.grid)
    T = len(sc.tris)
    bvh = torch.zeros(rt.rtsdf_bvh_bytes(T), dtype=torch.uint8, device="cuda")
    ws = torch.empty(rt.rtsdf_bvh_workspace(T), dtype=torch.uint8, device="cuda")
    rt.rtsdf_build_bvh(verts, tris, g, bvh, ws)
    return bvh


def _noalloc_build(sc, verts, tris):
    g = rt.make_grid(sc.grid)
    bvh = torch.zeros(rt.rtsdf_bvh_bytes(len(sc.tris)), dtype=torch.uint8, device="cuda")
    rt.rtsdf_build_bvh_noalloc(verts, tris, g, bvh)
    return bvh


def test_noalloc_bvh_equals_workspace_bvh_on_consecutive_calls():
    assert torch.cuda.is_available(), "GPU test"
    from paper_2210_06160_gb300 import build
    build.build()
    # two calls in a row on different meshes: the second reuses the scratch the
    # first left behind (largest mesh first, then a smaller one)
    for sc in (scenes.scene_room(), scenes.scene_tiny()):
        verts = torch.from_numpy(sc.verts).cuda()
        tris = torch.from_numpy(sc.tris).cuda()
        want = _workspace_build(sc, verts, tris)
        got = _noalloc_build(sc, verts, tris)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want.cpu().numpy())
        # the header's leaf count is the mesh's triangle count (all valid)
        n_leaves = int(got[:4].cpu().numpy().view(np.int32)[0])
        assert n_leaves == len(sc.tris)


def test_noalloc_bvh_rejects_meshes_above_its_limit():
    g = rt.make_grid(scenes.scene_tiny().grid)
    T = 131072 + 1
    P = C.c_void_p
    fake = 0x7F0000000000  # never dereferenced: the size check comes first
    st = rt.lib().rtsdf_build_bvh_noalloc(P(fake), 3, P(fake), T, C.byref(g), P(fake), 1 << 40, None, None)
    assert st == 2  # RTSDF_ENOMEM
