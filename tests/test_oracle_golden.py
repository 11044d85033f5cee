"""Regression of the oracle against its committed summary and the paper's printed
parameters (tests/golden/)."""
import json
import os

from paper_2210_06160_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_committed_summary(orc):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    want = json.load(open(os.path.join(GOLDEN, "tiny_icosphere_oracle.json")))
    got = mg.summary()
    for k, v in want.items():
        if isinstance(v, float):
            assert abs(got[k] - v) < 1e-6, k
        else:
            assert got[k] == v, k


def test_workloads_use_the_paper_parameters():
    p = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    room = scenes.scene_room.__defaults__  # (seed, nx, ny, nz, ...)
    assert list(room[1:4]) == p["fine_sdf_texture_size"]["value"]
    sc = scenes.scene_tiny()
    # max raymarch step 0.05 scene units, in voxels of the grid
    assert abs(sc.shadow.max_step_vox * sc.grid.h - p["max_raymarch_step"]["value"]) < 1e-12
    assert sc.jfa_steps[0] == int(64 * p["jfa_first_offset_of_n"]["value"])
