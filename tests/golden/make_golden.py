"""Writes `tiny_icosphere_oracle.json`: a regression summary of the oracle on the
64^3 icosphere workload.  Calls only the CPU oracle (`oracle/`) and the seeded
scene generator; rerun it only when a change to the oracle's arithmetic is
justified by the paper (the commit names the passage).

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2210_06160_gb300 import scenes  # noqa: E402


def summary():
    sc = scenes.scene_tiny(shadow_res=64)
    r = oracle.rebuild(sc)
    m = r["mask"].astype(bool)
    vis = oracle.shadow(sc.grid, r["sdf"], sc.recv_pos, sc.recv_nrm, sc.shadow)

    def h(a):
        return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]

    return {
        "workload": "icosphere subdiv 3 (1280 tris), 64^3, 16 rays, key 0; 64x64 shadow",
        "seeds": int((r["seed"] >= 0).sum()),
        "masked": int(m.sum()),
        "front_total": int(r["front"][m].sum()),
        "back_total": int(r["back"][m].sum()),
        "negative_voxels": int((r["sdf"] < 0).sum()),
        "sha_seed": h(r["seed"]),
        "sha_nearest": h(r["nearest"]),
        "sha_dist_masked": h(r["dist_bits"][m]),
        "sha_sdf": h(r["sdf"]),
        "vis_mean": float(np.mean(vis)),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_icosphere_oracle.json")
    with open(out, "w") as f:
        json.dump(summary(), f, indent=1)
    print(open(out).read())
