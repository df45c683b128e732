"""Writes the oracle regression fixtures in this folder.

Calls only the FP64 oracle (and the seeded scene generators).  The values
pin the oracle against unintended drift; what pins it against the paper is
tests/test_oracle_pins.py.  Re-run only when a change to the oracle's
arithmetic is justified by a passage of the paper:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2603_00413_gb300 import scenes as S  # noqa: E402

PIXELS = [(32, 32), (20, 40), (10, 31), (50, 12), (0, 0), (45, 45)]


def icosphere_fixture():
    """The one-icosphere workload: subdivision 3, IoR 1.5, no absorption,
    64x64 at pixel centres, depth 4, 64x32 SH environment (seed 0)."""
    sc = S.glass_icosphere_scene()
    r = O.render(sc.V, sc.F, sc.ior, sc.sigma, sc.env, sc.cams[0], sc.max_depth)
    img = r["img"]
    return {
        "workload": "glass icosphere s3, ior 1.5, sigma 0, 64x64, spp 1, depth 4, env 64x32 SH seed 0",
        "counters": r["counters"],
        "image_sum": img.sum(axis=(0, 1)).tolist(),
        "pixels": {f"{y},{x}": img[y, x].tolist() for (y, x) in PIXELS},
    }


def absorbing_fixture():
    """Same sphere, sigma = (0.5, 1.0, 1.5), IoR 1.45, 32x32, depth 6."""
    sc = S.glass_icosphere_scene(width=32, height=32)
    sigma = np.array([0.5, 1.0, 1.5], np.float32)
    ior = float(np.float32(1.45))
    r = O.render(sc.V, sc.F, ior, sigma, sc.env, sc.cams[0], 6)
    img = r["img"]
    return {
        "workload": "glass icosphere s3, ior 1.45, sigma (0.5,1,1.5), 32x32, spp 1, depth 6",
        "counters": r["counters"],
        "image_sum": img.sum(axis=(0, 1)).tolist(),
        "pixels": {f"{y},{x}": img[y, x].tolist() for (y, x) in [(16, 16), (8, 20), (24, 10)]},
    }


def textured_fixture():
    """Same sphere, sigma = (0.2, 0.1, 0.3), IoR 1.5, 24x24, depth 5, with a
    dense 5x6x4 absorption grid (seed 9) and, separately, a three-level hash
    texture (2^8 entries per level, 3 to 12 nodes per axis, seed 9), both over
    [-1.25, 1.25]^3 (Eq. 11 with a spatially varying rate)."""
    sc = S.glass_icosphere_scene(width=24, height=24)
    sigma = np.array([0.2, 0.1, 0.3], np.float32)
    lo, hi = (-1.25, -1.25, -1.25), (1.25, 1.25, 1.25)
    grid = S.random_absorption_grid((5, 6, 4), lo, hi, seed=9, scale=1.0)
    tex = S.random_hash_texture(3, 8, 3, 12, lo, hi, seed=9, scale=1.0)
    out = {"workload": "glass icosphere s3, ior 1.5, sigma (0.2,0.1,0.3), 24x24, spp 1, depth 5; "
                       "grid 5x6x4 seed 9 / hash texture 3 levels x 2^8, 3..12 nodes, seed 9"}
    for name, med in (("grid", grid), ("hash_texture", tex)):
        r = O.render(sc.V, sc.F, 1.5, sigma, sc.env, sc.cams[0], 5, medium=med)
        img = r["img"]
        out[name] = {"counters": r["counters"], "image_sum": img.sum(axis=(0, 1)).tolist(),
                     "pixels": {f"{y},{x}": img[y, x].tolist() for (y, x) in [(12, 12), (6, 15), (18, 8)]}}
    return out


if __name__ == "__main__":
    out = {"icosphere": icosphere_fixture(), "icosphere_absorbing": absorbing_fixture(),
           "icosphere_textured": textured_fixture()}
    with open(os.path.join(HERE, "oracle_icosphere.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("wrote", os.path.join(HERE, "oracle_icosphere.json"))
