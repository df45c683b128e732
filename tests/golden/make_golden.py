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


if __name__ == "__main__":
    out = {"icosphere": icosphere_fixture(), "icosphere_absorbing": absorbing_fixture()}
    with open(os.path.join(HERE, "oracle_icosphere.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("wrote", os.path.join(HERE, "oracle_icosphere.json"))
