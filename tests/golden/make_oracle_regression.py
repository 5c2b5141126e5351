"""Writes oracle_regression_tiny.json: the FP64 oracle's outputs on two small
seeded scenes, so that any later change to the oracle's arithmetic shows up
in tests/test_oracle_pins.py.  Calls only oracle/ (and the seeded scene
generators); run from the repository root:

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2603_09277_gb300 import scenes  # noqa: E402

CASES = [  # (seed, sh_degree, tile)
    (0, 0, 16),
    (1, 3, 8),
]


def case(seed, deg, tile):
    scene, cams, targets, prm = scenes.tiny_scene(8, seed=seed, width=40, height=36, sh_degree=deg)
    prm["tile"] = tile
    L, views, grads, _ = oracle.step(scene, cams, targets, prm, scenes.GAMMA)
    f = views[0]["fwd"]
    K = (deg + 1) ** 2
    return {
        "seed": seed, "sh_degree": deg, "tile": tile, "loss": L,
        "image_sum": float(np.sum(f["image"])), "final_T_sum": float(np.sum(f["final_T"])),
        "entropy_sum": float(np.sum(f["entropy"])), "last_sum": int(np.sum(f["last"])),
        "brightest_pixel": [int(i) for i in np.unravel_index(np.argmax(f["image"].sum(-1)),
                                                             f["image"].shape[:2])],
        "brightest_rgb": [float(x) for x in
                          f["image"].reshape(-1, 3)[np.argmax(f["image"].sum(-1))]],
        "grads": {k: [float(x) for x in np.asarray(grads[k])[:, :K].ravel()] if k == "sh"
                  else [float(x) for x in np.asarray(grads[k]).ravel()]
                  for k in ("means", "log_scales", "quats", "opacity_logits", "sh")},
    }


if __name__ == "__main__":
    out = {"note": "written by tests/golden/make_oracle_regression.py from the FP64 oracle",
           "cases": [case(*c) for c in CASES]}
    with open(os.path.join(HERE, "oracle_regression_tiny.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", len(out["cases"]), "cases")
