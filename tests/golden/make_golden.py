"""Writes tests/golden/tiny64_oracle_samples.json from the FP64 oracle only.

Run from the repository root: python tests/golden/make_golden.py
The samples pin the oracle's tiny 64x64 workload against later drift; no value in
the file comes from the CUDA path.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2405_05446_gb300 import scenes as S  # noqa: E402


def main():
    sc, cam, mean, _ = S.workload("tiny64")
    img, maps, amb = O.render_view(sc, cam, mean)
    rng = np.random.default_rng(123)
    nz = np.argwhere(np.abs(maps[:, 0]) > 0)
    picks = nz[rng.choice(len(nz), 24, replace=False)]
    samples = [{"c": int(c), "i": int(i), "j": int(j), "gx": float(maps[c, 0, i, j]),
                "gy": float(maps[c, 1, i, j]), "img": float(img[c, i, j])} for c, i, j in picks]
    samples += [{"c": c, "i": i, "j": j, "gx": float(maps[c, 0, i, j]),
                 "gy": float(maps[c, 1, i, j]), "img": float(img[c, i, j])}
                for c, i, j in [(0, 0, 0), (2, 63, 63), (1, 31, 32)]]
    out = {"workload": "tiny64: 1000 Gaussians, 64x64, seed 0, mean 0.5",
           "written_by": "tests/golden/make_golden.py (oracle only)",
           "ambiguous": int(amb.sum()), "samples": samples}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny64_oracle_samples.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
