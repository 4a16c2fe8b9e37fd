"""Writes tests/golden/oracle_lapl3d_64.json: the FP64 oracle's result on the
benchmark workload (3D 7-point Laplacian 64^3, L = 10, eps = 1e-2, b seed 1),
reduced to what a full-size GPU test can compare: PCG iteration count,
true relative residual, size_Top, per-step size totals after sparsification,
||x|| and 256 sampled entries of x (fixed seeded positions).

Calls only oracle/ and the seeded input generators.  About 80 s on one core.
Run from the repository root:  python tests/golden/make_oracle_lapl3d_64.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import spand_oracle as O  # noqa: E402
from paper_1901_02971_gb300 import inputs as I  # noqa: E402

GRID, LEVELS, EPS, SEED = 64, 10, 1e-2, 1


def main():
    p = I.laplacian_3d(GRID)
    b = I.rhs(p.n, SEED)
    res = O.solve(p, b, LEVELS, EPS)
    idx = np.sort(I.rng(12345).choice(p.n, size=256, replace=False))
    out = {
        "workload": f"lapl3d_{GRID}^3_7pt_L{LEVELS}_eps{EPS}",
        "seed_b": SEED,
        "iters": int(res.iters),
        "relres": float(res.relres),
        "size_top": int(res.factor.size_top),
        "sizes_after_per_step": [int(s.sum()) for s in res.factor.sizes_after],
        "x_norm": float(np.linalg.norm(res.x)),
        "sample_idx": idx.tolist(),
        "sample_x": [float(v) for v in res.x[idx]],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_lapl3d_64.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out["iters"], out["relres"], out["size_top"], out["sizes_after_per_step"])


if __name__ == "__main__":
    main()
