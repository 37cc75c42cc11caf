"""Writes oracle_regression.json: FP64 oracle values on a small seeded complex.

The file pins the oracle against unintended changes of its arithmetic (it is
not a pin of the oracle against the paper: those are the closed forms,
invariants and brute-force checks in tests/test_oracle_*.py).  It calls only
oracle/ and the seeded input generator; nothing comes from the CUDA path.
Regenerate it only for an intended change of the oracle, and name the passage
of the paper (or the reading of it) that justifies the change in the commit.

Quantities (non-chaotic: no Monte Carlo or optimiser trajectories, which may
separate across machines by one ulp of a libm call):
  pair terms f(t_i, t_j, r)       Vina-form score (Sec. 2; constants: the Vina reading)
  grid vertices                   Eq. 1 maps and the gradient maps of Eq. 4
  score + gradient at poses       Eq. 2 with Eq. 4 (mode 0) and Eq. 3 (mode 1), kinematics and chain rule
  exact gridless score at poses   the plain definition the rescoring uses (Fig. 4 postprocess)
  Philox4x32-10 blocks            Salmon et al. (SC'11)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2303_09916_gb300 import synth  # noqa: E402


def compute():
    rec = synth.receptor(300, 17)
    s = synth.ligand(9, 3, 17, center=rec.pocket_center)
    lig = oracle.Ligand(s.xyz.astype(np.float64), s.xs_type, s.bonds, s.rotatable)
    rec_xyz = rec.xyz.astype(np.float64)
    size = np.array([8.0, 8.0, 8.0])
    grid = oracle.grid_build(rec_xyz, rec.xs_type, rec.pocket_center, size, 0.5)
    out = {}
    out["pair"] = [[ti, tj, r, *oracle.pair(ti, tj, r)] for ti, tj, r in
                   [(0, 0, 3.1), (0, 5, 4.4), (3, 5, 2.9), (6, 4, 3.3), (7, 2, 6.5), (1, 6, 7.9)]]
    m = grid.maps  # (8, nz, ny, nx, 4)
    idx = [(t, z, y, x) for t, z, y, x in [(0, 0, 0, 0), (1, 3, 5, 7), (2, 8, 8, 8), (3, 15, 2, 9), (4, 5, 15, 0),
                                            (5, 10, 11, 12), (6, 15, 15, 15), (7, 7, 1, 14)]]
    out["vertices"] = [[*k, *m[k].tolist()] for k in idx]
    rng = np.random.default_rng(5)
    poses = []
    for _ in range(4):
        c = lig.identity_conf()
        c[:3] = rec.pocket_center + rng.uniform(-1.5, 1.5, 3)
        q = rng.normal(size=4)
        c[3:7] = q / np.linalg.norm(q)
        c[7:] = rng.uniform(-3, 3, lig.T)
        poses.append(c)
    out["poses"] = [c.tolist() for c in poses]
    out["score_grid"] = []
    for mode in (0, 1):
        for c in poses:
            terms, g = lig.score_grid(grid, mode, c)
            out["score_grid"].append([mode, *terms.tolist(), *g.tolist()])
    out["score_exact"] = [lig.score_exact(rec_xyz, rec.xs_type, c)[0].tolist() for c in poses[:2]]
    out["coords"] = lig.coords(poses[0]).tolist()
    out["philox"] = [oracle.philox([c, 3, 1, 0], [7, 0]).tolist() for c in range(3)]
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(compute(), f, indent=1)
    print("written")
