"""Helpers shared by the GPU parity tests: tolerances, ambiguity filters and
seeded complexes.  Expected values always come from the oracle."""
import math

import numpy as np

import oracle
from paper_2303_09916_gb300 import synth

RADIUS = [1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0, 1.8]
HYD = [1, 0, 0, 0, 0, 0, 0, 0, 0]
DON = [0, 0, 0, 1, 0, 0, 1, 0, 1]
ACC = [0, 0, 0, 0, 1, 1, 1, 0, 1]

# Tolerances of the FP32 device path against the FP64 oracle (relative 1e-4 of
# the scale of the summed terms, since FP32 sums carry error relative to their
# terms, not to a result that may cancel):
#   conformation energy   |dE| <= 1e-4 * max(sum_i |e_i|, 1)  (per-atom grid and per-pair terms)
#   conformation gradient ||dg||_inf <= 1e-4 * max(||g||_inf, 1e-2)
#   map vertex            |dE| <= 1e-4 * max(sum_j |f_j|, 1), |dg| <= 1e-4 * max(sum_j |f'_j|, 1e-2)
E_REL = 1e-4
G_REL = 1e-4
# FP32 gradient error of the GPU path relative to the largest component, the size
# of the gradient probe in the chain tests' divergence explanations; the score
# tests assert that the measured errors stay within it (measured on Eq. 4 maps:
# 2e-6 - 1.1e-5).
G_FP32 = 2e-5


def kinks(ti, tj):
    """Surface distances where the pair term's slope jumps, plus the cutoff (as r)."""
    d = []
    if HYD[ti] and HYD[tj]:
        d += [0.5, 1.5]
    if (DON[ti] and ACC[tj]) or (ACC[ti] and DON[tj]):
        d += [-0.7, 0.0]
    return d


def pair_is_ambiguous(ti, tj, r, eps):
    if abs(r - 8.0) < eps:
        return True
    dd = r - (RADIUS[ti] + RADIUS[tj])
    return any(abs(dd - k) < eps for k in kinks(ti, tj))


class Complex:
    def __init__(self, n_rec, box, n_lig, T, seed, spacing=0.375):
        self.rec = synth.receptor(n_rec, seed)
        self.lig = synth.ligand(n_lig, T, seed, center=self.rec.pocket_center)
        self.olig = oracle.Ligand(self.lig.xyz.astype(np.float64), self.lig.xs_type, self.lig.bonds,
                                  self.lig.rotatable)
        self.center = self.rec.pocket_center.astype(np.float64)
        self.size = np.array([box] * 3, dtype=np.float64)
        self.spacing = spacing
        self.rec_xyz64 = self.rec.xyz.astype(np.float64)
        self._grid = None

    @property
    def T(self):
        return self.olig.T

    def oracle_grid(self):
        if self._grid is None:
            self._grid = oracle.grid_build(self.rec_xyz64, self.rec.xs_type, self.center, self.size, self.spacing)
        return self._grid

    def box_lo(self):
        return self.center - self.size / 2

    def random_confs(self, n, seed, spread=2.0):
        rng = np.random.default_rng(seed)
        out = []
        for _ in range(n):
            c = self.olig.identity_conf()
            c[:3] = self.center + rng.uniform(-spread, spread, 3)
            q = rng.normal(size=4)
            c[3:7] = q / np.linalg.norm(q)
            c[7:] = rng.uniform(-math.pi, math.pi, self.T)
            out.append(c)
        return np.array(out)

    def abs_terms(self, grid, mode, conf):
        """sum_i |e_i| over per-atom grid terms and per-pair intra terms (oracle)."""
        x = self.olig.coords(conf)
        s = 0.0
        for t in set(self.lig.xs_type.tolist()):
            idx = np.nonzero(self.lig.xs_type == t)[0]
            e, _ = oracle.interpolate(grid, mode, int(t), x[idx])
            s += np.abs(e).sum()
        for i, j in self.olig.pairs():
            r = float(np.linalg.norm(x[i] - x[j]))
            s += abs(oracle.pair(int(self.lig.xs_type[i]), int(self.lig.xs_type[j]), r)[0])
        return s

    def conf_is_ambiguous(self, grid, mode, conf, eps=2e-4):
        """True where FP32 and FP64 may take different branches: an intra pair near a kink
        or the cutoff, an atom near the grid's edge (wall), or near a cell face (Eq. 3)."""
        x = self.olig.coords(conf)
        t = self.lig.xs_type
        for i, j in self.olig.pairs():
            if pair_is_ambiguous(int(t[i]), int(t[j]), float(np.linalg.norm(x[i] - x[j])), eps):
                return True
        u = (x - grid.origin) / grid.h
        hi = grid.n - 1
        if np.any(np.abs(u) < eps / grid.h) or np.any(np.abs(u - hi) < eps / grid.h):
            return True
        if mode == 1:
            inside = (u > 0) & (u < hi)
            frac = u - np.floor(u)
            if np.any(inside & ((frac < eps / grid.h) | (frac > 1 - eps / grid.h))):
                return True
        return False


def vertex_ambiguity(rec_xyz, rec_type, grid_origin, n, h, eps=5e-5):
    """Boolean (8, nz, ny, nx): vertex/type pairs where some receptor atom sits
    within eps of the cutoff or of a slope kink, so FP32 and FP64 may branch
    differently there."""
    from scipy.spatial import cKDTree

    nx, ny, nz = n
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([grid_origin[0] + h * xs, grid_origin[1] + h * ys, grid_origin[2] + h * zs], -1).reshape(-1, 3)
    tree = cKDTree(rec_xyz)
    amb = np.zeros((8, len(pts)), dtype=bool)
    nbrs = tree.query_ball_point(pts, 8.0 + 1e-3)
    for v, js in enumerate(nbrs):
        if not js:
            continue
        js = np.array(js)
        r = np.linalg.norm(rec_xyz[js] - pts[v], axis=1)
        near_cut = np.any(np.abs(r - 8.0) < eps)
        for t in range(8):
            if near_cut:
                amb[t, v] = True
                continue
            for j, rj in zip(js, r):
                tj = int(rec_type[j])
                dd = rj - (RADIUS[t] + RADIUS[tj])
                if any(abs(dd - k) < eps for k in kinks(t, tj)):
                    amb[t, v] = True
                    break
    return amb.reshape(8, nz, ny, nx)


def vertex_scales(cx, og):
    """(8, nz, ny, nx, 2): sum_j |f| and sum_j |df/dr| at every vertex (oracle)."""
    nx, ny, nz = og.n
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([og.origin[0] + og.h * xs, og.origin[1] + og.h * ys, og.origin[2] + og.h * zs],
                   -1).reshape(-1, 3)
    out = np.zeros((8, len(pts), 2))
    for t in range(8):
        out[t] = oracle.receptor_field_abs(cx.rec_xyz64, cx.rec.xs_type, t, pts)
    return out.reshape(8, nz, ny, nx, 2)
