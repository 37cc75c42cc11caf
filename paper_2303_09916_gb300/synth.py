"""Seeded synthetic inputs shaped like DSDP's docking workloads.

This module holds no arithmetic of the docking method: it only draws receptor
atoms, ligand trees and job shapes.  Both the CUDA path and the FP64 oracle take
their inputs from here; neither one's results ever feed back into it.

The paper docks real complexes (its scPDB-derived 995-complex set, PDBBind
time-split and DUD-E, Sec. 2 "Data Set preparation"); none is available here, so
these seeded stand-ins reproduce their shapes instead:

* receptor: heavy atoms at protein density 0.05 / A^3 with minimum separation
  2.8 A, built as a jittered FCC lattice (lattice constant (4 / 0.05)^(1/3) =
  4.309 A, nearest neighbours 3.047 A, jitter uniform in a 0.12 A ball) inside a
  sphere, minus a 6 A spherical pocket whose centre sits at 0.6 R; element mix
  C 62 % / N 17 % / O 19 % / S 2 %; C hydrophobic with p = 0.7; N donor 0.5 and
  acceptor 0.3 independently; O always acceptor, donor 0.3; S polar.
* ligand: random self-avoiding tree of heavy atoms, 1.5 A bonds, tetrahedral
  angles, dihedrals from {60, 180, 300} degrees, atoms three or more bonds apart
  at least 2.5 A apart, degree <= 3; T rotatable bonds drawn among non-terminal
  bonds (capped at their number); C hydrophobic when it has no N/O neighbour;
  N drawn among N_P / N_D / N_A; O as in the receptor.
* the docking box is centred on the pocket; the ligand's reference pose is
  centred there too.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# XS type codes used across the C ABI (include/dsdp.h): ligand map types 0..7,
# N_DA only on receptor atoms.
C_H, C_P, N_P, N_D, N_A, O_A, O_DA, S_P, N_DA = range(9)

DENSITY = 0.05
FCC_A = (4.0 / DENSITY) ** (1.0 / 3.0)
JITTER = 0.12
POCKET_RADIUS = 6.0


def _rng(seed: int, tag: str) -> np.random.Generator:
    key = (int(seed) * 0x9E3779B1 + sum(ord(c) << (8 * i) for i, c in enumerate(tag))) & ((1 << 63) - 1)
    return np.random.Generator(np.random.Philox(key))


def _ball(rng, n, radius):
    out = np.empty((0, 3))
    while len(out) < n:
        p = rng.uniform(-1, 1, size=(2 * n + 8, 3))
        p = p[(p * p).sum(1) <= 1.0]
        out = np.concatenate([out, p])
    return out[:n] * radius


@dataclass
class Receptor:
    xyz: np.ndarray          # (n, 3) float32
    xs_type: np.ndarray      # (n,) uint8
    pocket_center: np.ndarray  # (3,) float64


@dataclass
class Ligand:
    xyz: np.ndarray          # (n, 3) float32, reference pose
    xs_type: np.ndarray      # (n,) uint8
    bonds: np.ndarray        # (n_bonds, 2) int32
    rotatable: np.ndarray    # (n_bonds,) uint8
    n_torsions: int = 0

    @property
    def n_atoms(self):
        return len(self.xs_type)


@dataclass
class Box:
    center: np.ndarray
    size: np.ndarray
    spacing: float = 0.375


def receptor(n_atoms: int, seed: int = 0) -> Receptor:
    rng = _rng(seed, "RECP")
    pocket_vol_atoms = DENSITY * 4.0 / 3.0 * math.pi * POCKET_RADIUS ** 3
    R = ((n_atoms + pocket_vol_atoms) / (DENSITY * 4.0 / 3.0 * math.pi)) ** (1.0 / 3.0) + 1.0
    direction = rng.normal(size=3)
    direction /= np.linalg.norm(direction)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    while True:
        m = int(math.ceil((R + 2) / FCC_A)) + 1
        g = np.arange(-m, m + 1)
        cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        sites = (cells[:, None, :] + basis[None]).reshape(-1, 3) * FCC_A
        sites = sites + _ball(rng, len(sites), JITTER)
        pocket = 0.6 * R * direction
        keep = (np.linalg.norm(sites - pocket, axis=1) > POCKET_RADIUS)
        sites = sites[keep]
        r = np.linalg.norm(sites, axis=1)
        order = np.argsort(r, kind="stable")
        if len(order) >= n_atoms and r[order[n_atoms - 1]] <= R:
            sites = sites[order[:n_atoms]]
            break
        R += 1.0
    u = rng.uniform(size=n_atoms)
    element = np.where(u < 0.62, 0, np.where(u < 0.79, 1, np.where(u < 0.98, 2, 3)))
    types = np.empty(n_atoms, dtype=np.uint8)
    hyd = rng.uniform(size=n_atoms) < 0.7
    don = rng.uniform(size=n_atoms) < 0.5
    acc = rng.uniform(size=n_atoms) < 0.3
    odon = rng.uniform(size=n_atoms) < 0.3
    for i in range(n_atoms):
        e = element[i]
        if e == 0:
            types[i] = C_H if hyd[i] else C_P
        elif e == 1:
            types[i] = [N_P, N_A, N_D, N_DA][int(don[i]) * 2 + int(acc[i])]
        elif e == 2:
            types[i] = O_DA if odon[i] else O_A
        else:
            types[i] = S_P
    return Receptor(sites.astype(np.float32), types, pocket.astype(np.float64))


def _place(a, b, c, bond, angle, dihedral):
    """Atom d with |cd| = bond, angle(b, c, d) = angle, dihedral(a, b, c, d) = dihedral."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.stack([bc, np.cross(n, bc), n], axis=1)
    d2 = np.array([-bond * math.cos(angle), bond * math.sin(angle) * math.cos(dihedral),
                   bond * math.sin(angle) * math.sin(dihedral)])
    return c + m @ d2


def _perp(v, rng):
    w = rng.normal(size=3)
    w -= w.dot(v) * v
    return w / np.linalg.norm(w)


def ligand(n_atoms: int, n_torsions: int, seed: int = 0, center=None) -> Ligand:
    rng = _rng(seed, "LIGD")
    tet = math.radians(109.47)
    bond = 1.5
    for _attempt in range(1000):
        xyz = [np.zeros(3)]
        nbr = [[]]
        ok = True
        while len(xyz) < n_atoms and ok:
            placed = False
            for _try in range(200):
                cand = [i for i in range(len(xyz)) if len(nbr[i]) < 3]
                a = int(rng.choice(cand))
                A = xyz[a]
                if not nbr[a]:
                    v = rng.normal(size=3)
                    p = A + bond * v / np.linalg.norm(v)
                elif len(nbr[a]) == 1:
                    b = nbr[a][0]
                    B = xyz[b]
                    others = [c for c in nbr[b] if c != a]
                    if others:
                        C = xyz[others[0]]
                    else:
                        u = (A - B) / np.linalg.norm(A - B)
                        C = B + _perp(u, rng)
                    dih = math.radians(float(rng.choice([60.0, 180.0, 300.0])))
                    p = _place(C, B, A, bond, tet, dih)
                else:
                    u1 = (xyz[nbr[a][0]] - A) / bond
                    u2 = (xyz[nbr[a][1]] - A) / bond
                    bis = -(u1 + u2)
                    bis /= np.linalg.norm(bis)
                    nn = np.cross(u1, u2)
                    nn /= np.linalg.norm(nn)
                    half = math.radians(109.47 / 2.0)
                    sign = 1.0 if rng.uniform() < 0.5 else -1.0
                    p = A + bond * (math.cos(half) * bis + sign * math.sin(half) * nn)
                # topological distance from the new atom (bonded to a)
                dist = {a: 1}
                frontier = [a]
                while frontier:
                    nxt = []
                    for x in frontier:
                        for y in nbr[x]:
                            if y not in dist:
                                dist[y] = dist[x] + 1
                                nxt.append(y)
                    frontier = nxt
                clash = False
                for j in range(len(xyz)):
                    if dist.get(j, 99) >= 3 and np.linalg.norm(xyz[j] - p) < 2.5:
                        clash = True
                        break
                if clash:
                    continue
                xyz.append(p)
                nbr.append([a])
                nbr[a].append(len(xyz) - 1)
                placed = True
                break
            if not placed:
                ok = False
        if ok:
            break
    else:
        raise RuntimeError("ligand generator failed")
    xyz = np.array(xyz)
    bonds = np.array([(i, j) for i in range(n_atoms) for j in nbr[i] if i < j], dtype=np.int32).reshape(-1, 2)
    deg = np.array([len(x) for x in nbr])
    nonterminal = [k for k, (i, j) in enumerate(bonds) if deg[i] >= 2 and deg[j] >= 2]
    T = min(n_torsions, len(nonterminal))
    rot = np.zeros(len(bonds), dtype=np.uint8)
    if T > 0:
        rot[rng.choice(nonterminal, size=T, replace=False)] = 1
    # elements then XS types
    u = rng.uniform(size=n_atoms)
    element = np.where(u < 0.62, 0, np.where(u < 0.79, 1, np.where(u < 0.98, 2, 3)))
    un = rng.uniform(size=n_atoms)
    uo = rng.uniform(size=n_atoms)
    types = np.empty(n_atoms, dtype=np.uint8)
    for i in range(n_atoms):
        e = element[i]
        if e == 0:
            polar_nbr = any(element[j] in (1, 2) for j in nbr[i])
            types[i] = C_P if polar_nbr else C_H
        elif e == 1:
            types[i] = N_P if un[i] < 0.35 else (N_D if un[i] < 0.70 else N_A)
        elif e == 2:
            types[i] = O_DA if uo[i] < 0.3 else O_A
        else:
            types[i] = S_P
    xyz -= xyz.mean(0)
    if center is not None:
        xyz += np.asarray(center, dtype=np.float64)
    return Ligand(xyz.astype(np.float32), types, bonds, rot, int(T))


def site_points(rec: Receptor, n_points: int = 100, seed: int = 0, spread: float = POCKET_RADIUS) -> np.ndarray:
    """Stand-in for the binding-site network's output (its top-scored voxel
    centres): n_points uniform in a ball of radius `spread` around the
    receptor's pocket centre, float32 [n_points][3]."""
    rng = _rng(seed, "SITE")
    return (rec.pocket_center + _ball(rng, n_points, spread)).astype(np.float32)


def shell_receptor(lig: Ligand, seed: int = 0, per_atom: int = 24, radius: float = 4.0, gap: float = 3.6,
                   spacing: float = 2.2, mouth_deg: float = 0.0) -> Receptor:
    """A redocking receptor built around a ligand's own pose: points `radius`
    from each ligand atom in random directions, none closer than `gap` to any
    ligand atom, thinned to one per `spacing`; all hydrophobic carbons (C_H),
    so the pose they were built around is the deepest minimum (dense enough
    that it also ranks first by the exact inter score, which the rescoring
    sorts by).  pocket_center = the ligand's centroid."""
    rng = _rng(seed, "SHEL")
    xyz = lig.xyz.astype(np.float64)
    d = rng.normal(size=(len(xyz), per_atom, 3))
    pts = (xyz[:, None, :] + radius * d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3)
    pts = pts[np.min(np.linalg.norm(pts[:, None] - xyz[None], axis=-1), axis=1) > gap]
    if mouth_deg > 0:  # an opening: no shell atom within mouth_deg of +z, seen from the centroid
        v = pts - xyz.mean(axis=0)
        pts = pts[v[:, 2] < np.cos(np.radians(mouth_deg)) * np.linalg.norm(v, axis=1)]
    out = []
    for p in pts:
        if all(np.linalg.norm(p - q) >= spacing for q in out):
            out.append(p)
    out = np.array(out, dtype=np.float32).reshape(-1, 3)
    return Receptor(out, np.zeros(len(out), dtype=np.uint8), xyz.mean(axis=0))


# Per-atom inputs of the receptor voxel features (the binding-site network's
# input, Sec. 2): 17 chemistry features -- 8 element classes with S and Se in one
# class (B, C, N, O, P, S/Se, halogen, metal) and 9 atom properties
# (hybridisation, heavy-atom valence, hetero-atom valence, partial charge,
# hydrophobic, aromatic, H-bond acceptor, H-bond donor, ring) -- and the
# Bondi van der Waals radius.  A synthetic receptor carries elements and XS
# donor / acceptor / hydrophobic flags only: the other properties are 0.
VOXEL_FEATURE_NAMES = ["B", "C", "N", "O", "P", "S/Se", "halogen", "metal", "hybridisation", "heavy_valence",
                       "hetero_valence", "partial_charge", "hydrophobic", "aromatic", "acceptor", "donor", "ring"]
_ELEMENT_OF_XS = {C_H: 1, C_P: 1, N_P: 2, N_D: 2, N_A: 2, O_A: 3, O_DA: 3, S_P: 5, N_DA: 2}
_BONDI = {1: 1.70, 2: 1.55, 3: 1.52, 5: 1.80}


def receptor_voxel_inputs(rec: Receptor):
    """(radius [n] float32, features [n][17] float32) of a synthetic receptor."""
    n = len(rec.xs_type)
    feats = np.zeros((n, len(VOXEL_FEATURE_NAMES)), dtype=np.float32)
    radius = np.zeros(n, dtype=np.float32)
    for i, t in enumerate(rec.xs_type.tolist()):
        e = _ELEMENT_OF_XS[t]
        feats[i, e] = 1.0
        radius[i] = _BONDI[e]
        feats[i, 12] = 1.0 if t == C_H else 0.0
        feats[i, 14] = 1.0 if t in (N_A, O_A, O_DA, N_DA) else 0.0
        feats[i, 15] = 1.0 if t in (N_D, O_DA, N_DA) else 0.0
    return radius, feats


def protein_center(rec: Receptor) -> np.ndarray:
    """Centre of the voxel cube: the mean of the heavy-atom coordinates."""
    return rec.xyz.astype(np.float64).mean(axis=0)


def box_around(center, size, spacing=0.375) -> Box:
    s = np.array(size if np.ndim(size) else [size] * 3, dtype=np.float64)
    return Box(np.asarray(center, dtype=np.float64), s, float(spacing))


@dataclass
class DockJob:
    receptor_seed: int
    receptor: Receptor
    box: Box
    ligands: list
    n_chains: int
    n_mc_steps: int
    seed: int = 0
    top_k: int = 9
    extra: dict = field(default_factory=dict)


def config(name: str, seed: int = 0) -> DockJob:
    """The docking workloads by name.

    plain-2k:   2,000-atom receptor, 20 A box at 0.375 A (54^3), ligand 20 atoms /
                4 torsions, 64 chains x 100 MC steps.
    typical-4k: 4,000-atom receptor, 30 A box (80^3), ligand 30 atoms / 8 torsions,
                384 chains x 40 MC steps, top-9 rescored in FP64.
    uneven-5k:  5,000-atom receptor, 26 A box (70^3), 256 ligands with 10-60 atoms
                and 0-15 torsions (capped by the tree), 128 chains x 40 steps each.
    typical-4k-batch16: the typical-4k receptor with 16 ligands (seeds 0..15).
    """
    if name == "plain-2k":
        rec = receptor(2000, seed)
        box = box_around(rec.pocket_center, 20.0)
        lig = ligand(20, 4, seed, center=rec.pocket_center)
        return DockJob(seed, rec, box, [lig], 64, 100, seed=seed)
    if name == "typical-4k":
        rec = receptor(4000, seed)
        box = box_around(rec.pocket_center, 30.0)
        lig = ligand(30, 8, seed, center=rec.pocket_center)
        return DockJob(seed, rec, box, [lig], 384, 40, seed=seed)
    if name == "typical-4k-batch16":
        rec = receptor(4000, seed)
        box = box_around(rec.pocket_center, 30.0)
        ligs = [ligand(30, 8, seed + i, center=rec.pocket_center) for i in range(16)]
        return DockJob(seed, rec, box, ligs, 384, 40, seed=seed)
    if name == "uneven-5k":
        rec = receptor(5000, seed)
        box = box_around(rec.pocket_center, 26.0)
        rng = _rng(seed, "UNEV")
        ligs = []
        for i in range(256):
            n = int(rng.integers(10, 61))
            t = int(rng.integers(0, 16))
            ligs.append(ligand(n, t, seed * 1000 + i, center=rec.pocket_center))
        return DockJob(seed, rec, box, ligs, 128, 40, seed=seed)
    raise KeyError(name)
