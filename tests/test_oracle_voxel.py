"""Pins of the oracle's receptor voxel features (Sec. 2, binding-site
prediction input: 36^3 voxels over 70 A, 18 channels -- 17 chemistry features
with S and Se merged, one surface channel) and of its Shrake-Rupley surface
atoms, against hand-placed atoms, closed forms and a brute-force recount."""
import math

import numpy as np

import oracle
from paper_2303_09916_gb300 import synth

H = 70.0 / 36.0


def _feat(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 3, size=(n, 17)).astype(np.float32)


def test_directions_are_the_98_primitive_integer_vectors():
    u = oracle.sas_directions()
    assert u.shape == (98, 3)
    assert np.allclose(np.linalg.norm(u.astype(np.float64), axis=1), 1.0, atol=1e-7)
    # each direction is a normalised integer vector with entries in -2..2 and gcd 1, all distinct
    seen = set()
    for v in u.astype(np.float64):
        k = np.round(v / np.abs(v[np.abs(v) > 1e-6]).min()).astype(int)
        assert np.allclose(k / np.linalg.norm(k), v, atol=1e-6) and np.abs(k).max() <= 2
        assert math.gcd(math.gcd(abs(k[0]), abs(k[1])), abs(k[2])) == 1
        seen.add(tuple(k))
    assert len(seen) == 98
    assert np.allclose(u.astype(np.float64).sum(0), 0.0, atol=1e-6)  # symmetric set


def test_a_single_atom_lands_in_its_voxel_with_its_features_and_is_surface():
    c = np.array([10.0, -4.0, 3.0])
    for k in (0, 7, 18, 35):
        # the centre of voxel k along x (y, z: voxel 18)
        x = np.array([[c[0] - 35.0 + (k + 0.5) * H, c[1] + 0.5 * H, c[2] + 0.5 * H]], dtype=np.float32)
        f = _feat(1, k)
        out, inside = oracle.voxelize(x, [1.7], f, c)
        assert inside == 1
        nz = np.argwhere(out.any(-1))
        assert nz.tolist() == [[18, 18, k]]  # (z, y, x)
        assert np.array_equal(out[18, 18, k, :17], f[0])
        assert out[18, 18, k, 17] == 1.0  # an isolated atom exposes all 98 points
        assert oracle.sas_exposed(x, [1.7]).tolist() == [98]


def test_atoms_outside_the_cube_are_dropped_and_sums_add():
    c = np.zeros(3)
    inside_pts = [[0.1, 0.2, 0.3], [0.2, 0.3, 0.4], [-34.9, 0.0, 0.0], [34.9, 34.9, -34.9]]
    outside_pts = [[35.5, 0, 0], [0, -35.01, 0], [0, 0, 100.0]]
    x = np.array(inside_pts + outside_pts, dtype=np.float32)
    f = _feat(len(x), 3)
    out, inside = oracle.voxelize(x, np.full(len(x), 1.5), f, c)
    assert inside == 4
    # the first two atoms share voxel (18, 18, 18): their features add
    assert np.array_equal(out[18, 18, 18, :17], f[0] + f[1])
    assert out[18, 18, 18, 17] == 2.0  # both on the surface (nothing else nearby)
    assert np.array_equal(out[18, 18, 0, :17], f[2]) and np.array_equal(out[0, 35, 35, :17], f[3])
    assert out[..., :17].sum() == f[:4].sum()


def test_a_buried_atom_is_not_surface_and_its_shell_is():
    # an atom at the centre of the 12 face-centred-cubic neighbours at 2.6 A:
    # every test point of the centre lies within 45 deg of a neighbour direction,
    # inside that neighbour's sphere (cos > 2.6 / (2 x 3.1) = 0.42)
    dirs = np.array([[a, b, 0] for a in (-1, 1) for b in (-1, 1)] + [[a, 0, b] for a in (-1, 1) for b in (-1, 1)]
                    + [[0, a, b] for a in (-1, 1) for b in (-1, 1)], dtype=np.float64) / math.sqrt(2)
    x = np.vstack([np.zeros((1, 3)), 2.6 * dirs]).astype(np.float32)
    ex = oracle.sas_exposed(x, np.full(13, 1.7))
    assert ex[0] == 0 and np.all(ex[1:] > 0)
    out, _ = oracle.voxelize(x, np.full(13, 1.7), np.zeros((13, 17), np.float32), np.zeros(3))
    assert out[..., 17].sum() == 12.0


def test_exposed_points_of_two_spheres_follow_the_cap_geometry():
    # two atoms of radius r at distance d: a test point u of atom 0 lies in atom 1's
    # sphere iff u . e > d / (2 (r + 1.4)), e the unit vector from 0 to 1
    u = oracle.sas_directions().astype(np.float64)
    e = np.array([1.0, 2.0, 2.0]) / 3.0
    for d in (1.0, 2.5, 3.3, 4.9, 6.5):
        R = 1.7 + 1.4
        x = np.array([[0, 0, 0], d * e], dtype=np.float32)
        expect = int(np.sum(u @ e <= d / (2 * R) + 1e-9))
        ex = oracle.sas_exposed(x, [1.7, 1.7])
        assert ex[0] == expect and ex[1] == expect, (d, ex, expect)
        # and the buried fraction is near the cap area fraction (R - d/2) / (2 R)
        assert abs((98 - expect) / 98 - max(R - d / 2, 0) / (2 * R)) < 0.12


def test_brute_force_recount_and_atom_order_independence():
    rec = synth.receptor(400, 5)
    radius, feats = synth.receptor_voxel_inputs(rec)
    c = synth.protein_center(rec)
    out, inside = oracle.voxelize(rec.xyz, radius, feats, c)
    x = rec.xyz.astype(np.float32)
    lo = (c - 35.0).astype(np.float32)
    k = np.floor((x - lo) * np.float32(36.0 / 70.0)).astype(int)
    ok = np.all((k >= 0) & (k < 36), axis=1)
    assert inside == ok.sum() == 400  # a 400-atom protein fits the 70 A cube
    ref = np.zeros((36, 36, 36, 18))
    surf = oracle.sas_exposed(x, radius) > 0
    for i in np.nonzero(ok)[0]:
        ref[k[i, 2], k[i, 1], k[i, 0], :17] += feats[i]
        ref[k[i, 2], k[i, 1], k[i, 0], 17] += surf[i]
    assert np.array_equal(out, ref.astype(np.float32))
    assert 0 < surf.sum() < 400
    perm = np.random.default_rng(1).permutation(400)
    out2, _ = oracle.voxelize(rec.xyz[perm], radius[perm], feats[perm], c)
    assert np.array_equal(out, out2)
    # non-integer features: exact fixed-point sums, the same in any order
    fr = np.random.default_rng(2).uniform(-1, 1, size=feats.shape).astype(np.float32)
    o1, _ = oracle.voxelize(rec.xyz, radius, fr, c)
    o2, _ = oracle.voxelize(rec.xyz[perm], radius[perm], fr[perm], c)
    assert np.array_equal(o1, o2)
    assert np.allclose(o1[..., :17].sum(), fr.astype(np.float64).sum(), atol=1e-3)
