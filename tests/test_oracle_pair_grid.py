"""Pins of the oracle's pair score, grid maps and interpolation (CPU only).

Each expected value here comes from a closed form, an identity of the
mathematics or a brute-force sum on a tiny input -- never from the oracle
calling itself with the same formula.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

# Vina weights as published with the scoring function DSDP adopts (paper Sec. 2,
# its ref. 6); written out here independently of the oracle source.
W_G1, W_G2, W_REP, W_HYD, W_HB = -0.0356, -0.00516, 0.840, -0.0351, -0.587
C_H, C_P, N_P, N_D, N_A, O_A, O_DA, S_P, N_DA = range(9)


def test_constants_are_the_vina_reading():
    c = oracle.constants()
    assert (c["w_gauss1"], c["w_gauss2"], c["w_repulsion"], c["w_hydrophobic"], c["w_hbond"]) == (
        W_G1, W_G2, W_REP, W_HYD, W_HB)
    assert c["cutoff"] == 8.0 and c["w_rot"] == 0.0585


@pytest.mark.parametrize("ti,tj,r,expected", [
    # polar carbons, d = 0: gauss1 = 1, gauss2 = e^-2.25, nothing else
    (C_P, C_P, 3.8, W_G1 + W_G2 * math.exp(-2.25)),
    # d = -1: gauss1 = e^-4, gauss2 = e^-4, repulsion = 1
    (C_P, C_P, 2.8, W_G1 * math.exp(-4) + W_G2 * math.exp(-4) + W_REP),
    # hydrophobic pair at d = 0 -> hydrophobic term fully on
    (C_H, C_H, 3.8, W_G1 + W_G2 * math.exp(-2.25) + W_HYD),
    # hydrophobic pair at d = 1 -> half way down the ramp; gauss1 = e^-4, gauss2 = e^-1
    (C_H, C_H, 4.8, W_G1 * math.exp(-4) + W_G2 * math.exp(-1) + 0.5 * W_HYD),
    # hydrophobic with polar: no hydrophobic term
    (C_H, C_P, 4.8, W_G1 * math.exp(-4) + W_G2 * math.exp(-1)),
    # donor N with acceptor O (R sum 3.5), d = -0.35: H-bond half on, repulsion d^2
    (N_D, O_A, 3.15, W_G1 * math.exp(-0.49) + W_G2 * math.exp(-(3.35 / 2) ** 2) + W_REP * 0.1225 + 0.5 * W_HB),
    # the same pair the other way round
    (O_A, N_D, 3.15, W_G1 * math.exp(-0.49) + W_G2 * math.exp(-(3.35 / 2) ** 2) + W_REP * 0.1225 + 0.5 * W_HB),
    # acceptor-acceptor: no H-bond
    (N_A, O_A, 3.15, W_G1 * math.exp(-0.49) + W_G2 * math.exp(-(3.35 / 2) ** 2) + W_REP * 0.1225),
    # donor-acceptor deep inside: H-bond saturated (d = -1)
    (O_DA, N_DA, 2.5, W_G1 * math.exp(-4) + W_G2 * math.exp(-4) + W_REP + W_HB),
    # sulfur radius 2.0: S_P-S_P d = 0 at r = 4
    (S_P, S_P, 4.0, W_G1 + W_G2 * math.exp(-2.25)),
    # beyond the cutoff
    (C_H, C_H, 8.0, 0.0),
    (C_H, C_H, 9.5, 0.0),
])
def test_pair_closed_forms(ti, tj, r, expected):
    e, _ = oracle.pair(ti, tj, r)
    assert e == pytest.approx(expected, rel=1e-13, abs=1e-15)


def test_pair_just_inside_cutoff_is_gauss2_tail():
    e, _ = oracle.pair(C_P, C_P, 7.999)
    d = 7.999 - 3.8
    assert e == pytest.approx(W_G1 * math.exp(-(d / 0.5) ** 2) + W_G2 * math.exp(-((d - 3) / 2) ** 2), rel=1e-13)


def test_pair_derivative_matches_central_difference():
    rng = np.random.default_rng(1)
    kinks = []
    for ti in range(8):
        for tj in range(9):
            R = [1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0, 1.8]
            kinks = [R[ti] + R[tj] + k for k in (-0.7, 0.0, 0.5, 1.5)] + [8.0]
            for r in rng.uniform(1.0, 8.5, size=20):
                if min(abs(r - k) for k in kinks) < 1e-4:
                    continue
                h = 1e-6
                _, de = oracle.pair(ti, tj, r)
                fd = (oracle.pair(ti, tj, r + h)[0] - oracle.pair(ti, tj, r - h)[0]) / (2 * h)
                assert de == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_pair_symmetric():
    for ti in range(8):
        for tj in range(8):
            for r in (2.5, 3.3, 4.1, 6.0):
                assert oracle.pair(ti, tj, r) == oracle.pair(tj, ti, r)


def test_grid_dims_match_workload_sizes():
    assert list(oracle.grid_dims([20, 20, 20], 0.375)) == [54, 54, 54]
    assert list(oracle.grid_dims([30, 30, 30], 0.375)) == [80, 80, 80]
    assert list(oracle.grid_dims([26, 26, 26], 0.375)) == [70, 70, 70]


def _small_receptor(n=60, seed=0, spread=6.0):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-spread, spread, size=(n, 3))
    types = rng.integers(0, 9, size=n)
    return xyz, types


def test_grid_single_atom_closed_form():
    # one receptor atom placed so that vertex (2, 3, 4) sits exactly r = 3.8 away along x:
    # a C_P ligand type there sees d = 0 against a C_P receptor atom.
    h = 0.5
    center = np.zeros(3)
    size = np.array([4.0, 4.0, 4.0])
    n = oracle.grid_dims(size, h)
    origin = center - (n - 1) * h / 2
    vertex = origin + h * np.array([2, 3, 4])
    atom = vertex + np.array([3.8, 0.0, 0.0])
    g = oracle.grid_build(atom[None], [C_P], center, size, h)
    node = g.maps[C_P, 4, 3, 2]
    assert node[0] == pytest.approx(W_G1 + W_G2 * math.exp(-2.25), rel=1e-12)
    # gradient w.r.t. the vertex: df/dd at d = 0 is gauss2' = W_G2 e^-2.25 * (-2 (0 - 3) / 4) = 1.5 W_G2 e^-2.25;
    # the vertex lies on the -x side, so dE/dx = -slope.
    slope = 1.5 * W_G2 * math.exp(-2.25)
    assert node[1] == pytest.approx(-slope, rel=1e-12)
    assert abs(node[2]) < 1e-15 and abs(node[3]) < 1e-15


def test_grid_superposition():
    xyz, types = _small_receptor()
    center, size, h = np.zeros(3), np.array([3.0, 3.0, 3.0]), 0.75
    ga = oracle.grid_build(xyz[:30], types[:30], center, size, h)
    gb = oracle.grid_build(xyz[30:], types[30:], center, size, h)
    gab = oracle.grid_build(xyz, types, center, size, h)
    assert np.allclose(gab.maps, ga.maps + gb.maps, rtol=1e-12, atol=1e-14)


def test_grid_matches_brute_force_pair_sum():
    # tiny brute force: vertex by vertex, atom by atom, with the pinned pair function
    xyz, types = _small_receptor(n=12, spread=4.0)
    center, size, h = np.array([0.3, -0.2, 0.1]), np.array([1.5, 1.5, 1.5]), 0.5
    g = oracle.grid_build(xyz, types, center, size, h)
    n = g.n
    for t in range(8):
        for iz in range(n[2]):
            for iy in range(n[1]):
                for ix in range(n[0]):
                    m = g.origin + h * np.array([ix, iy, iz])
                    e = 0.0
                    grad = np.zeros(3)
                    for j in range(len(types)):
                        dv = m - xyz[j]
                        r = float(np.linalg.norm(dv))
                        f, df = oracle.pair(t, int(types[j]), r)
                        e += f
                        if r > 0:
                            grad += df * dv / r
                    node = g.maps[t, iz, iy, ix]
                    assert node[0] == pytest.approx(e, rel=1e-12, abs=1e-15)
                    assert np.allclose(node[1:], grad, rtol=1e-12, atol=1e-14)


def test_gradient_channels_are_the_derivative_of_the_score_field():
    xyz, types = _small_receptor(n=40)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-2, 2, size=(25, 3))
    h = 1e-6
    for t in range(8):
        f = oracle.receptor_field(xyz, types, t, pts)
        for a in range(3):
            dp = pts.copy()
            dm = pts.copy()
            dp[:, a] += h
            dm[:, a] -= h
            fd = (oracle.receptor_field(xyz, types, t, dp)[:, 0] - oracle.receptor_field(xyz, types, t, dm)[:, 0]) / (2 * h)
            # skip points whose stencil straddles a kink or the cutoff
            ok = np.abs(fd - f[:, 1 + a]) < 1e-5 * np.maximum(1, np.abs(fd))
            assert ok.mean() > 0.9
            assert np.allclose(f[ok, 1 + a], fd[ok], rtol=1e-5, atol=1e-7)


def test_grid_integer_node_translation():
    xyz, types = _small_receptor(n=50)
    h = 0.5
    center, size = np.zeros(3), np.array([3.0, 3.0, 3.0])
    shift = h * np.array([3, -2, 5])
    g0 = oracle.grid_build(xyz, types, center, size, h)
    g1 = oracle.grid_build(xyz + shift, types, center + shift, size, h)
    assert np.allclose(g0.maps, g1.maps, rtol=1e-10, atol=1e-12)


def test_grid_rotation_90_about_z():
    xyz, types = _small_receptor(n=50)
    h = 0.5
    center, size = np.zeros(3), np.array([3.0, 3.0, 3.0])
    rot = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], dtype=float)  # (x, y) -> (-y, x)
    g0 = oracle.grid_build(xyz, types, center, size, h)
    g1 = oracle.grid_build(xyz @ rot.T, types, center, size, h)
    n = g0.n[0]
    # vertex (ix, iy) of the rotated grid sits at rot^T applied: original vertex (iy, n-1-ix)
    for t in range(8):
        for iy in range(n):
            for ix in range(n):
                a = g1.maps[t, :, iy, ix]
                b = g0.maps[t, :, n - 1 - ix, iy]
                assert np.allclose(a[:, 0], b[:, 0], rtol=1e-10, atol=1e-12)
                assert np.allclose(a[:, 1:], b[:, 1:] @ rot.T, rtol=1e-10, atol=1e-12)


def _grid_from_field(fn, n=6, h=0.7, origin=(-1.0, 0.5, 2.0), grad_fn=None):
    origin = np.array(origin)
    maps = np.zeros((8, n, n, n, 4))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                p = origin + h * np.array([ix, iy, iz])
                for t in range(8):
                    maps[t, iz, iy, ix, 0] = fn(p, t)
                    if grad_fn is not None:
                        maps[t, iz, iy, ix, 1:] = grad_fn(p, t)
    return oracle.Grid(maps, [n, n, n], origin, h)


def _multilinear(p, t):
    x, y, z = p
    return 0.3 + t + 1.1 * x - 0.7 * y + 0.2 * z + 0.5 * x * y - 0.3 * y * z + 0.25 * x * z + 0.15 * x * y * z


def _multilinear_grad(p, t):
    x, y, z = p
    return np.array([1.1 + 0.5 * y + 0.25 * z + 0.15 * y * z,
                     -0.7 + 0.5 * x - 0.3 * z + 0.15 * x * z,
                     0.2 - 0.3 * y + 0.25 * x + 0.15 * x * y])


def test_interpolation_reproduces_multilinear_fields():
    g = _grid_from_field(_multilinear, grad_fn=_multilinear_grad)
    rng = np.random.default_rng(0)
    pts = g.origin + rng.uniform(0, 5 * g.h, size=(200, 3))
    for t in (0, 3, 7):
        exact = np.array([_multilinear(p, t) for p in pts])
        exact_g = np.array([_multilinear_grad(p, t) for p in pts])
        for mode in (0, 1):
            e, grad = oracle.interpolate(g, mode, t, pts)
            assert np.allclose(e, exact, rtol=1e-12, atol=1e-12)  # Eq. 2
            # Eq. 4 interpolates exact multilinear gradient maps; Eq. 3 differentiates the
            # (exact) interpolant.  Both reproduce the gradient of a multilinear field.
            assert np.allclose(grad, exact_g, rtol=1e-10, atol=1e-10), mode


def test_eq3_is_the_derivative_of_eq2():
    g = _grid_from_field(lambda p, t: math.sin(p[0]) * math.cos(1.3 * p[1]) + p[2] ** 2 + t)
    rng = np.random.default_rng(5)
    pts = g.origin + rng.uniform(0.05, 4.95 * g.h, size=(100, 3))
    # stay away from cell faces where Eq. 3 jumps
    frac = ((pts - g.origin) / g.h) % 1.0
    pts = pts[np.all((frac > 1e-3) & (frac < 1 - 1e-3), axis=1)]
    e, grad = oracle.interpolate(g, 1, 2, pts)
    h = 1e-7
    for a in range(3):
        dp, dm = pts.copy(), pts.copy()
        dp[:, a] += h
        dm[:, a] -= h
        fd = (oracle.interpolate(g, 1, 2, dp)[0] - oracle.interpolate(g, 1, 2, dm)[0]) / (2 * h)
        assert np.allclose(grad[:, a], fd, rtol=1e-6, atol=1e-7)


def test_eq4_converges_second_order():
    f = lambda p, t: math.sin(p[0]) * math.cos(p[1]) * math.sin(0.5 * p[2] + 0.3)
    gf = lambda p, t: np.array([math.cos(p[0]) * math.cos(p[1]) * math.sin(0.5 * p[2] + 0.3),
                                -math.sin(p[0]) * math.sin(p[1]) * math.sin(0.5 * p[2] + 0.3),
                                0.5 * math.sin(p[0]) * math.cos(p[1]) * math.cos(0.5 * p[2] + 0.3)])
    rng = np.random.default_rng(2)
    pts = rng.uniform(0.2, 1.8, size=(300, 3))
    errs = []
    for h, n in ((0.2, 11), (0.1, 21), (0.05, 41)):
        g = _grid_from_field(f, n=n, h=h, origin=(0, 0, 0), grad_fn=gf)
        e, grad = oracle.interpolate(g, 0, 0, pts)
        exact_g = np.array([gf(p, 0) for p in pts])
        errs.append(np.abs(grad - exact_g).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_outside_the_grid_pays_the_wall():
    g = _grid_from_field(_multilinear, grad_fn=_multilinear_grad)
    top = g.origin + (g.n - 1) * g.h
    inside = np.array([g.origin[0] + 1.0, top[1], g.origin[2] + 0.5])
    outside = inside + np.array([0.0, 0.8, 0.0])
    below = np.array([g.origin[0] - 0.3, g.origin[1] + 1.0, g.origin[2] + 1.0])
    e_in, g_in = oracle.interpolate(g, 0, 1, inside[None])
    e_out, g_out = oracle.interpolate(g, 0, 1, outside[None])
    assert e_out[0] == pytest.approx(e_in[0] + 10.0 * 0.8, rel=1e-12)
    assert g_out[0, 1] == 10.0
    assert g_out[0, 0] == pytest.approx(g_in[0, 0]) and g_out[0, 2] == pytest.approx(g_in[0, 2])
    e_b, g_b = oracle.interpolate(g, 0, 1, below[None])
    clamped = below.copy()
    clamped[0] = g.origin[0]
    e_c, _ = oracle.interpolate(g, 0, 1, clamped[None])
    assert e_b[0] == pytest.approx(e_c[0] + 10.0 * 0.3, rel=1e-12)
    assert g_b[0, 0] == -10.0


def test_interpolation_continuous_across_cell_faces():
    xyz, types = _small_receptor(n=40)
    g = oracle.grid_build(xyz, types, np.zeros(3), np.array([3.0, 3.0, 3.0]), 0.5)
    face = g.origin[0] + 3 * g.h
    rng = np.random.default_rng(9)
    for _ in range(20):
        y, z = rng.uniform(g.origin[1], g.origin[1] + 5 * g.h, size=2)
        a = np.array([[face - 1e-9, y, z]])
        b = np.array([[face + 1e-9, y, z]])
        for mode in (0, 1):
            ea, ga = oracle.interpolate(g, mode, 2, a)
            eb, gb = oracle.interpolate(g, mode, 2, b)
            assert ea[0] == pytest.approx(eb[0], abs=1e-7)
        # Eq. 4 gradients are continuous too (the paper's reason for the gradient maps)
        ea, ga = oracle.interpolate(g, 0, 2, a)
        eb, gb = oracle.interpolate(g, 0, 2, b)
        assert np.allclose(ga, gb, atol=1e-7)


def test_synthetic_receptor_shape():
    rec = synth.receptor(2000, 0)
    assert rec.xyz.shape == (2000, 3)
    d = np.linalg.norm(rec.xyz[:, None, :] - rec.xyz[None, :, :], axis=-1)
    np.fill_diagonal(d, 1e9)
    assert d.min() >= 2.8
    frac = np.bincount(rec.xs_type, minlength=9) / 2000.0
    carbon = frac[C_H] + frac[C_P]
    assert 0.58 < carbon < 0.66


@pytest.mark.parametrize("mouth", [0.0, 60.0])
def test_shell_receptor_shape(mouth):
    """The redocking shell keeps its stated geometry: every atom between the gap
    and the radius from the nearest ligand atom (and exactly the radius from the
    ligand atom it was drawn around), at least the thinning spacing apart, none
    in the mouth, and the same shell from the same seed."""
    lig = synth.ligand(20, 4, 3)
    rec = synth.shell_receptor(lig, 7, mouth_deg=mouth)
    xyz = lig.xyz.astype(np.float64)
    pts = rec.xyz.astype(np.float64)
    assert len(pts) > 20 and np.all(rec.xs_type == 0)
    d = np.linalg.norm(pts[:, None] - xyz[None], axis=-1)
    assert np.all(d.min(axis=1) > 3.6 - 1e-5) and np.all(d.min(axis=1) <= 4.0 + 1e-5)
    assert np.all(np.abs(d - 4.0).min(axis=1) < 1e-5)
    pp = np.linalg.norm(pts[:, None] - pts[None], axis=-1) + np.eye(len(pts)) * 1e9
    assert pp.min() >= 2.2 - 1e-5
    assert np.allclose(rec.pocket_center, xyz.mean(axis=0))
    if mouth:
        v = pts - xyz.mean(axis=0)
        assert np.all(v[:, 2] < np.cos(np.radians(mouth)) * np.linalg.norm(v, axis=1) + 1e-5)
    again = synth.shell_receptor(lig, 7, mouth_deg=mouth)
    assert np.array_equal(again.xyz, rec.xyz)
