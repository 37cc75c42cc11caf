"""Pins of the oracle's adaptive search space (Sec. 2, third modification;
Fig. 3): initial positions uniform in the box intersected with the union of
balls around the predicted binding-site points (CPU)."""
import numpy as np

import oracle
from paper_2303_09916_gb300 import synth


def _lig(seed=0):
    s = synth.ligand(12, 3, seed)
    return oracle.Ligand(s.xyz.astype(np.float64), s.xs_type, s.bonds, s.rotatable)


LO, SIZE = np.array([-10.0, -10.0, -10.0]), np.array([20.0, 20.0, 20.0])


def _starts(lig, dp, n, seed=3):
    return np.array([oracle.chain_init(lig, dp, seed, c)[:3] for c in range(n)])


def test_every_start_lies_in_the_box_and_in_some_ball():
    lig = _lig()
    rng = np.random.default_rng(0)
    sites = rng.uniform(-6, 12, size=(40, 3)).astype(np.float32)  # some balls stick out of the box
    R = 3.0
    p = _starts(lig, oracle.dock_params_array(1, 0, 1.2, LO, SIZE, sites, R), 400)
    assert np.all(p >= LO) and np.all(p <= LO + SIZE)
    d = np.linalg.norm(p[:, None, :] - sites[None].astype(np.float64), axis=2).min(1)
    assert np.all(d <= R + 1e-5), d.max()  # the decision is FP32: allow its rounding at the sphere


def test_balls_covering_the_box_give_the_plain_box_start():
    """With one ball containing the whole box the first attempt (block 0, the
    box draw) is always accepted: the start is the box start, bitwise."""
    lig = _lig(1)
    box_dp = oracle.dock_params_array(1, 0, 1.2, LO, SIZE)
    ball_dp = oracle.dock_params_array(1, 0, 1.2, LO, SIZE, [[0.0, 0.0, 0.0]], 18.0)  # half-diagonal 17.3
    for c in range(50):
        assert np.array_equal(oracle.chain_init(lig, box_dp, 9, c), oracle.chain_init(lig, ball_dp, 9, c))


def test_starts_are_uniform_in_a_ball_inside_the_box():
    """One ball of radius R inside the box: the region is the ball.  Uniform in a
    ball: mean at the centre, E|p - c|^2 = 3 R^2 / 5, P(|p - c| < R / 2) = 1 / 8."""
    lig = _lig(2)
    c0 = np.array([2.0, -1.0, 0.5], dtype=np.float32)
    R = 5.0
    n = 3000
    p = _starts(lig, oracle.dock_params_array(1, 0, 1.2, LO, SIZE, [c0], R), n)
    r = np.linalg.norm(p - c0.astype(np.float64), axis=1)
    assert np.all(r <= R + 1e-5)
    sd = R / np.sqrt(5.0)  # per-axis standard deviation of the uniform ball
    assert np.all(np.abs(p.mean(0) - c0) < 4 * sd / np.sqrt(n))
    m2, var_r2 = 3 * R ** 2 / 5, (3 / 7 - 9 / 25) * R ** 4
    assert abs(np.mean(r ** 2) - m2) < 4 * np.sqrt(var_r2 / n)
    f = np.mean(r < R / 2)
    assert abs(f - 1 / 8) < 4 * np.sqrt(1 / 8 * 7 / 8 / n)


def test_no_intersection_falls_back_to_the_first_point():
    lig = _lig(3)
    sites = np.array([[50.0, 50.0, 50.0], [60.0, 0.0, 0.0]], dtype=np.float32)
    p = _starts(lig, oracle.dock_params_array(1, 0, 1.2, LO, SIZE, sites, 2.0), 5)
    assert np.all(p == sites[0].astype(np.float64))


def test_orientation_and_torsions_do_not_depend_on_the_region():
    lig = _lig(4)
    box_dp = oracle.dock_params_array(1, 0, 1.2, LO, SIZE)
    ball_dp = oracle.dock_params_array(1, 0, 1.2, LO, SIZE, [[1.0, 2.0, 3.0]], 4.0)
    for c in range(20):
        a, b = oracle.chain_init(lig, box_dp, 5, c), oracle.chain_init(lig, ball_dp, 5, c)
        assert np.array_equal(a[3:], b[3:])
