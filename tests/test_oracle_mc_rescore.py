"""Pins of the oracle's Monte Carlo chains and its rescoring / top-k (CPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth


def _complex(seed=0, n_lig=10, T=3, n_rec=300, box=14.0):
    rec = synth.receptor(n_rec, seed)
    s = synth.ligand(n_lig, T, seed, center=rec.pocket_center)
    lig = oracle.Ligand(s.xyz.astype(np.float64), s.xs_type, s.bonds, s.rotatable)
    size = np.array([box] * 3)
    grid = oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, size, 0.5)
    lo = rec.pocket_center - size / 2
    return rec, s, lig, grid, lo, size


def test_chain_is_deterministic_and_independent_of_the_batch():
    rec, s, lig, grid, lo, size = _complex()
    dp = oracle.dock_params_array(4, 0, 1.2, lo, size)
    opt = dict(max_iters=20)
    best, e_best, evals = oracle.dock(lig, grid, 0, dp, seed=5, n_chains=4, n_threads=2, opt=opt)
    for c in range(4):
        r = oracle.run_chain(lig, grid, 0, dp, 5, c, opt=opt)
        assert np.array_equal(r["best"], best[c]) and r["e_best"] == e_best[c] and r["evals"] == evals[c]
    # a sub-batch starting at chain 2 gives the same chains 2, 3
    b2, e2, _ = oracle.dock(lig, grid, 0, dp, seed=5, n_chains=2, chain0=2, opt=opt)
    assert np.array_equal(b2, best[2:]) and np.array_equal(e2, e_best[2:])
    # another seed gives another chain
    b3, e3, _ = oracle.dock(lig, grid, 0, dp, seed=6, n_chains=1, opt=opt)
    assert not np.array_equal(b3[0], best[0])


def test_metropolis_and_best_tracking_rules_hold_along_the_trace():
    rec, s, lig, grid, lo, size = _complex(1)
    dp = oracle.dock_params_array(30, 0, 1.2, lo, size)
    for chain in range(3):
        r = oracle.run_chain(lig, grid, 0, dp, 9, chain, opt=dict(max_iters=15))
        tr = r["trace_rec"]
        e_prev = tr[0, 3]
        best = e_prev
        n_acc = 0
        for st in range(1, 31):
            mode, acc, e_cand, e_cur, _ = tr[st]
            assert 0 <= mode < 2 + lig.T
            if e_cand < e_prev:
                assert acc == 1
            if acc:
                assert e_cur == e_cand
                best = min(best, e_cur)
                n_acc += 1
            else:
                assert e_cur == e_prev
            e_prev = e_cur
        assert r["e_best"] == pytest.approx(best)
        assert lig.score_grid(grid, 0, r["best"])[0].sum() == pytest.approx(r["e_best"], rel=1e-12)


def test_metropolis_acceptance_rate_follows_exp():
    # The acceptance test compares a Philox uniform with exp(-dE/T): over many
    # uphill candidates the mean acceptance must equal the mean of min(1, exp(-dE/T)).
    rec, s, lig, grid, lo, size = _complex(2)
    T = 1.2
    dp = oracle.dock_params_array(1, 0, T, lo, size)
    probs, accs = [], []
    for chain in range(300):
        c0 = oracle.chain_init(lig, dp, 3, chain)
        c, e, _, _ = lig.local_opt(grid, 0, 0, c0, opt=dict(max_iters=5))
        e_cur = e - 0.5  # pretend the current state sits 0.5 lower, so most candidates are uphill
        _, _, rec_ = oracle.mc_step(lig, grid, 0, dp, 3, chain, 1, c, e_cur, opt=dict(max_iters=5))
        de = rec_[2] - e_cur
        probs.append(1.0 if de < 0 else math.exp(-de / T))
        accs.append(rec_[1])
    probs, accs = np.array(probs), np.array(accs)
    assert abs(accs.mean() - probs.mean()) < 4 * math.sqrt(probs.mean() * (1 - probs.mean()) / len(probs)) + 0.01


def test_chain_init_lies_in_the_box_with_unit_quaternion():
    rec, s, lig, grid, lo, size = _complex(3)
    dp = oracle.dock_params_array(1, 0, 1.2, lo, size)
    P = np.array([oracle.chain_init(lig, dp, 0, c) for c in range(500)])
    assert np.all(P[:, :3] >= lo) and np.all(P[:, :3] < lo + size)
    assert np.allclose(np.linalg.norm(P[:, 3:7], axis=1), 1.0, atol=1e-12)
    assert np.all(np.abs(P[:, 7:]) <= math.pi)
    # Shoemake's construction is uniform on SO(3): E[w^2] = 1/4 for each component
    assert np.allclose((P[:, 3:7] ** 2).mean(0), 0.25, atol=0.03)


def test_self_docking_finds_the_reference_pose():
    """Sanity, not parity: a receptor shell built around the ligand's own pose."""
    s = synth.ligand(10, 2, 4)
    lig = oracle.Ligand(s.xyz.astype(np.float64), s.xs_type, s.bonds, s.rotatable)
    rng = np.random.default_rng(0)
    shell = []
    for x in s.xyz.astype(np.float64):
        for _ in range(12):
            d = rng.normal(size=3)
            shell.append(x + 4.2 * d / np.linalg.norm(d))
    shell = np.array(shell)
    keep = np.min(np.linalg.norm(shell[:, None] - s.xyz[None].astype(np.float64), axis=-1), axis=1) > 3.8
    rec_xyz = shell[keep]
    rec_t = np.full(len(rec_xyz), 0)  # hydrophobic carbons: attractive everywhere near contact
    size = np.array([12.0] * 3)
    grid = oracle.grid_build(rec_xyz, rec_t, np.zeros(3), size, 0.4)
    dp = oracle.dock_params_array(15, 0, 1.2, -size / 2, size)
    best, e_best, _ = oracle.dock(lig, grid, 0, dp, seed=1, n_chains=24, n_threads=4, opt=dict(max_iters=60))
    top = int(np.argmin(e_best))
    x = lig.coords(best[top])
    rmsd = float(np.sqrt(((x - s.xyz) ** 2).sum(1).mean()))
    assert rmsd < 2.0, rmsd


def test_rescore_is_sorted_deduplicated_and_brute_force_exact():
    rec, s, lig, grid, lo, size = _complex(4, n_lig=7, T=2, n_rec=150)
    rng = np.random.default_rng(5)
    confs = []
    for _ in range(12):
        c = lig.identity_conf()
        c[:3] += rng.uniform(-2, 2, 3)
        q = rng.normal(size=4)
        c[3:7] = q / np.linalg.norm(q)
        c[7:] = rng.uniform(-math.pi, math.pi, lig.T)
        confs.append(c)
    confs.append(confs[3] + np.r_[1e-3, 0, 0, np.zeros(lig.nx - 3)])  # a near-duplicate of pose 3
    confs = np.array(confs)
    rxyz = rec.xyz.astype(np.float64)
    scores, idx, terms = oracle.rescore_topk(lig, rxyz, rec.xs_type, confs, k=5, rmsd_cut=1.0)
    # brute-force exact inter energy with the pinned pair function
    for p in (0, 3, 12):
        x = lig.coords(confs[p])
        inter = 0.0
        for i in range(len(x)):
            d = np.linalg.norm(rxyz - x[i], axis=1)
            for j in np.nonzero(d < 8.0)[0]:
                inter += oracle.pair(int(s.xs_type[i]), int(rec.xs_type[j]), float(d[j]))[0]
        assert scores[p] == pytest.approx(inter / (1 + 0.0585 * lig.T), rel=1e-12)
    assert len(idx) == 5
    assert np.all(np.diff(terms[:, 0]) >= 0)
    assert terms[0, 0] == scores.min()
    coords = [lig.coords(confs[i]) for i in idx]
    for a in range(len(idx)):
        for b in range(a + 1, len(idx)):
            assert np.sqrt(((coords[a] - coords[b]) ** 2).sum(1).mean()) >= 1.0
    assert not (3 in idx and 12 in idx)
    # every dropped pose that ranks above the last kept one is within 1 A of a kept one
    order = np.argsort(scores, kind="stable")
    last = list(order).index(idx[-1])
    for p in order[:last]:
        if p in idx:
            continue
        xp = lig.coords(confs[p])
        assert min(np.sqrt(((xp - lig.coords(confs[q])) ** 2).sum(1).mean()) for q in idx) < 1.0


def test_mutations_follow_the_stated_moves():
    """With local optimisation off (0 iterations) and every candidate accepted
    (current energy +inf), one MC step returns the mutation itself.  The mode is
    uniform over the 2 + T choices; a position move adds 2 A times a point
    uniform in the unit ball and keeps q and the torsions; an orientation move
    keeps p and the torsions and rotates by (2 / R_gyr) times a unit-ball point
    (R_gyr about the root origin: the lowest atom of the body with most atoms);
    a torsion move re-draws that torsion alone, in (-pi, pi]."""
    rec, s, lig, grid, lo, size = _complex(3, n_lig=12, T=4)
    body_of, _, _ = lig.bodies()
    members = [np.flatnonzero(body_of == b) for b in range(lig.n_bodies)]
    root = max(range(lig.n_bodies), key=lambda b: (len(members[b]), -members[b].min()))
    xyz = s.xyz.astype(np.float64)
    r_gyr = math.sqrt(np.mean(np.sum((xyz - xyz[members[root].min()]) ** 2, axis=1)))
    assert lig.gyration_radius == pytest.approx(r_gyr, rel=1e-12)
    k_rot = 2.0 / r_gyr
    dp = oracle.dock_params_array(1, 0, 1.2, lo, size)
    off = dict(max_iters=0)
    n = 1500
    modes, r3_pos, dirs, r3_rot = [], [], [], []
    for chain in range(n):
        cur = oracle.chain_init(lig, dp, 11, chain, opt=off)
        new, _, rec_ = oracle.mc_step(lig, grid, 0, dp, 11, chain, 1, cur, 1e300, opt=off)
        m = int(rec_[0])
        assert rec_[1] == 1
        modes.append(m)
        d_p, th0, th1 = new[:3] - cur[:3], cur[7:], new[7:]
        if m == 0:
            assert np.array_equal(new[3:], cur[3:])
            r = np.linalg.norm(d_p)
            assert r <= 2.0 + 1e-12
            r3_pos.append((r / 2.0) ** 3)
            dirs.append(d_p / r)
        elif m == 1:
            assert np.array_equal(new[:3], cur[:3]) and np.array_equal(th1, th0)
            dot = min(1.0, abs(float(np.dot(new[3:7], cur[3:7]))) / np.linalg.norm(new[3:7]) / np.linalg.norm(cur[3:7]))
            angle = 2.0 * math.acos(dot)
            assert angle <= k_rot + 1e-7
            r3_rot.append((angle / k_rot) ** 3)
        else:
            t = m - 2
            assert np.array_equal(new[:7], cur[:7])
            assert np.array_equal(np.delete(th1, t), np.delete(th0, t))
            assert -math.pi < th1[t] <= math.pi
    counts = np.bincount(modes, minlength=2 + lig.T)
    assert len(counts) == 2 + lig.T
    expected = n / (2 + lig.T)
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 20.5  # 5 degrees of freedom: p ~ 1e-3
    # |ball point|^3 is uniform on [0, 1] for a point uniform in the ball; directions isotropic
    for r3 in (np.array(r3_pos), np.array(r3_rot)):
        assert abs(r3.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(r3))
    assert np.linalg.norm(np.mean(dirs, axis=0)) < 4 * math.sqrt(1 / 3 / len(dirs))
