"""FP64 CPU oracle of the DSDP docking hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product (``paper_2303_09916_gb300``)
never imports it and shares no code with it.

The arithmetic lives in ``dsdp_oracle.cpp`` (plain C++17, FP64, compiled with
``-ffp-contract=off`` so x86 and Arm hosts round identically); this module only
builds it and marshals numpy arrays through ctypes.  Parity status of every
function is written next to it in the C++ source; in short:

* pair score, grid maps, interpolation (Eq. 1-4), kinematics and gradient,
  BFGS / Barzilai-Borwein on test objectives, Philox4x32-10, rescoring: pinned
  by the ``-m "not gpu"`` tests;
* Vina constants, MC mutation rules, BFGS/BB constants: parity unpinned against
  the paper (it does not print them; they are the stated Vina reading).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsdp_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdsdp_oracle.so")
_lock = threading.Lock()
_lib = None

N_MAP_TYPES = 8
XS_NAMES = ["C_H", "C_P", "N_P", "N_D", "N_A", "O_A", "O_DA", "S_P", "N_DA"]

# [max_iters, c1, shrink, max_trials, min_curvature, bb_alpha0, bb_alpha_min, bb_alpha_max, step_scale,
#  grad_perturb].  Sensitivity probes for the tests (not part of the method): step_scale multiplies every
# step the optimisers take (1: exact); grad_perturb adds delta |g|_inf p_i to every gradient (0: exact).
DEFAULT_OPT = dict(max_iters=100, c1=1e-4, shrink=0.5, max_trials=10, min_curvature=1e-10,
                   bb_alpha0=1e-3, bb_alpha_min=1e-4, bb_alpha_max=0.1, step_scale=1.0, grad_perturb=0.0)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, no GPU needed)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        dp, ip = P(d), P(i)
        u32p = P(ctypes.c_uint32)
        sig = {
            "orc_pair": (None, [i, i, d, dp, dp]),
            "orc_constants": (None, [dp]),
            "orc_grid_dims": (None, [dp, d, ip]),
            "orc_receptor_field": (None, [i, dp, ip, i, i, dp, d, dp]),
            "orc_grid_build": (None, [i, dp, ip, dp, dp, d, d, i, dp]),
            "orc_receptor_field_abs": (None, [i, dp, ip, i, i, dp, d, dp]),
            "orc_interpolate": (None, [dp, ip, dp, d, i, i, i, dp, dp, dp]),
            "orc_ligand_new": (vp, [i, dp, ip, i, ip, ip]),
            "orc_ligand_free": (None, [vp]),
            "orc_ligand_info": (None, [vp, ip, dp]),
            "orc_ligand_pairs": (None, [vp, ip]),
            "orc_ligand_bodies": (None, [vp, ip, ip, ip]),
            "orc_ligand_coords": (None, [vp, dp, dp]),
            "orc_score_grid": (None, [vp, dp, ip, dp, d, i, dp, i, dp, dp]),
            "orc_score_exact": (None, [vp, i, dp, ip, dp, i, dp, dp]),
            "orc_apply_step": (None, [vp, dp, dp]),
            "orc_local_opt": (None, [vp, dp, ip, dp, d, i, i, dp, dp, dp]),
            "orc_opt_test": (None, [i, i, i, dp, dp, dp, dp, dp]),
            "orc_opt_test_log": (None, [i, i, i, dp, dp, dp, dp, dp, dp, i, ip]),
            "orc_local_opt_log": (None, [vp, dp, ip, dp, d, i, i, dp, dp, dp, dp, i, ip]),
            "orc_mc_step_log": (None, [vp, dp, ip, dp, d, i, dp, dp, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, dp, dp, dp, dp, i, ip]),
            "orc_bfgs_update": (None, [i, dp, dp, dp]),
            "orc_philox": (None, [u32p, u32p, u32p]),
            "orc_unit_ball": (None, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, dp]),
            "orc_chain_init": (None, [vp, dp, dp, ctypes.c_uint64, ctypes.c_uint32, dp]),
            "orc_run_chain": (None, [vp, dp, ip, dp, d, i, dp, dp, ctypes.c_uint64, ctypes.c_uint32, dp, dp, dp, dp]),
            "orc_mc_step": (None, [vp, dp, ip, dp, d, i, dp, dp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   dp, dp, dp]),
            "orc_dock": (None, [vp, dp, ip, dp, d, i, dp, dp, ctypes.c_uint64, i, i, i, dp, dp, dp]),
            "orc_rescore_topk": (i, [vp, i, dp, ip, i, dp, i, d, dp, ip, dp]),
            "orc_sas_directions": (i, [P(ctypes.c_float)]),
            "orc_sas_exposed": (None, [i, P(ctypes.c_float), P(ctypes.c_float), ip]),
            "orc_voxelize": (i, [i, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float), dp,
                                 P(ctypes.c_float)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _opt_array(opt=None):
    o = dict(DEFAULT_OPT)
    if opt:
        o.update(opt)
    return np.array([o["max_iters"], o["c1"], o["shrink"], o["max_trials"], o["min_curvature"],
                     o["bb_alpha0"], o["bb_alpha_min"], o["bb_alpha_max"], o["step_scale"], o["grad_perturb"]],
                    dtype=np.float64)


def constants():
    out = np.zeros(8)
    lib().orc_constants(_d(out)[1])
    keys = ["w_gauss1", "w_gauss2", "w_repulsion", "w_hydrophobic", "w_hbond", "w_rot", "cutoff", "wall_slope"]
    return dict(zip(keys, out.tolist()))


def pair(ti: int, tj: int, r: float):
    e, de = ctypes.c_double(), ctypes.c_double()
    lib().orc_pair(int(ti), int(tj), float(r), ctypes.byref(e), ctypes.byref(de))
    return e.value, de.value


def grid_dims(size, h):
    size, sp = _d(size)
    n = np.zeros(3, dtype=np.int32)
    lib().orc_grid_dims(sp, float(h), _i(n)[1])
    return n


class Grid:
    """FP64 maps [K][nz][ny][nx][4] with geometry (n, origin, h)."""

    def __init__(self, maps, n, origin, h):
        self.maps = np.ascontiguousarray(maps, dtype=np.float64)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.origin = np.ascontiguousarray(origin, dtype=np.float64)
        self.h = float(h)

    def cargs(self):
        return (self.maps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                self.origin.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.h)


def receptor_field(rec_xyz, rec_type, t, pts, cutoff=8.0):
    rx, rxp = _d(rec_xyz)
    rt, rtp = _i(rec_type)
    p, pp = _d(pts)
    out = np.zeros((len(p), 4))
    lib().orc_receptor_field(len(rt), rxp, rtp, int(t), len(p), pp, float(cutoff), _d(out)[1])
    return out


def receptor_field_abs(rec_xyz, rec_type, t, pts, cutoff=8.0):
    """(sum |f|, sum |df/dr|) over the receptor atoms within the cutoff, per point."""
    rx, rxp = _d(rec_xyz)
    rt, rtp = _i(rec_type)
    p, pp = _d(pts)
    out = np.zeros((len(p), 2))
    lib().orc_receptor_field_abs(len(rt), rxp, rtp, int(t), len(p), pp, float(cutoff), _d(out)[1])
    return out


def grid_build(rec_xyz, rec_type, center, size, h, cutoff=8.0, n_threads=None) -> Grid:
    n = grid_dims(size, h)
    rx, rxp = _d(rec_xyz)
    rt, rtp = _i(rec_type)
    c, cp = _d(center)
    s, sp = _d(size)
    maps = np.zeros((N_MAP_TYPES, n[2], n[1], n[0], 4))
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    lib().orc_grid_build(len(rt), rxp, rtp, cp, sp, float(h), float(cutoff), int(n_threads), _d(maps)[1])
    origin = c - (n - 1) * h / 2.0
    return Grid(maps, n, origin, h)


def interpolate(grid: Grid, mode: int, t: int, pts):
    p, pp = _d(pts)
    e = np.zeros(len(p))
    g = np.zeros((len(p), 3))
    m, n, o, h = grid.cargs()
    lib().orc_interpolate(m, n, o, h, int(mode), int(t), len(p), pp, _d(e)[1], _d(g)[1])
    return e, g


class Ligand:
    def __init__(self, xyz, types, bonds, rotatable):
        self._xyz, xp = _d(xyz)
        self._types, tp = _i(types)
        self._bonds, bp = _i(np.asarray(bonds, dtype=np.int32).reshape(-1))
        self._rot, rp = _i(rotatable)
        self.h = lib().orc_ligand_new(len(self._types), xp, tp, len(self._rot), bp, rp)
        if not self.h:
            raise ValueError("oracle rejected the ligand topology")
        info = np.zeros(6, dtype=np.int32)
        gr = ctypes.c_double()
        lib().orc_ligand_info(self.h, _i(info)[1], ctypes.byref(gr))
        (self.n_atoms, self.T, self.n_bodies, self.root_body, self.root_atom, self.n_pairs) = [int(v) for v in info]
        self.gyration_radius = gr.value

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_ligand_free(h)
            self.h = None

    @property
    def nx(self):
        return 7 + self.T

    @property
    def nd(self):
        return 6 + self.T

    def pairs(self):
        out = np.zeros((self.n_pairs, 2), dtype=np.int32)
        lib().orc_ligand_pairs(self.h, _i(out)[1])
        return out

    def bodies(self):
        body_of = np.zeros(self.n_atoms, dtype=np.int32)
        parent = np.zeros(self.n_bodies, dtype=np.int32)
        tb = np.zeros(max(self.T, 1), dtype=np.int32)
        lib().orc_ligand_bodies(self.h, _i(body_of)[1], _i(parent)[1], _i(tb)[1])
        return body_of, parent, tb[: self.T]

    def identity_conf(self):
        c = np.zeros(self.nx)
        c[:3] = self._xyz.reshape(-1, 3)[self.root_atom]
        c[3] = 1.0
        return c

    def coords(self, conf):
        c, cp = _d(conf)
        out = np.zeros((self.n_atoms, 3))
        lib().orc_ligand_coords(self.h, cp, _d(out)[1])
        return out

    def score_grid(self, grid: Grid, mode: int, conf, flags: int = 3):
        c, cp = _d(conf)
        terms = np.zeros(2)
        grad = np.zeros(self.nd)
        m, n, o, h = grid.cargs()
        lib().orc_score_grid(self.h, m, n, o, h, int(mode), cp, int(flags), _d(terms)[1], _d(grad)[1])
        return terms, grad

    def score_exact(self, rec_xyz, rec_type, conf, flags: int = 3):
        rx, rxp = _d(rec_xyz)
        rt, rtp = _i(rec_type)
        c, cp = _d(conf)
        terms = np.zeros(2)
        grad = np.zeros(self.nd)
        lib().orc_score_exact(self.h, len(rt), rxp, rtp, cp, int(flags), _d(terms)[1], _d(grad)[1])
        return terms, grad

    def apply_step(self, conf, step):
        c = np.array(conf, dtype=np.float64)
        s, sp = _d(step)
        lib().orc_apply_step(self.h, _d(c)[1], sp)
        return c

    def local_opt(self, grid: Grid, mode: int, optimizer: int, conf, opt=None, log=False):
        """Returns (conf, E, evals, iters), plus the decisions taken (Decisions) when log."""
        c = np.array(conf, dtype=np.float64)
        o, op = _d(_opt_array(opt))
        out = np.zeros(3)
        m, n, og, h = grid.cargs()
        if not log:
            lib().orc_local_opt(self.h, m, n, og, h, int(mode), int(optimizer), op, _d(c)[1], _d(out)[1])
            return c, out[0], int(out[1]), int(out[2])
        buf, cnt = _log_buffer(o)
        lib().orc_local_opt_log(self.h, m, n, og, h, int(mode), int(optimizer), op, _d(c)[1], _d(out)[1],
                                _d(buf)[1], len(buf), ctypes.byref(cnt))
        return c, out[0], int(out[1]), int(out[2]), Decisions(buf, cnt.value)


DECISION_KINDS = {0: "armijo", 1: "bb_best", 2: "metropolis", 3: "bfgs_curvature", 4: "bb_curvature",
                  5: "eq3_cell_face"}


class Decisions:
    """Decisions a local optimisation or MC step took, in order: kind (see
    DECISION_KINDS), margin (the quantity whose sign picks the branch) and scale
    (|s|_1 (|g|_inf + |g'|_inf) for the curvature tests, else 0)."""

    def __init__(self, buf, count):
        if count > len(buf):
            raise RuntimeError(f"decision log overflow: {count} > {len(buf)}")
        self.kind = buf[:count, 0].astype(np.int32)
        self.margin = buf[:count, 1].copy()
        self.scale = buf[:count, 2].copy()

    def __len__(self):
        return len(self.kind)

    def taken(self):
        """The branch of each decision: True for accept / update / new best."""
        return np.where((self.kind == 0), self.margin <= 0,
                        np.where((self.kind == 1) | (self.kind == 2), self.margin < 0,
                                 np.where(self.kind == 5, True, self.margin > 0)))


def _log_buffer(opt_arr):
    # per local optimisation at most max_iters x (max_trials + 1) + 1 decisions and one cell-face
    # record per evaluation (Eq. 3), + 1 Metropolis
    cap = 2 * int(opt_arr[0]) * (int(opt_arr[3]) + 2) + 8
    return np.zeros((cap, 3)), ctypes.c_int()


def dock_params_array(n_mc_steps, optimizer, temperature, box_lo, box_size, sites=None, site_radius=7.0):
    """[n_mc_steps, optimizer, temperature, box_lo, box_size, site_radius, n_sites, sites...]; sites ([n][3],
    FP32-representable) select the adaptive search space for the initial positions."""
    pts = np.zeros((0, 3)) if sites is None else np.asarray(sites, dtype=np.float32).astype(np.float64).reshape(-1, 3)
    return np.array([n_mc_steps, optimizer, temperature, *box_lo, *box_size, float(np.float32(site_radius)),
                     len(pts), *pts.ravel()], dtype=np.float64)


def chain_init(lig: Ligand, dock_params, seed, chain, opt=None):
    dp, dpp = _d(dock_params)
    o, op = _d(_opt_array(opt))
    c = np.zeros(lig.nx)
    lib().orc_chain_init(lig.h, dpp, op, int(seed), int(chain), _d(c)[1])
    return c


def run_chain(lig: Ligand, grid: Grid, mode, dock_params, seed, chain, opt=None, trace=True):
    dp, dpp = _d(dock_params)
    o, op = _d(_opt_array(opt))
    S = int(dock_params[0])
    best = np.zeros(lig.nx)
    out = np.zeros(2)
    tc = np.zeros((S + 1, lig.nx)) if trace else None
    tr = np.zeros((S + 1, 5)) if trace else None
    m, n, og, h = grid.cargs()
    lib().orc_run_chain(lig.h, m, n, og, h, int(mode), dpp, op, int(seed), int(chain), _d(best)[1], _d(out)[1],
                        _d(tc)[1] if trace else None, _d(tr)[1] if trace else None)
    return dict(best=best, e_best=out[0], evals=int(out[1]), trace_conf=tc, trace_rec=tr)


def mc_step(lig: Ligand, grid: Grid, mode, dock_params, seed, chain, step, cur, e_cur, opt=None, log=False):
    """One MC step replayed from (cur, e_cur): (state, energy, record[mode, accepted,
    e_candidate, e_current, evals]), plus the decisions taken (Decisions) when log."""
    dp, dpp = _d(dock_params)
    o, op = _d(_opt_array(opt))
    c = np.array(cur, dtype=np.float64)
    e = ctypes.c_double(float(e_cur))
    rec = np.zeros(5)
    m, n, og, h = grid.cargs()
    if not log:
        lib().orc_mc_step(lig.h, m, n, og, h, int(mode), dpp, op, int(seed), int(chain), int(step), _d(c)[1],
                          ctypes.byref(e), _d(rec)[1])
        return c, e.value, rec
    buf, cnt = _log_buffer(o)
    lib().orc_mc_step_log(lig.h, m, n, og, h, int(mode), dpp, op, int(seed), int(chain), int(step), _d(c)[1],
                          ctypes.byref(e), _d(rec)[1], _d(buf)[1], len(buf), ctypes.byref(cnt))
    return c, e.value, rec, Decisions(buf, cnt.value)


def dock(lig: Ligand, grid: Grid, mode, dock_params, seed, n_chains, chain0=0, n_threads=1, opt=None):
    dp, dpp = _d(dock_params)
    o, op = _d(_opt_array(opt))
    best = np.zeros((n_chains, lig.nx))
    e_best = np.zeros(n_chains)
    evals = np.zeros(n_chains)
    m, n, og, h = grid.cargs()
    lib().orc_dock(lig.h, m, n, og, h, int(mode), dpp, op, int(seed), int(chain0), int(n_chains), int(n_threads),
                   _d(best)[1], _d(e_best)[1], _d(evals)[1])
    return best, e_best, evals


def rescore_topk(lig: Ligand, rec_xyz, rec_type, confs, k, rmsd_cut=1.0):
    """FP64 rescoring of every conformation and the top k after RMSD de-duplication.
    Returns (scores, idx, terms): scores[n] of every conformation in input order,
    idx the kept top-k input indices (best first), terms[kept, 3] their (score,
    inter, intra)."""
    rx, rxp = _d(rec_xyz)
    rt, rtp = _i(rec_type)
    c, cp = _d(confs)
    n = c.shape[0]
    scores = np.zeros(n)
    idx = np.zeros(k, dtype=np.int32)
    terms = np.zeros((k, 3))
    kept = lib().orc_rescore_topk(lig.h, len(rt), rxp, rtp, n, cp, int(k), float(rmsd_cut), _d(scores)[1],
                                  _i(idx)[1], _d(terms)[1])
    return scores, idx[:kept], terms[:kept]


def opt_test(kind, optimizer, x0, A=None, b=None, opt=None, log=False):
    x = np.array(x0, dtype=np.float64)
    n = len(x)
    A_, Ap = _d(A if A is not None else np.zeros((1,)))
    b_, bp = _d(b if b is not None else np.zeros((1,)))
    o, op = _d(_opt_array(opt))
    out = np.zeros(3)
    if not log:
        lib().orc_opt_test(int(kind), int(optimizer), n, Ap, bp, op, _d(x)[1], _d(out)[1])
        return x, out[0], int(out[1]), int(out[2])
    buf, cnt = _log_buffer(o)
    lib().orc_opt_test_log(int(kind), int(optimizer), n, Ap, bp, op, _d(x)[1], _d(out)[1], _d(buf)[1], len(buf),
                           ctypes.byref(cnt))
    return x, out[0], int(out[1]), int(out[2]), Decisions(buf, cnt.value)


def bfgs_update(H, s, y):
    Hc = np.array(H, dtype=np.float64)
    s_, sp = _d(s)
    y_, yp = _d(y)
    lib().orc_bfgs_update(len(s_), _d(Hc)[1], sp, yp)
    return Hc


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib().orc_philox(c.ctypes.data_as(P), k.ctypes.data_as(P), out.ctypes.data_as(P))
    return out


def unit_ball(seed, chain, step):
    out = np.zeros(3)
    lib().orc_unit_ball(int(seed), int(chain), int(step), _d(out)[1])
    return out


# ---------------------------------------------------------------- voxel features
VOX_N, VOX_FEATURES, VOX_CHANNELS = 36, 17, 18


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def sas_directions():
    """The 98 unit test directions of the surface test, FP32 [98][3]."""
    u = np.zeros((98, 3), dtype=np.float32)
    m = lib().orc_sas_directions(_f(u)[1])
    return u[:m]


def sas_exposed(xyz, radius):
    """Exposed solvent-accessible test points per atom (of 98)."""
    x, xp = _f(xyz)
    r, rp = _f(radius)
    out = np.zeros(len(r), dtype=np.int32)
    lib().orc_sas_exposed(len(r), xp, rp, _i(out)[1])
    return out


def voxelize(xyz, radius, features, center):
    """Voxel features [36][36][36][18] (z, y, x, channel) of a receptor and the
    number of atoms inside the 70 A cube."""
    x, xp = _f(xyz)
    r, rp = _f(radius)
    f, fp = _f(features)
    if f.shape != (len(r), VOX_FEATURES):
        raise ValueError("features must be [n][17]")
    c, cp = _d(center)
    out = np.zeros((VOX_N, VOX_N, VOX_N, VOX_CHANNELS), dtype=np.float32)
    inside = lib().orc_voxelize(len(r), xp, rp, fp, cp, _f(out)[1])
    return out, inside
