"""Thin ctypes binding of libdsdp (include/dsdp.h): the same names, argument
marshalling only.  Every step of the docking path runs in the library's CUDA
kernels; nothing here computes.

Importing this module loads ``_build/libdsdp.so`` and raises ImportError if it
is missing: there is no CPU fallback.  Build it with
``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_2303_09916_gb300/build.py``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdsdp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdsdp.so not built ({LIB_PATH}); run paper_2303_09916_gb300/build.py")
_lib = C.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants
DSDP_OK, DSDP_PENDING = 0, 1
DSDP_ERR_INVALID_ARG, DSDP_ERR_OUT_OF_MEMORY, DSDP_ERR_NOT_FOUND = -1, -2, -3
DSDP_ERR_TIMEOUT, DSDP_ERR_CANCELLED, DSDP_ERR_DEVICE, DSDP_ERR_INTERNAL = -4, -5, -6, -7
DSDP_MAP_F32, DSDP_MAP_BF16, DSDP_MAP_F16 = 0, 1, 2
DSDP_GRID_EQ4, DSDP_GRID_EQ3 = 0, 1
DSDP_OPT_BFGS, DSDP_OPT_BB = 0, 1
DSDP_TERM_INTER, DSDP_TERM_INTRA, DSDP_TERM_ALL, DSDP_TERM_NORMALISED = 1, 2, 3, 4
DSDP_PLAN_PERSISTENT, DSDP_PLAN_NO_RESCORE = 1, 2
DSDP_STAGE_CHAINS, DSDP_STAGE_RESCORE, DSDP_STAGE_ALL = 1, 2, 3
DSDP_NUM_MAP_TYPES = 8
DSDP_MAX_LIGAND_ATOMS, DSDP_MAX_TORSIONS, DSDP_MAX_CHAINS, DSDP_MAX_TOP_K = 64, 15, 8192, 64
DSDP_NOALLOC_MAX_CHAINS, DSDP_NOALLOC_SCRATCH_BYTES = 1024, 1600000


class DSDPError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{dsdp_status_string(status)}: {message}")
        self.status = status


# ------------------------------------------------------------------ structs
class dsdp_receptor(C.Structure):
    _fields_ = [("n", C.c_int32), ("xyz", C.c_void_p), ("xs_type", C.c_void_p)]


class dsdp_box(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("size", C.c_double * 3), ("spacing", C.c_double)]


class dsdp_ligand(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("xyz", C.c_void_p), ("xs_type", C.c_void_p), ("n_bonds", C.c_int32),
                ("bonds", C.c_void_p), ("rotatable", C.c_void_p)]


class dsdp_dock_params(C.Structure):
    _fields_ = [("n_chains", C.c_int32), ("n_mc_steps", C.c_int32), ("n_opt_iters", C.c_int32),
                ("optimizer", C.c_int32), ("temperature", C.c_double), ("seed", C.c_uint64), ("top_k", C.c_int32),
                ("rmsd_dedup", C.c_double), ("trace", C.c_int32), ("site_radius", C.c_float),
                ("n_site_points", C.c_int32), ("reserved0", C.c_int32), ("site_points", C.c_void_p),
                ("reserved", C.c_int32 * 2)]


class dsdp_dock_result(C.Structure):
    _fields_ = [("capacity", C.c_int32), ("n_out", C.c_int32), ("n_atoms", C.c_int32), ("n_torsions", C.c_int32),
                ("score", C.c_void_p), ("inter", C.c_void_p), ("intra", C.c_void_p), ("conf", C.c_void_p),
                ("coords", C.c_void_p), ("chain", C.c_void_p), ("chain_best_e", C.c_void_p),
                ("chain_best_conf", C.c_void_p), ("trace", C.c_void_p), ("n_evals", C.c_uint64),
                ("device_ms", C.c_double), ("latency_ms", C.c_double)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class dsdp_create_params(C.Structure):
    _fields_ = [("device", C.c_int32), ("mem_budget_bytes", C.c_uint64), ("n_streams", C.c_int32),
                ("max_inflight_jobs", C.c_int32), ("alloc", _ALLOC), ("free", _FREE), ("alloc_user", C.c_void_p),
                ("max_batch_chains", C.c_int32), ("stream", C.c_void_p)]


class dsdp_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("cancelled", C.c_uint64), ("queued", C.c_int32), ("running", C.c_int32),
                ("bytes_in_use", C.c_uint64), ("bytes_budget", C.c_uint64), ("batches", C.c_uint64)]


class dsdp_grid_view(C.Structure):
    _fields_ = [("d_maps", C.c_void_p), ("n", C.c_int32 * 3), ("origin", C.c_double * 3), ("spacing", C.c_double),
                ("dtype", C.c_int32), ("mode", C.c_int32)]


class dsdp_job_device(C.Structure):
    _fields_ = [("grid", dsdp_grid_view), ("receptor", dsdp_receptor), ("h_blob", C.c_void_p),
                ("d_blob", C.c_void_p), ("params", dsdp_dock_params), ("box_lo", C.c_double * 3),
                ("box_size", C.c_double * 3), ("d_chain_best_conf", C.c_void_p), ("d_chain_best_e", C.c_void_p),
                ("d_chain_evals", C.c_void_p), ("d_trace", C.c_void_p), ("d_out_n", C.c_void_p),
                ("d_out_chain", C.c_void_p), ("d_out_score", C.c_void_p), ("d_out_inter", C.c_void_p),
                ("d_out_intra", C.c_void_p), ("d_out_conf", C.c_void_p), ("d_out_coords", C.c_void_p),
                ("d_site_points", C.c_void_p)]


P = C.POINTER
_sig = {
    "dsdp_status_string": (C.c_char_p, [C.c_int32]),
    "dsdp_last_error": (C.c_char_p, []),
    "dsdp_version": (C.c_char_p, []),
    "dsdp_create": (C.c_int32, [P(dsdp_create_params), P(C.c_void_p)]),
    "dsdp_destroy": (C.c_int32, [C.c_void_p]),
    "dsdp_grid_build": (C.c_int32, [C.c_void_p, P(dsdp_receptor), P(dsdp_box), C.c_int, C.c_int, P(C.c_void_p)]),
    "dsdp_grid_from_maps": (C.c_int32, [C.c_void_p, P(dsdp_receptor), P(dsdp_box), C.c_int, C.c_int, C.c_void_p,
                                        P(C.c_void_p)]),
    "dsdp_grid_download": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "dsdp_grid_info": (C.c_int32, [C.c_void_p, P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_uint64)]),
    "dsdp_grid_free": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "dsdp_score_eval": (C.c_int32, [C.c_void_p, C.c_void_p, P(dsdp_ligand), C.c_void_p, C.c_int32, C.c_void_p,
                                    C.c_void_p, C.c_uint32]),
    "dsdp_dock_submit": (C.c_int32, [C.c_void_p, C.c_void_p, P(dsdp_ligand), P(dsdp_dock_params),
                                     P(C.c_uint64)]),
    "dsdp_dock_submit_many": (C.c_int32, [C.c_void_p, C.c_int32, P(C.c_void_p), P(dsdp_ligand), P(dsdp_dock_params),
                                          P(C.c_uint64)]),
    "dsdp_dock_poll": (C.c_int32, [C.c_void_p, C.c_uint64, P(dsdp_dock_result), C.c_int32]),
    "dsdp_dock_cancel": (C.c_int32, [C.c_void_p, C.c_uint64]),
    "dsdp_get_stats": (C.c_int32, [C.c_void_p, P(dsdp_stats)]),
    "dsdp_grid_map_bytes": (C.c_uint64, [P(dsdp_box), C.c_int, C.c_int]),
    "dsdp_grid_build_device": (C.c_int32, [P(dsdp_receptor), P(dsdp_box), C.c_int, C.c_int, C.c_void_p,
                                           C.c_uint64, C.c_void_p]),
    "dsdp_ligand_pack": (C.c_int32, [P(dsdp_ligand), C.c_void_p, C.c_uint64, P(C.c_uint64)]),
    "dsdp_ligand_blob_info": (C.c_int32, [C.c_void_p, P(C.c_int32), P(C.c_int32), P(C.c_int32), P(C.c_int32)]),
    "dsdp_score_eval_device": (C.c_int32, [P(dsdp_grid_view), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p]),
    "dsdp_plan_create": (C.c_int32, [C.c_void_p, C.c_int32, P(dsdp_job_device), C.c_uint32, C.c_int32,
                                     P(C.c_void_p)]),
    "dsdp_plan_launch": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "dsdp_plan_launch_stage": (C.c_int32, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "dsdp_plan_kernel_count": (C.c_int32, [C.c_void_p]),
    "dsdp_plan_autotune": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, P(C.c_int32), P(C.c_float)]),
    "dsdp_plan_destroy": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "dsdp_gather_bench_device": (C.c_int32, [P(dsdp_grid_view), C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                             C.c_void_p, C.c_void_p]),
    "dsdp_rescore_topk_noalloc": (C.c_int32, [P(dsdp_job_device), C.c_void_p]),
    "dsdp_voxel_work_bytes": (C.c_uint64, []),
    "dsdp_voxelize_device": (C.c_int32, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_double), C.c_void_p,
                                         C.c_void_p, C.c_uint64, C.c_void_p]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = sorted(_sig)


def dsdp_status_string(s: int) -> str:
    return _lib.dsdp_status_string(int(s)).decode()


def dsdp_last_error() -> str:
    return _lib.dsdp_last_error().decode()


def dsdp_version() -> str:
    return _lib.dsdp_version().decode()


def _check(status):
    if status < 0:
        raise DSDPError(status, dsdp_last_error())
    return status


# ------------------------------------------------------------------ marshalling helpers
def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_box(center, size, spacing) -> dsdp_box:
    b = dsdp_box()
    size = np.broadcast_to(np.asarray(size, dtype=np.float64), (3,))
    for a in range(3):
        b.center[a] = float(center[a])
        b.size[a] = float(size[a])
    b.spacing = float(spacing)
    return b


class _Keep:
    """Holds numpy arrays alive while a struct points into them."""

    def __init__(self, struct, *arrays):
        self.struct = struct
        self.arrays = arrays


def make_receptor(xyz, xs_type):
    xyz = _np(xyz, np.float32).reshape(-1, 3)
    t = _np(xs_type, np.uint8)
    r = dsdp_receptor(len(t), xyz.ctypes.data, t.ctypes.data)
    return _Keep(r, xyz, t)


def make_ligand(lig):
    """lig: object with xyz (n, 3), xs_type (n,), bonds (m, 2), rotatable (m,)."""
    xyz = _np(lig.xyz, np.float32).reshape(-1, 3)
    t = _np(lig.xs_type, np.uint8)
    bonds = _np(lig.bonds, np.int32).reshape(-1, 2)
    rot = _np(lig.rotatable, np.uint8)
    s = dsdp_ligand(len(t), xyz.ctypes.data, t.ctypes.data, len(rot), bonds.ctypes.data if len(rot) else None,
                    rot.ctypes.data if len(rot) else None)
    return _Keep(s, xyz, t, bonds, rot)


def make_params(n_chains=0, n_mc_steps=0, n_opt_iters=0, optimizer=DSDP_OPT_BFGS, temperature=0.0, seed=0,
                top_k=0, rmsd_dedup=0.0, trace=0, site_points=None, site_radius=0.0) -> dsdp_dock_params:
    """Dock parameters; site_points ([n][3] float32, host) selects the adaptive search space."""
    p = dsdp_dock_params(int(n_chains), int(n_mc_steps), int(n_opt_iters), int(optimizer), float(temperature),
                         int(seed), int(top_k), float(rmsd_dedup), int(trace), float(site_radius))
    if site_points is not None and len(site_points):
        pts = np.ascontiguousarray(site_points, dtype=np.float32).reshape(-1, 3)
        p.n_site_points = len(pts)
        p.site_points = pts.ctypes.data
        p._keep_sites = pts  # alive as long as the params
    return p


# ------------------------------------------------------------------ context / grids
def dsdp_create(device=0, mem_budget_bytes=0, n_streams=0, max_inflight_jobs=0, max_batch_chains=0, stream=None):
    """stream: a cudaStream_t (int) for the context's synchronous work, e.g. torch.cuda.Stream().cuda_stream."""
    p = dsdp_create_params(int(device), int(mem_budget_bytes), int(n_streams), int(max_inflight_jobs))
    p.max_batch_chains = int(max_batch_chains)
    p.stream = stream
    out = C.c_void_p()
    _check(_lib.dsdp_create(C.byref(p), C.byref(out)))
    return out.value


def dsdp_destroy(ctx):
    _check(_lib.dsdp_destroy(ctx))


def dsdp_grid_build(ctx, rec_xyz, rec_type, box: dsdp_box, dtype=DSDP_MAP_F32, mode=DSDP_GRID_EQ4):
    r = make_receptor(rec_xyz, rec_type)
    out = C.c_void_p()
    _check(_lib.dsdp_grid_build(ctx, C.byref(r.struct), C.byref(box), int(dtype), int(mode), C.byref(out)))
    return out.value


def dsdp_grid_from_maps(ctx, rec_xyz, rec_type, box: dsdp_box, dtype, mode, maps):
    m = _np(maps, np.float32)
    out = C.c_void_p()
    if rec_xyz is None:
        _check(_lib.dsdp_grid_from_maps(ctx, None, C.byref(box), int(dtype), int(mode), m.ctypes.data, C.byref(out)))
    else:
        r = make_receptor(rec_xyz, rec_type)
        _check(_lib.dsdp_grid_from_maps(ctx, C.byref(r.struct), C.byref(box), int(dtype), int(mode), m.ctypes.data,
                                        C.byref(out)))
    return out.value


def dsdp_grid_info(grid):
    n = (C.c_int32 * 3)()
    o = (C.c_double * 3)()
    h = C.c_double()
    b = C.c_uint64()
    _check(_lib.dsdp_grid_info(grid, n, o, C.byref(h), C.byref(b)))
    return dict(n=list(n), origin=list(o), spacing=h.value, map_bytes=b.value)


def dsdp_grid_download(ctx, grid, mode=DSDP_GRID_EQ4):
    info = dsdp_grid_info(grid)
    nx, ny, nz = info["n"]
    ch = 4 if mode == DSDP_GRID_EQ4 else 1
    out = np.zeros((DSDP_NUM_MAP_TYPES, nz, ny, nx, ch), dtype=np.float32)
    _check(_lib.dsdp_grid_download(ctx, grid, out.ctypes.data, out.size))
    return out


def dsdp_grid_free(ctx, grid):
    _check(_lib.dsdp_grid_free(ctx, grid))


def dsdp_grid_map_bytes(box: dsdp_box, dtype=DSDP_MAP_F32, mode=DSDP_GRID_EQ4) -> int:
    return int(_lib.dsdp_grid_map_bytes(C.byref(box), int(dtype), int(mode)))


# ------------------------------------------------------------------ scoring / docking (host arrays)
def dsdp_score_eval(ctx, grid, ligand, conf, flags=DSDP_TERM_ALL):
    lig = make_ligand(ligand)
    conf = _np(conf, np.float64)
    n = conf.shape[0]
    T = conf.shape[1] - 7
    e = np.zeros(n)
    g = np.zeros((n, 6 + T))
    _check(_lib.dsdp_score_eval(ctx, grid, C.byref(lig.struct), conf.ctypes.data, n, e.ctypes.data, g.ctypes.data,
                                int(flags)))
    return e, g


def dsdp_dock_submit(ctx, grid, ligand, params: dsdp_dock_params) -> int:
    lig = make_ligand(ligand)
    jid = C.c_uint64()
    _check(_lib.dsdp_dock_submit(ctx, grid, C.byref(lig.struct), C.byref(params), C.byref(jid)))
    return jid.value


def dsdp_dock_submit_many(ctx, grids, ligands, params) -> list:
    """Submit len(ligands) jobs at once (grids[i], ligands[i], params[i]); the job ids."""
    n = len(ligands)
    if len(grids) != n or len(params) != n:
        raise ValueError("grids, ligands and params differ in length")
    keep = [make_ligand(l) for l in ligands]
    g_arr = (C.c_void_p * max(n, 1))(*grids)
    l_arr = (dsdp_ligand * max(n, 1))(*[k.struct for k in keep])
    p_arr = (dsdp_dock_params * max(n, 1))(*params)
    ids = (C.c_uint64 * max(n, 1))()
    _check(_lib.dsdp_dock_submit_many(ctx, n, g_arr, l_arr, p_arr, ids))
    return [ids[i] for i in range(n)]


class DockResult(dict):
    pass


def result_buffers(n_atoms, n_torsions, params: dsdp_dock_params, chains=True):
    k = params.top_k or 9
    nc = params.n_chains or 384
    nx = 7 + n_torsions
    bufs = dict(score=np.zeros(k), inter=np.zeros(k), intra=np.zeros(k), conf=np.zeros((k, nx)),
                coords=np.zeros((k, n_atoms, 3), dtype=np.float32), chain=np.zeros(k, dtype=np.int32))
    if chains:
        bufs["chain_best_e"] = np.zeros(nc, dtype=np.float32)
        bufs["chain_best_conf"] = np.zeros((nc, nx), dtype=np.float32)
    if params.trace:
        bufs["trace"] = np.zeros((nc, (params.n_mc_steps or 40) + 1, nx + 4), dtype=np.float32)
    return bufs


def dsdp_dock_poll(ctx, job_id, bufs: dict, wait_ms=-1):
    """Fills `bufs` (from result_buffers) and returns a dict; None while pending
    (wait_ms = 0); a positive wait that expires raises DSDPError (DSDP_ERR_TIMEOUT)."""
    r = dsdp_dock_result()
    r.capacity = len(bufs["score"])
    for key in ("score", "inter", "intra", "conf", "coords", "chain", "chain_best_e", "chain_best_conf", "trace"):
        if key in bufs:
            setattr(r, key, bufs[key].ctypes.data)
    s = _lib.dsdp_dock_poll(ctx, int(job_id), C.byref(r), int(wait_ms))
    if s == DSDP_PENDING:
        return None
    _check(s)
    out = DockResult({k: (v[: r.n_out] if k in ("score", "inter", "intra", "conf", "coords", "chain") else v)
                      for k, v in bufs.items()})
    out.update(n_out=r.n_out, n_evals=int(r.n_evals), device_ms=r.device_ms, latency_ms=r.latency_ms,
               n_atoms=r.n_atoms, n_torsions=r.n_torsions)
    return out


def dsdp_dock_cancel(ctx, job_id) -> int:
    return _check(_lib.dsdp_dock_cancel(ctx, int(job_id)))


def dsdp_get_stats(ctx) -> dict:
    s = dsdp_stats()
    _check(_lib.dsdp_get_stats(ctx, C.byref(s)))
    return {f: getattr(s, f) for f, _ in dsdp_stats._fields_}


# ------------------------------------------------------------------ device-resident path
def dsdp_ligand_pack(ligand) -> np.ndarray:
    lig = make_ligand(ligand)
    n = C.c_uint64()
    _check(_lib.dsdp_ligand_pack(C.byref(lig.struct), None, 0, C.byref(n)))
    blob = np.zeros(n.value, dtype=np.uint8)
    _check(_lib.dsdp_ligand_pack(C.byref(lig.struct), blob.ctypes.data, n.value, C.byref(n)))
    return blob


def dsdp_ligand_blob_info(blob):
    v = [C.c_int32() for _ in range(4)]
    _check(_lib.dsdp_ligand_blob_info(_np(blob, np.uint8).ctypes.data, *[C.byref(x) for x in v]))
    return dict(n_atoms=v[0].value, n_torsions=v[1].value, n_pairs=v[2].value, n_bodies=v[3].value)


def grid_view(d_maps: int, n, origin, spacing, dtype=DSDP_MAP_F32, mode=DSDP_GRID_EQ4) -> dsdp_grid_view:
    v = dsdp_grid_view()
    v.d_maps = int(d_maps)
    for a in range(3):
        v.n[a] = int(n[a])
        v.origin[a] = float(origin[a])
    v.spacing = float(spacing)
    v.dtype = int(dtype)
    v.mode = int(mode)
    return v


def dsdp_grid_build_device(n_rec, d_xyz: int, d_type: int, box: dsdp_box, dtype, mode, d_maps: int,
                           maps_bytes: int, stream: int = 0):
    r = dsdp_receptor(int(n_rec), int(d_xyz), int(d_type))
    _check(_lib.dsdp_grid_build_device(C.byref(r), C.byref(box), int(dtype), int(mode), int(d_maps),
                                       int(maps_bytes), stream or None))


def dsdp_score_eval_device(view: dsdp_grid_view, h_blob, d_blob: int, d_conf: int, n_conf: int, d_energy: int,
                           d_grad: int, flags=DSDP_TERM_ALL, stream: int = 0):
    hb = _np(h_blob, np.uint8)
    _check(_lib.dsdp_score_eval_device(C.byref(view), hb.ctypes.data, int(d_blob), int(d_conf), int(n_conf),
                                       int(d_energy), int(d_grad) or None, int(flags), stream or None))


def dsdp_plan_create(ctx, jobs, flags=0, tile_config=0):
    arr = (dsdp_job_device * len(jobs))(*jobs)
    out = C.c_void_p()
    _check(_lib.dsdp_plan_create(ctx, len(jobs), arr, int(flags), int(tile_config), C.byref(out)))
    return out.value


def dsdp_plan_autotune(plan, stream: int = 0, repeats: int = 1, with_times: bool = False):
    """The chosen configuration (1 + variant + 4 log2 W + 12 persistent); with
    with_times also {configuration: ms per chain launch} of every one measured."""
    chosen = C.c_int32()
    ms = (C.c_float * 24)()
    _check(_lib.dsdp_plan_autotune(plan, stream or None, int(repeats), C.byref(chosen), ms))
    if not with_times:
        return chosen.value
    return chosen.value, {k + 1: float(ms[k]) for k in range(24) if ms[k] >= 0}


def dsdp_plan_launch(plan, stream: int = 0):
    _check(_lib.dsdp_plan_launch(plan, stream or None))


def dsdp_plan_launch_stage(plan, stages, stream: int = 0):
    _check(_lib.dsdp_plan_launch_stage(plan, int(stages), stream or None))


def dsdp_plan_kernel_count(plan) -> int:
    return int(_lib.dsdp_plan_kernel_count(plan))


def dsdp_plan_destroy(ctx, plan):
    _check(_lib.dsdp_plan_destroy(ctx, plan))


def dsdp_gather_bench_device(view: dsdp_grid_view, d_points: int, d_types: int, n_points: int, repeats: int,
                             d_out: int, stream: int = 0):
    _check(_lib.dsdp_gather_bench_device(C.byref(view), int(d_points), int(d_types), int(n_points), int(repeats),
                                         int(d_out), stream or None))


DSDP_VOXEL_N, DSDP_VOXEL_FEATURES, DSDP_VOXEL_CHANNELS = 36, 17, 18


def dsdp_voxel_work_bytes() -> int:
    return int(_lib.dsdp_voxel_work_bytes())


def dsdp_voxelize_device(n_atoms: int, d_xyz: int, d_radius: int, d_features: int, center, d_out: int, d_work: int,
                         work_bytes: int, stream: int = 0):
    """Receptor voxel features [36][36][36][18] into d_out (see include/dsdp.h)."""
    c = (C.c_double * 3)(*[float(v) for v in center])
    _check(_lib.dsdp_voxelize_device(int(n_atoms), int(d_xyz) or None, int(d_radius) or None, int(d_features) or None,
                                     c, int(d_out) or None, int(d_work) or None, int(work_bytes), stream or None))


def dsdp_rescore_topk_noalloc(job: dsdp_job_device, stream: int = 0):
    """FP64 rescoring + top-k of one job with no device allocation (see include/dsdp.h)."""
    _check(_lib.dsdp_rescore_topk_noalloc(C.byref(job), stream or None))
