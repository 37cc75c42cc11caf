"""Redocking through the host API (the paper's accuracy measure: the top pose
within 2 A heavy-atom RMSD of the crystal pose).  Sanity, not parity: each
synthetic ligand gets a receptor shell built around its own pose (atoms 4.2 A
from its atoms, none closer than 3.8 A to any of them), so the pose it was
built around is the deepest minimum; 256 chains x 30 Monte Carlo steps of BFGS
start from random poses in a 16 A box and must find it."""
import numpy as np
import pytest

from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402

CASES = [(12, 2, 3), (18, 4, 5), (24, 6, 6), (30, 8, 7)]  # (atoms, torsions, seed)


def _shell(xyz, seed):
    rng = np.random.default_rng(seed)
    pts = []
    for x in xyz:
        for _ in range(14):
            d = rng.normal(size=3)
            pts.append(x + 4.2 * d / np.linalg.norm(d))
    pts = np.array(pts)
    keep = np.min(np.linalg.norm(pts[:, None] - xyz[None], axis=-1), axis=1) > 3.8
    pts = pts[keep]
    # thin the shell to at most one atom per 2.8 A
    out = []
    for p in pts:
        if all(np.linalg.norm(p - q) >= 2.8 for q in out):
            out.append(p)
    return np.array(out, dtype=np.float32)


@pytest.mark.parametrize("dtype", [dsdp.DSDP_MAP_F32, dsdp.DSDP_MAP_BF16])
def test_redocking_recovers_the_crystal_pose(dtype):
    ctx = dsdp.dsdp_create(0)
    rmsds = []
    try:
        for n, t, seed in CASES:
            lig = synth.ligand(n, t, seed)
            xyz = lig.xyz.astype(np.float64)
            rec_xyz = _shell(xyz, seed)
            rec_t = np.zeros(len(rec_xyz), dtype=np.uint8)  # C_H: attractive at contact
            center = xyz.mean(axis=0)
            grid = dsdp.dsdp_grid_build(ctx, rec_xyz, rec_t, dsdp.make_box(center, 16.0, 0.375), dtype)
            try:
                params = dsdp.make_params(n_chains=256, n_mc_steps=30, n_opt_iters=100, seed=seed, top_k=3)
                jid = dsdp.dsdp_dock_submit(ctx, grid, lig, params)
                r = dsdp.dsdp_dock_poll(ctx, jid, dsdp.result_buffers(n, t, params), wait_ms=-1)
            finally:
                dsdp.dsdp_grid_free(ctx, grid)
            top = r["coords"][0].astype(np.float64)
            rmsds.append(float(np.sqrt(((top - xyz) ** 2).sum(-1).mean())))
    finally:
        dsdp.dsdp_destroy(ctx)
    print(f"maps {['f32', 'bf16', 'f16'][dtype]}: top-1 RMSD to the crystal pose per ligand "
          f"{[round(x, 3) for x in rmsds]} A")
    assert sum(x < 2.0 for x in rmsds) == len(CASES), rmsds
