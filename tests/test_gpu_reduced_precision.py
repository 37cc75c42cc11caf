"""Grid maps stored in BF16 and FP16 (accumulation stays FP32, the final
rescoring FP64): the error of every reported score against the FP64 oracle and
against the FP32-map run, on the typical-4k grid (4,000-atom receptor, 80^3
maps) docked with 16 ligands of 30 atoms and 8 torsions (seeds 0-15), 384
chains x 40 steps each.

Reported (printed) and bounded:
* search energy of each sampled chain's best pose (grid score with the stored
  maps) against the oracle's FP64-map score of that pose: bounded by the
  storage format's rounding of the summed corner values (2^-8 relative for
  BF16, 2^-11 for FP16) on top of the FP32 tolerance;
* the final FP64 rescoring of the poses: exact against the oracle (1e-10);
* top pose against the FP32-map run: score difference and heavy-atom RMSD;
* top pose of every map format against the FP64 oracle's own search of the
  system (FP64 maps, the same Philox streams and parameters): score
  difference and heavy-atom RMSD (the chains separate chaotically, so this
  measures whether both searches reach the same best pose, not rounding).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402

from gpu_util import E_REL  # noqa: E402

BOX, H = 30.0, 0.375
UNIT_ROUNDOFF = {dsdp.DSDP_MAP_F32: 2.0 ** -24, dsdp.DSDP_MAP_BF16: 2.0 ** -8, dsdp.DSDP_MAP_F16: 2.0 ** -11}
N_LIGANDS = 16
NAMES = ["f32", "bf16", "f16"]


@pytest.fixture(scope="module")
def system():
    cfg = synth.config("typical-4k", seed=0)
    rec = cfg.receptor
    ligs = [synth.ligand(30, 8, s, center=rec.pocket_center) for s in range(N_LIGANDS)]
    oligs = [oracle.Ligand(lg.xyz.astype(np.float64), lg.xs_type, lg.bonds, lg.rotatable) for lg in ligs]
    cores = os.cpu_count() or 1
    og = oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, np.array([BOX] * 3), H,
                           n_threads=cores)
    ctx = dsdp.dsdp_create(0, max_inflight_jobs=N_LIGANDS)
    runs = {}
    try:
        for dtype in (dsdp.DSDP_MAP_F32, dsdp.DSDP_MAP_BF16, dsdp.DSDP_MAP_F16):
            grid = dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(rec.pocket_center, BOX, H), dtype)
            try:
                params = [dsdp.make_params(n_chains=384, n_mc_steps=40, n_opt_iters=100, seed=s, top_k=9)
                          for s in range(N_LIGANDS)]
                ids = dsdp.dsdp_dock_submit_many(ctx, [grid] * N_LIGANDS, ligs, params)
                runs[dtype] = [dsdp.dsdp_dock_poll(ctx, j, dsdp.result_buffers(lg.n_atoms, ol.T, p), -1)
                               for j, lg, ol, p in zip(ids, ligs, oligs, params)]
            finally:
                dsdp.dsdp_grid_free(ctx, grid)
    finally:
        dsdp.dsdp_destroy(ctx)
    # the oracle's own search of each ligand: 384 chains x 40 steps of BFGS on its FP64 maps, FP64 top 9
    dp = oracle.dock_params_array(40, 0, 1.2, rec.pocket_center - BOX / 2, np.array([BOX] * 3))
    o_top = []
    for s, ol in enumerate(oligs):
        best, _, _ = oracle.dock(ol, og, 0, dp, s, 384, n_threads=cores, opt=dict(max_iters=100))
        _, o_idx, o_terms = oracle.rescore_topk(ol, rec.xyz.astype(np.float64), rec.xs_type, best, 9, 1.0)
        o_top.append(dict(score=float(o_terms[0, 0]), coords=ol.coords(best[o_idx[0]])))
    return dict(rec=rec, ligs=ligs, oligs=oligs, og=og, runs=runs, oracle_top=o_top)


def _corner_abs_scale(olig, og, lig, conf):
    """sum over atoms of the trilinear sum of |score| at the 8 corners (oracle maps)."""
    x = olig.coords(conf)
    s = 0.0
    absmaps = oracle.Grid(np.abs(og.maps), og.n, og.origin, og.h)
    for t in set(lig.xs_type.tolist()):
        idx = np.nonzero(lig.xs_type == t)[0]
        e, _ = oracle.interpolate(absmaps, 0, int(t), x[idx])
        s += np.abs(e).sum()
    return s


def _rmsd(a, b):
    return float(np.sqrt(((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2).sum(-1).mean()))


def _top1_against(runs, other):
    """Median |top-1 FP64 score difference| and median top-1 pose RMSD over the ligands."""
    d = [abs(float(r["score"][0]) - o["score"]) for r, o in zip(runs, other)]
    x = [_rmsd(r["coords"][0], o["coords"]) for r, o in zip(runs, other)]
    return float(np.median(d)), float(np.median(x))


def test_fp32_map_run_against_the_oracle_search(system):
    runs, o_top = system["runs"][dsdp.DSDP_MAP_F32], system["oracle_top"]
    for r in runs:
        assert r["n_out"] >= 1 and np.isfinite(r["score"][: r["n_out"]]).all()
    d, x = _top1_against(runs, o_top)
    print(f"maps f32 ({N_LIGANDS} ligands): top-1 against the oracle's search: median |score diff| {d:.4f}, "
          f"median pose RMSD {x:.3f} A; mean top-1 {np.mean([r['score'][0] for r in runs]):.4f} vs the oracle's "
          f"{np.mean([o['score'] for o in o_top]):.4f}")


@pytest.mark.parametrize("dtype", [dsdp.DSDP_MAP_BF16, dsdp.DSDP_MAP_F16])
def test_reduced_precision_map_errors(system, dtype):
    rec, og = system["rec"], system["og"]
    u = UNIT_ROUNDOFF[dtype]
    rel = []
    for lig, olig, r in zip(system["ligs"], system["oligs"], system["runs"][dtype]):
        for c in range(0, 384, 16):  # 24 sampled chains per ligand
            pose = r["chain_best_conf"][c].astype(np.float64)
            terms, _ = olig.score_grid(og, 0, pose)
            err = abs(float(r["chain_best_e"][c]) - terms.sum())
            scale = _corner_abs_scale(olig, og, lig, pose)
            # rounding of each stored corner value (u relative), plus the FP32 path's own tolerance
            assert err <= 2 * u * scale + E_REL * max(scale, 1.0) + 1e-3, (c, err, scale)
            rel.append(err / max(abs(terms.sum()), 1.0))
        # the FP64 rescoring of the reported poses is exact whatever the maps were
        confs = r["chain_best_conf"].astype(np.float64)
        scores, idx, terms = oracle.rescore_topk(olig, rec.xyz.astype(np.float64), rec.xs_type, confs, 9, 1.0)
        assert list(r["chain"]) == list(idx)
        assert np.allclose(r["score"], terms[:, 0], rtol=1e-10, atol=1e-12)
    f32 = [dict(score=float(f["score"][0]), coords=f["coords"][0]) for f in system["runs"][dsdp.DSDP_MAP_F32]]
    d32, x32 = _top1_against(system["runs"][dtype], f32)
    d_o, x_o = _top1_against(system["runs"][dtype], system["oracle_top"])
    print(f"maps {NAMES[dtype]} ({N_LIGANDS} ligands x 24 chains): search-energy error vs FP64 oracle maps, "
          f"relative: median {np.median(rel):.2e}, p95 {np.percentile(rel, 95):.2e}, max {max(rel):.2e}; top-1 "
          f"against the FP32-map run: median |score diff| {d32:.4f}, median pose RMSD {x32:.3f} A; against the "
          f"oracle's search: {d_o:.4f}, {x_o:.3f} A")
