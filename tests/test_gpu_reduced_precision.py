"""Grid maps stored in BF16 and FP16 (accumulation stays FP32, the final
rescoring FP64): the error of every reported score against the FP64 oracle and
against the FP32-map run, on a typical-4k system (4,000-atom receptor, 80^3
maps, 30-atom ligand with 8 torsions, 384 chains x 40 steps).

Reported (printed) and bounded:
* search energy of each chain's best pose (grid score with the stored maps)
  against the oracle's FP64-map score of that pose: bounded by the storage
  format's rounding of the summed corner values (2^-8 relative for BF16,
  2^-11 for FP16) on top of the FP32 tolerance;
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


@pytest.fixture(scope="module")
def system():
    cfg = synth.config("typical-4k", seed=0)
    rec, lig = cfg.receptor, cfg.ligands[0]
    olig = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    og = oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, np.array([BOX] * 3), H)
    ctx = dsdp.dsdp_create(0)
    runs = {}
    try:
        for dtype in (dsdp.DSDP_MAP_F32, dsdp.DSDP_MAP_BF16, dsdp.DSDP_MAP_F16):
            grid = dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(rec.pocket_center, BOX, H), dtype)
            try:
                params = dsdp.make_params(n_chains=384, n_mc_steps=40, n_opt_iters=100, seed=0, top_k=9)
                jid = dsdp.dsdp_dock_submit(ctx, grid, lig, params)
                runs[dtype] = dsdp.dsdp_dock_poll(ctx, jid, dsdp.result_buffers(lig.n_atoms, olig.T, params), -1)
            finally:
                dsdp.dsdp_grid_free(ctx, grid)
    finally:
        dsdp.dsdp_destroy(ctx)
    # the oracle's own search: 384 chains x 40 steps of BFGS on its FP64 maps, FP64 top 9
    lo = rec.pocket_center - BOX / 2
    dp = oracle.dock_params_array(40, 0, 1.2, lo, np.array([BOX] * 3))
    best, _, _ = oracle.dock(olig, og, 0, dp, 0, 384, n_threads=os.cpu_count() or 1, opt=dict(max_iters=100))
    o_scores, o_idx, _ = oracle.rescore_topk(olig, rec.xyz.astype(np.float64), rec.xs_type, best, 9, 1.0)
    o_top = dict(score=float(o_scores[0]), coords=olig.coords(best[o_idx[0]]))
    return dict(rec=rec, lig=lig, olig=olig, og=og, runs=runs, oracle_top=o_top)


def _against_the_oracle_search(r, o_top):
    rmsd = float(np.sqrt(((r["coords"][0] - o_top["coords"]) ** 2).sum(-1).mean()))
    return float(r["score"][0] - o_top["score"]), rmsd


def test_fp32_map_run_against_the_oracle_search(system):
    r, o_top = system["runs"][dsdp.DSDP_MAP_F32], system["oracle_top"]
    d, rmsd = _against_the_oracle_search(r, o_top)
    assert np.isfinite(d) and np.isfinite(rmsd) and r["score"][0] < 0 and o_top["score"] < 0
    print(f"maps f32: top-1 FP64 score {r['score'][0]:.4f} vs the oracle search's {o_top['score']:.4f} "
          f"(diff {d:+.4f}), top-1 pose RMSD {rmsd:.3f} A")


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


@pytest.mark.parametrize("dtype", [dsdp.DSDP_MAP_BF16, dsdp.DSDP_MAP_F16])
def test_reduced_precision_map_errors(system, dtype):
    rec, lig, olig, og, runs = system["rec"], system["lig"], system["olig"], system["og"], system["runs"]
    r = runs[dtype]
    u = UNIT_ROUNDOFF[dtype]
    rel = []
    for c in range(0, 384, 4):  # 96 sampled chains
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
    # against the FP32-map run
    f32 = runs[dsdp.DSDP_MAP_F32]
    top_rmsd = float(np.sqrt(((r["coords"][0] - f32["coords"][0]) ** 2).sum(-1).mean()))
    d_score = float(r["score"][0] - f32["score"][0])
    print(f"maps {['f32', 'bf16', 'f16'][dtype]}: search-energy error vs FP64 oracle maps over 96 chains: "
          f"median {np.median(rel):.2e}, p95 {np.percentile(rel, 95):.2e}, max {max(rel):.2e} (relative); "
          f"top-1 FP64 score {r['score'][0]:.4f} vs FP32-map run {f32['score'][0]:.4f} (diff {d_score:+.4f}), "
          f"top-1 pose RMSD to the FP32-map top-1 {top_rmsd:.3f} A; "
          f"best of 9 {r['score'].min():.4f} vs {f32['score'].min():.4f}")
    d_o, rmsd_o = _against_the_oracle_search(r, system["oracle_top"])
    print(f"maps {['f32', 'bf16', 'f16'][dtype]}: top-1 against the oracle search: score diff {d_o:+.4f}, "
          f"pose RMSD {rmsd_o:.3f} A")
