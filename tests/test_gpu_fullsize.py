"""The typical-4k workload at full size, in the launch configuration bench.py
times (device-resident plan: grid build kernel, chain kernel, FP64 rescoring and
top-k), checked against the oracle on sampled outputs it can compute one by one:

* 4,096 sampled map vertices (all 8 types) against the receptor sum (Eq. 1),
* every chain's best energy against the oracle's score of that pose,
* the top-9 FP64 rescoring against the oracle's rescoring of all 384 poses,
* 24 sampled MC steps replayed by the oracle from the GPU's state.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402

from gpu_util import E_REL, G_REL, pair_is_ambiguous  # noqa: E402

N_CHAINS, N_STEPS, N_ITERS, TOP_K, BOX, H = 384, 40, 100, 9, 30.0, 0.375


@pytest.fixture(scope="module")
def run():
    cfg = synth.config("typical-4k", seed=0)
    rec, lig = cfg.receptor, cfg.ligands[0]
    dev = torch.device("cuda", 0)
    box = dsdp.make_box(rec.pocket_center, BOX, H)
    nbytes = dsdp.dsdp_grid_map_bytes(box)
    d_maps = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
    d_type = torch.from_numpy(rec.xs_type.copy()).to(dev)
    blob = dsdp.dsdp_ligand_pack(lig)
    info = dsdp.dsdp_ligand_blob_info(blob)
    T = info["n_torsions"]
    nx = 7 + T
    d_blob = torch.from_numpy(blob.copy()).to(dev)
    o = dict(conf=torch.zeros((N_CHAINS, nx), dtype=torch.float32, device=dev),
             e=torch.zeros(N_CHAINS, dtype=torch.float32, device=dev),
             evals=torch.zeros(N_CHAINS, dtype=torch.int32, device=dev),
             trace=torch.zeros((N_CHAINS, N_STEPS + 1, nx + 4), dtype=torch.float32, device=dev),
             n=torch.zeros(1, dtype=torch.int32, device=dev), chain=torch.zeros(TOP_K, dtype=torch.int32, device=dev),
             score=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
             inter=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
             intra=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
             oconf=torch.zeros((TOP_K, nx), dtype=torch.float64, device=dev),
             coords=torch.zeros((TOP_K, lig.n_atoms, 3), dtype=torch.float32, device=dev))
    n = [80, 80, 80]
    origin = [rec.pocket_center[a] - (n[a] - 1) * H / 2 for a in range(3)]
    j = dsdp.dsdp_job_device()
    j.grid = dsdp.grid_view(d_maps.data_ptr(), n, origin, H)
    j.receptor = dsdp.dsdp_receptor(len(rec.xs_type), d_xyz.data_ptr(), d_type.data_ptr())
    j.h_blob = blob.ctypes.data
    j.d_blob = d_blob.data_ptr()
    j.params = dsdp.make_params(n_chains=N_CHAINS, n_mc_steps=N_STEPS, n_opt_iters=N_ITERS, seed=0, top_k=TOP_K,
                                trace=1)
    for a in range(3):
        j.box_lo[a] = rec.pocket_center[a] - BOX / 2
        j.box_size[a] = BOX
    j.d_chain_best_conf, j.d_chain_best_e = o["conf"].data_ptr(), o["e"].data_ptr()
    j.d_chain_evals, j.d_trace = o["evals"].data_ptr(), o["trace"].data_ptr()
    j.d_out_n, j.d_out_chain = o["n"].data_ptr(), o["chain"].data_ptr()
    j.d_out_score, j.d_out_inter = o["score"].data_ptr(), o["inter"].data_ptr()
    j.d_out_intra, j.d_out_conf = o["intra"].data_ptr(), o["oconf"].data_ptr()
    j.d_out_coords = o["coords"].data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    dsdp.dsdp_grid_build_device(len(rec.xs_type), d_xyz.data_ptr(), d_type.data_ptr(), box, dsdp.DSDP_MAP_F32,
                                dsdp.DSDP_GRID_EQ4, d_maps.data_ptr(), nbytes, stream)
    plan = dsdp.dsdp_plan_create(None, [j], 0, 0)
    dsdp.dsdp_plan_launch(plan, stream)
    torch.cuda.synchronize()
    dsdp.dsdp_plan_destroy(None, plan)
    maps = d_maps.view(torch.float32).reshape(8, 80, 80, 80, 4).cpu().numpy()
    res = {k: v.cpu().numpy() for k, v in o.items()}
    olig = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    return dict(rec=rec, lig=lig, olig=olig, maps=maps, res=res, origin=np.array(origin), T=T, nx=nx)


@pytest.fixture(scope="module")
def oracle_maps(run):
    rec = run["rec"]
    return oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, np.array([BOX] * 3), H)


def test_sampled_vertices_match_the_receptor_sum(run):
    rec, maps, origin = run["rec"], run["maps"], run["origin"]
    rng = np.random.default_rng(0)
    idx = rng.integers(0, 80, size=(4096, 3))
    pts = origin + H * idx
    xyz = rec.xyz.astype(np.float64)
    checked = 0
    for t in range(8):
        ref = oracle.receptor_field(xyz, rec.xs_type, t, pts)
        scale = oracle.receptor_field_abs(xyz, rec.xs_type, t, pts)  # sum |f|, sum |f'| of the summed terms
        got = maps[t, idx[:, 2], idx[:, 1], idx[:, 0]].astype(np.float64)
        for v in range(len(pts)):
            d = np.linalg.norm(xyz - pts[v], axis=1)
            near = np.nonzero(d < 8.01)[0]
            if any(pair_is_ambiguous(t, int(rec.xs_type[k]), float(d[k]), 5e-5) for k in near):
                continue
            assert abs(got[v, 0] - ref[v, 0]) <= E_REL * max(scale[v, 0], 1.0)
            assert np.abs(got[v, 1:] - ref[v, 1:]).max() <= G_REL * max(scale[v, 1], 1e-2)
            checked += 1
    assert checked >= 0.99 * 8 * len(pts)


def test_chain_energies_are_the_oracle_score_of_their_poses(run, oracle_maps):
    res, olig = run["res"], run["olig"]
    assert np.all(res["evals"] > 0)
    bad = 0
    for c in range(N_CHAINS):
        terms, _ = olig.score_grid(oracle_maps, 0, res["conf"][c].astype(np.float64))
        if abs(terms.sum() - res["e"][c]) > E_REL * max(abs(terms.sum()), 1.0) * 10:
            bad += 1
    # the pose is FP32 and the maps differ by FP32 rounding: a pose on a repulsive
    # wall can amplify that; allow at most 1 % outliers
    assert bad <= N_CHAINS // 100, bad


def test_top_k_matches_the_oracle_rescoring(run):
    res, olig, rec = run["res"], run["olig"], run["rec"]
    confs = res["conf"].astype(np.float64)
    scores, idx, terms = oracle.rescore_topk(olig, rec.xyz.astype(np.float64), rec.xs_type, confs, TOP_K, 1.0)
    n = int(res["n"][0])
    assert n == len(idx)
    assert list(res["chain"][:n]) == list(idx)
    assert np.allclose(res["score"][:n], terms[:, 0], rtol=1e-10, atol=1e-12)
    assert np.allclose(res["inter"][:n], terms[:, 1], rtol=1e-10, atol=1e-12)
    assert np.allclose(res["intra"][:n], terms[:, 2], rtol=1e-10, atol=1e-12)


def test_sampled_steps_replay_on_the_oracle(run, oracle_maps):
    """24 sampled steps replayed by the oracle from the GPU's state: the mutation
    matches exactly; the candidate energies agree about as often as the oracle
    agrees with itself when its start moves by one FP32 ulp."""
    res, olig, nx, T = run["res"], run["olig"], run["nx"], run["T"]
    rec = run["rec"]
    tr = res["trace"].astype(np.float64)
    dp = oracle.dock_params_array(N_STEPS, 0, 1.2, rec.pocket_center - BOX / 2, np.array([BOX] * 3))
    rng = np.random.default_rng(1)
    match = base = 0
    samples = [(int(rng.integers(0, N_CHAINS)), int(rng.integers(1, N_STEPS + 1))) for _ in range(24)]
    for c, s in samples:
        cur, e_cur = tr[c, s - 1, :nx], tr[c, s - 1, nx + 1]
        _, _, rec_ = oracle.mc_step(olig, oracle_maps, 0, dp, 0, c, s, cur, e_cur, opt=dict(max_iters=N_ITERS))
        nudged = cur.copy()
        nudged[:3] = np.nextafter(cur[:3].astype(np.float32), np.float32(np.inf)).astype(np.float64)
        _, _, rec2 = oracle.mc_step(olig, oracle_maps, 0, dp, 0, c, s, nudged, e_cur, opt=dict(max_iters=N_ITERS))
        assert int(tr[c, s, nx + 2]) == int(rec_[0])
        tol = E_REL * max(abs(rec_[2]), 1.0) * 10
        match += abs(rec_[2] - tr[c, s, nx]) <= tol
        base += abs(rec_[2] - rec2[2]) <= tol
    print(f"full-size replay: GPU vs oracle {match}/24, oracle vs nudged oracle {base}/24")
    assert match >= base - 4, (match, base)
