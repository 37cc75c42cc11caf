"""dsdp_rescore_topk_noalloc: the FP64 rescoring + top-k for callers that cannot
allocate device memory when they run it (allocator locks, memory-planning
phases, real-time threads, fixed device budgets).  It must give what the plan's
own rescoring stage gives for the same chain poses, on two calls in a row
(the shared scratch array keeps the previous call's contents).

Named to be collected last, so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402

N_CHAINS, TOP_K, BOX, H = 96, 9, 14.0, 0.375


def _outputs(dev, nx, n_atoms):
    return dict(n=torch.zeros(1, dtype=torch.int32, device=dev), chain=torch.zeros(TOP_K, dtype=torch.int32, device=dev),
                score=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                inter=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                intra=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                conf=torch.zeros((TOP_K, nx), dtype=torch.float64, device=dev),
                coords=torch.zeros((TOP_K, n_atoms, 3), dtype=torch.float32, device=dev))


def _point_outputs(j, o):
    j.d_out_n, j.d_out_chain = o["n"].data_ptr(), o["chain"].data_ptr()
    j.d_out_score, j.d_out_inter = o["score"].data_ptr(), o["inter"].data_ptr()
    j.d_out_intra, j.d_out_conf = o["intra"].data_ptr(), o["conf"].data_ptr()
    j.d_out_coords = o["coords"].data_ptr()


def test_noalloc_rescoring_matches_the_plan_twice_in_a_row():
    dev = torch.device("cuda", 0)
    rec = synth.receptor(1500, 41)
    lig = synth.ligand(18, 5, 41, center=rec.pocket_center)
    box = dsdp.make_box(rec.pocket_center, BOX, H)
    nbytes = dsdp.dsdp_grid_map_bytes(box)
    d_maps = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d_xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
    d_type = torch.from_numpy(rec.xs_type.copy()).to(dev)
    blob = dsdp.dsdp_ligand_pack(lig)
    nx = 7 + dsdp.dsdp_ligand_blob_info(blob)["n_torsions"]
    d_blob = torch.from_numpy(blob.copy()).to(dev)
    conf = torch.zeros((N_CHAINS, nx), dtype=torch.float32, device=dev)
    n = [int(np.ceil(BOX / H))] * 3
    origin = [rec.pocket_center[a] - (n[a] - 1) * H / 2 for a in range(3)]
    j = dsdp.dsdp_job_device()
    j.grid = dsdp.grid_view(d_maps.data_ptr(), n, origin, H)
    j.receptor = dsdp.dsdp_receptor(len(rec.xs_type), d_xyz.data_ptr(), d_type.data_ptr())
    j.h_blob = blob.ctypes.data
    j.d_blob = d_blob.data_ptr()
    j.params = dsdp.make_params(n_chains=N_CHAINS, n_mc_steps=4, n_opt_iters=25, seed=3, top_k=TOP_K)
    for a in range(3):
        j.box_lo[a] = rec.pocket_center[a] - BOX / 2
        j.box_size[a] = BOX
    j.d_chain_best_conf = conf.data_ptr()
    ref = _outputs(dev, nx, lig.n_atoms)
    _point_outputs(j, ref)
    stream = torch.cuda.current_stream().cuda_stream
    dsdp.dsdp_grid_build_device(len(rec.xs_type), d_xyz.data_ptr(), d_type.data_ptr(), box, dsdp.DSDP_MAP_F32,
                                dsdp.DSDP_GRID_EQ4, d_maps.data_ptr(), nbytes, stream)
    plan = dsdp.dsdp_plan_create(None, [j], 0, 0)
    try:
        dsdp.dsdp_plan_launch(plan, stream)  # chains, then the allocating rescoring path
        torch.cuda.synchronize()
    finally:
        dsdp.dsdp_plan_destroy(None, plan)
    for call in range(2):
        got = _outputs(dev, nx, lig.n_atoms)
        _point_outputs(j, got)
        dsdp.dsdp_rescore_topk_noalloc(j, stream)
        torch.cuda.synchronize()
        k = int(ref["n"].item())
        assert int(got["n"].item()) == k >= 1, call
        assert torch.equal(got["chain"][:k], ref["chain"][:k]), call
        for key in ("score", "inter", "intra", "conf"):
            assert np.allclose(got[key][:k].cpu().numpy(), ref[key][:k].cpu().numpy(), rtol=1e-10, atol=1e-12), key
        assert np.allclose(got["coords"][:k].cpu().numpy(), ref["coords"][:k].cpu().numpy(), atol=1e-6)


def test_noalloc_rejects_more_chains_than_its_scratch_holds():
    rec = synth.receptor(300, 42)
    lig = synth.ligand(8, 2, 42, center=rec.pocket_center)
    blob = dsdp.dsdp_ligand_pack(lig)
    j = dsdp.dsdp_job_device()
    j.h_blob = blob.ctypes.data
    j.d_blob = 1  # never dereferenced: the size check comes first
    j.d_chain_best_conf = 1
    j.receptor = dsdp.dsdp_receptor(300, 1, 1)
    j.params = dsdp.make_params(n_chains=dsdp.DSDP_NOALLOC_MAX_CHAINS + 1)
    with pytest.raises(dsdp.DSDPError) as ei:
        dsdp.dsdp_rescore_topk_noalloc(j, 0)
    assert ei.value.status == dsdp.DSDP_ERR_INVALID_ARG
    assert "no-alloc limit" in dsdp.dsdp_last_error()


# Run in a fresh interpreter: the no-alloc call is the first thing this library
# runs on the GPU (no plan, no grid build, no score kernel before it), on poses
# uploaded from the host, so its first call is also the call that resolves the
# scratch array and loads the rescoring kernels.
_FIRST_CALL = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2303_09916_gb300 import dsdp, synth

dev = torch.device("cuda", 0)
rec = synth.receptor(1500, 43)
lig = synth.ligand(18, 5, 43, center=rec.pocket_center)
olig = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
n_chains, top_k = 200, 9
rng = np.random.default_rng(5)
poses = np.zeros((n_chains, olig.nx))
for c in range(n_chains):
    poses[c] = olig.identity_conf()
    poses[c, :3] = rec.pocket_center + rng.uniform(-2.0, 2.0, 3)
    q = rng.normal(size=4)
    poses[c, 3:7] = q / np.linalg.norm(q)
    poses[c, 7:] = rng.uniform(-np.pi, np.pi, olig.T)
poses32 = poses.astype(np.float32)
blob = dsdp.dsdp_ligand_pack(lig)
d_xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
d_type = torch.from_numpy(rec.xs_type.copy()).to(dev)
d_blob = torch.from_numpy(blob.copy()).to(dev)
d_conf = torch.from_numpy(poses32.copy()).to(dev)
out = dict(n=torch.zeros(1, dtype=torch.int32, device=dev), chain=torch.zeros(top_k, dtype=torch.int32, device=dev),
           score=torch.zeros(top_k, dtype=torch.float64, device=dev),
           inter=torch.zeros(top_k, dtype=torch.float64, device=dev),
           intra=torch.zeros(top_k, dtype=torch.float64, device=dev),
           conf=torch.zeros((top_k, olig.nx), dtype=torch.float64, device=dev),
           coords=torch.zeros((top_k, lig.n_atoms, 3), dtype=torch.float32, device=dev))
j = dsdp.dsdp_job_device()
j.receptor = dsdp.dsdp_receptor(len(rec.xs_type), d_xyz.data_ptr(), d_type.data_ptr())
j.h_blob, j.d_blob = blob.ctypes.data, d_blob.data_ptr()
j.params = dsdp.make_params(n_chains=n_chains, top_k=top_k)
j.d_chain_best_conf = d_conf.data_ptr()
j.d_out_n, j.d_out_chain = out["n"].data_ptr(), out["chain"].data_ptr()
j.d_out_score, j.d_out_inter = out["score"].data_ptr(), out["inter"].data_ptr()
j.d_out_intra, j.d_out_conf = out["intra"].data_ptr(), out["conf"].data_ptr()
j.d_out_coords = out["coords"].data_ptr()
stream = torch.cuda.current_stream().cuda_stream
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info(0)[0]
dsdp.dsdp_rescore_topk_noalloc(j, stream)  # the set-up call
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info(0)[0]
_, idx, terms = oracle.rescore_topk(olig, rec.xyz.astype(np.float64), rec.xs_type, poses32.astype(np.float64),
                                    k=top_k, rmsd_cut=1.0)
k = int(out["n"].item())
ok_first = (k == len(idx) and list(out["chain"][:k].cpu().numpy()) == list(idx)
            and np.allclose(out["score"][:k].cpu().numpy(), terms[:, 0], rtol=1e-10, atol=1e-12))
for key in out.values():
    key.zero_()
torch.cuda.synchronize()
free2 = torch.cuda.mem_get_info(0)[0]
dsdp.dsdp_rescore_topk_noalloc(j, stream)  # a later call: no allocation
torch.cuda.synchronize()
free3 = torch.cuda.mem_get_info(0)[0]
ok_second = (int(out["n"].item()) == k and list(out["chain"][:k].cpu().numpy()) == list(idx)
             and np.allclose(out["score"][:k].cpu().numpy(), terms[:, 0], rtol=1e-10, atol=1e-12))
print(json.dumps(dict(ok_first=bool(ok_first), ok_second=bool(ok_second), kept=k,
                      setup_bytes=int(free0 - free1), later_call_bytes=int(free2 - free3))))
'''


def test_noalloc_first_call_in_a_fresh_process():
    """The no-alloc call made first in a new process, before any plan or other
    kernel of the library, matches the oracle's FP64 rescoring of the same
    poses; a second call leaves the device's free memory exactly unchanged."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, root], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(f"no-alloc in a fresh process: {res}")
    assert res["ok_first"] and res["ok_second"], res
    assert res["kept"] >= 1
    assert res["later_call_bytes"] == 0, res
