"""Receptor voxel features (Sec. 2, the binding-site network's input: 36^3
voxels over 70 A, 17 chemistry channels with S and Se merged, one surface
channel) on the GPU against the oracle: bit-exact, since the voxel and surface
decisions are FP32 on both sides with the same operation order and the sums are
exact fixed-point integers."""
import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402


def _gpu_voxelize(xyz, radius, features, center, work=None):
    dev = torch.device("cuda", 0)
    n = len(radius)
    d_xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32)).to(dev)
    d_r = torch.from_numpy(np.ascontiguousarray(radius, dtype=np.float32)).to(dev)
    d_f = torch.from_numpy(np.ascontiguousarray(features, dtype=np.float32)).to(dev)
    out = torch.full((36, 36, 36, 18), -1.0, dtype=torch.float32, device=dev)
    if work is None:
        work = torch.full((dsdp.dsdp_voxel_work_bytes(),), 0xA5, dtype=torch.uint8, device=dev)  # stale contents
    stream = torch.cuda.current_stream().cuda_stream
    dsdp.dsdp_voxelize_device(n, d_xyz.data_ptr() if n else 0, d_r.data_ptr() if n else 0,
                              d_f.data_ptr() if n else 0, center, out.data_ptr(), work.data_ptr(), work.numel(),
                              stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n_atoms,seed", [(4000, 1), (8000, 2), (2000, 3)])
def test_voxel_features_match_the_oracle_bit_for_bit(n_atoms, seed):
    rec = synth.receptor(n_atoms, seed)
    radius, feats = synth.receptor_voxel_inputs(rec)
    c = synth.protein_center(rec)
    ref, inside = oracle.voxelize(rec.xyz, radius, feats, c)
    got = _gpu_voxelize(rec.xyz, radius, feats, c)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]
    surf = int(ref[..., 17].sum())
    print(f"{n_atoms} atoms: {inside} inside the cube, {surf} surface atoms")
    assert 0 < surf < inside
    # non-integer features (partial-charge-like): the same exact fixed-point sums
    fr = np.random.default_rng(seed).uniform(-1, 1, size=feats.shape).astype(np.float32)
    ref2, _ = oracle.voxelize(rec.xyz, radius, fr, c)
    assert np.array_equal(_gpu_voxelize(rec.xyz, radius, fr, c), ref2)


def test_voxel_edge_cases():
    c = np.array([1.0, 2.0, 3.0])
    # no atoms: all channels zero (the stale work buffer is cleared)
    assert not _gpu_voxelize(np.zeros((0, 3)), np.zeros(0), np.zeros((0, 17)), c).any()
    # atoms on the cube's faces and outside it, an isolated atom, and a buried
    # centre inside 12 face-centred-cubic neighbours
    dirs = np.array([[a, b, 0] for a in (-1, 1) for b in (-1, 1)] + [[a, 0, b] for a in (-1, 1) for b in (-1, 1)]
                    + [[0, a, b] for a in (-1, 1) for b in (-1, 1)], dtype=np.float64) / np.sqrt(2)
    cluster = np.vstack([np.zeros((1, 3)), 2.6 * dirs]) + c
    edge = np.array([[c[0] - 35.0, c[1], c[2]], [c[0] + 35.0, c[1], c[2]], [c[0], c[1] + 34.999, c[2]],
                     [c[0] + 20.0, c[1] - 20.0, c[2] + 20.0], [c[0] + 200.0, c[1], c[2]]])
    xyz = np.vstack([cluster, edge]).astype(np.float32)
    radius = np.full(len(xyz), 1.7, dtype=np.float32)
    feats = np.random.default_rng(0).integers(0, 4, size=(len(xyz), 17)).astype(np.float32)
    ref, inside = oracle.voxelize(xyz, radius, feats, c)
    got = _gpu_voxelize(xyz, radius, feats, c)
    assert np.array_equal(got, ref)
    assert ref[..., 17].sum() == 12 + (inside - 13)  # every atom but the buried centre is on the surface


def test_voxelize_rejects_bad_arguments():
    dev = torch.device("cuda", 0)
    out = torch.zeros((36, 36, 36, 18), dtype=torch.float32, device=dev)
    short = torch.zeros(1024, dtype=torch.uint8, device=dev)
    with pytest.raises(dsdp.DSDPError) as ei:
        dsdp.dsdp_voxelize_device(0, 0, 0, 0, [0, 0, 0], out.data_ptr(), short.data_ptr(), short.numel(), 0)
    assert ei.value.status == dsdp.DSDP_ERR_INVALID_ARG
    work = torch.zeros(dsdp.dsdp_voxel_work_bytes(), dtype=torch.uint8, device=dev)
    with pytest.raises(dsdp.DSDPError):
        dsdp.dsdp_voxelize_device(5, 0, 0, 0, [0, 0, 0], out.data_ptr(), work.data_ptr(), work.numel(), 0)
    with pytest.raises(dsdp.DSDPError):
        dsdp.dsdp_voxelize_device(0, 0, 0, 0, [0, float("nan"), 0], out.data_ptr(), work.data_ptr(), work.numel(), 0)
