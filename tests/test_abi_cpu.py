"""The C ABI library without a GPU: it loads, exports every declared symbol,
and its host-side ligand preparation and validation behave (CPU only)."""
import re
import struct

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

dsdp = pytest.importorskip("paper_2303_09916_gb300.dsdp", reason="libdsdp.so not built")

HEADER = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "include", "dsdp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dsdp_[a-z0-9_]+)\s*\(", text)) - {"dsdp_alloc_fn", "dsdp_free_fn"})


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(dsdp._lib, n), n
    assert sorted(dsdp.EXPORTED) == names


def test_status_strings_and_version():
    assert dsdp.dsdp_status_string(0) == "DSDP_OK"
    assert dsdp.dsdp_status_string(-5) == "DSDP_ERR_CANCELLED"
    assert re.match(r"\d+\.\d+\.\d+", dsdp.dsdp_version())


def _parse_blob(blob):
    hdr = struct.unpack_from("<2I5if3fi5Ii3IiIiI", blob, 0)
    keys = ["magic", "bytes", "n_atoms", "T", "n_bodies", "n_pairs", "rounds", "gyr", "rx", "ry", "rz", "root_atom",
            "off_atom", "off_user", "off_body", "off_pairs", "off_steps", "n_steps", "off_tb", "off_a64", "off_b64",
            "hyd_begin", "stage_bytes", "hb_begin", "off_lane_map"]
    h = dict(zip(keys, hdr))
    n, P = h["n_atoms"], h["n_pairs"]
    user = np.frombuffer(blob, dtype=np.int32, count=n, offset=h["off_user"])
    atom = np.frombuffer(blob, dtype=np.float32, count=4 * n, offset=h["off_atom"]).reshape(n, 4)
    body = atom[:, 3].copy().view(np.int32) >> 8
    rec = np.frombuffer(blob, dtype=np.uint32, count=2 * P, offset=h["off_pairs"]).reshape(P, 2)
    h["nrs"] = rec[:, 1].copy().view(np.float32)
    h["types"] = atom[:, 3].copy().view(np.int32) & 0xFF
    # the records hold byte offsets (16 B per atom slot); give back i | j << 8 for the checks below
    pairs = ((rec[:, 0] & 0xFFFF) >> 4) | ((rec[:, 0] >> 20) << 8)
    steps = np.frombuffer(blob, dtype=np.uint32, count=2 * 32 * h["n_steps"], offset=h["off_steps"]).reshape(
        h["n_steps"], 32, 2)
    brec = np.frombuffer(blob, dtype=np.int32, count=12 * h["n_bodies"], offset=h["off_body"]).reshape(-1, 12)
    h["lane_map"] = np.frombuffer(blob, dtype=np.int16, count=64, offset=h["off_lane_map"]).reshape(32, 2)
    return h, user, body, pairs, steps, brec


RADIUS = np.array([1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0])
XS_BITS = np.array([1, 0, 0, 2, 4, 4, 6, 0])


def _pair_class(ti, tj):
    hyd = (XS_BITS[ti] & XS_BITS[tj] & 1) > 0
    hb = ((XS_BITS[ti] & 2) & ((XS_BITS[tj] & 4) >> 1)) | ((XS_BITS[ti] & 4) >> 1 & (XS_BITS[tj] & 2))
    return np.where(hyd, 1, np.where(hb > 0, 2, 0))


def _check_steps(h, pairs, steps):
    """The intra-pair step table: every pair computed exactly once, no lane active
    or passive twice in a step, reaction forces routed back to the right lane."""
    n, P = h["n_atoms"], h["n_pairs"]
    lmap = h["lane_map"]
    # every atom in exactly one slot; up to 32 atoms atom i alone in lane i
    placed = sorted(int(a) for a in lmap.ravel() if a >= 0)
    assert placed == list(range(n))
    if n <= 32:
        assert all(lmap[i, 0] == (i if i < n else -1) and lmap[i, 1] == -1 for i in range(32))
    lane_of = {int(a): lane for lane in range(32) for a in lmap[lane] if a >= 0}
    assert h["n_steps"] % 2 == 0
    want = {(int(p & 0xFF), int((p >> 8) & 0xFF)): k for k, p in enumerate(pairs)}
    cls = _pair_class(h["types"][pairs & 0xFF], h["types"][(pairs >> 8) & 0xFF])
    seen = set()
    for st in steps:
        x, nrs = st[:, 0], st[:, 1].copy().view(np.float32)
        partner, pred = x & 31, (x >> 5) & 31
        act_slot, pas_slot = (x >> 10) & 1, (x >> 11) & 1
        active = nrs != np.float32(1.0e4)
        passive_of = {}
        step_cls = 0
        for lane in np.nonzero(active)[0]:
            a = int(lmap[lane, act_slot[lane]])
            pl = int(partner[lane])
            b = int(lmap[pl, pas_slot[pl]])
            assert 0 <= a < n and 0 <= b < n and a != b
            assert pl not in passive_of, "lane passive twice in one step"
            passive_of[pl] = int(lane)
            assert int(pred[pl]) == lane, "reaction force not routed to the passive lane"
            key = (min(a, b), max(a, b))
            assert key in want and key not in seen
            seen.add(key)
            k = want[key]
            assert nrs[lane] == h["nrs"][k]
            assert bool(x[lane] >> 12 & 1) == (cls[k] == 1) and bool(x[lane] >> 13 & 1) == (cls[k] == 2)
            step_cls |= 1 << (int(cls[k]) + 13) if cls[k] else 0
        for lane in range(32):
            if lane not in passive_of:  # takes its (zero) reaction force from an idle lane
                assert not active[pred[lane]]
            if not active[lane]:
                assert partner[lane] == lane and not (x[lane] >> 12 & 3)
        assert np.all((x >> 14 & 3) == step_cls >> 14)
    assert len(seen) == P
    # the schedule is as short as the busiest lane allows: with every lane
    # active about as often as passive, a lane of degree d needs ceil(d / 2)
    # steps, and the bipartite colouring reaches that bound exactly (Konig);
    # the packed loop takes steps two at a time, so an odd count gets a pad
    deg = np.zeros(32, int)
    for p in pairs:
        deg[lane_of[int(p & 0xFF)]] += 1
        deg[lane_of[int((p >> 8) & 0xFF)]] += 1
    bound = int(np.max((deg + 1) // 2))
    assert h["n_steps"] == bound + (bound & 1)
    if n > 32:
        # two atoms per lane: the 64 - n atoms with the most pairs alone in their lanes,
        # the others paired most with fewest, so no lane carries more pairs than
        # the busiest single atom and the largest pair sum of that pairing
        adeg = np.zeros(n, int)
        for p in pairs:
            adeg[int(p & 0xFF)] += 1
            adeg[int((p >> 8) & 0xFF)] += 1
        order = sorted(range(n), key=lambda a: -adeg[a])  # stable: ties by atom index
        shared = order[64 - n:]
        want = max([adeg[a] for a in order[:64 - n]] +
                   [adeg[shared[k]] + adeg[shared[-1 - k]] for k in range(len(shared) // 2)])
        assert deg.max() == want


@pytest.mark.parametrize("n,t,seed", [(8, 2, 0), (20, 4, 1), (30, 8, 2), (45, 12, 3), (60, 15, 4), (10, 0, 5),
                                      (64, 15, 6), (33, 6, 7)])
def test_ligand_pack_agrees_with_the_oracle_topology(n, t, seed):
    lig = synth.ligand(n, t, seed)
    blob = dsdp.dsdp_ligand_pack(lig)
    h, user, body, pairs, steps, brec = _parse_blob(bytes(blob))
    ol = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    assert h["magic"] == 0x50445344 and h["bytes"] == len(blob) and h["bytes"] % 16 == 0
    # the FP32 kernels stage a prefix holding every table they read; the pair list
    # (FP64 rescoring) and the FP64 geometry follow it
    assert h["stage_bytes"] % 16 == 0 and h["stage_bytes"] <= h["off_pairs"] <= h["off_a64"] < h["off_b64"] < h["bytes"]
    assert max(h["off_atom"], h["off_user"], h["off_body"], h["off_tb"] + 4 * h["T"],
               h["off_steps"] + 256 * h["n_steps"]) <= h["stage_bytes"]
    assert (h["n_atoms"], h["T"], h["n_bodies"], h["n_pairs"]) == (ol.n_atoms, ol.T, ol.n_bodies, ol.n_pairs)
    assert h["root_atom"] == ol.root_atom
    assert h["gyr"] == pytest.approx(ol.gyration_radius, rel=1e-6)
    assert sorted(user.tolist()) == list(range(n))
    # same pair set (mapped back to input indices)
    got = {tuple(sorted((int(user[p & 0xFF]), int(user[(p >> 8) & 0xFF])))) for p in pairs}
    assert got == {tuple(p) for p in ol.pairs()}
    # per pair -(R_i + R_j); term classes in three contiguous groups (none, hydrophobic, H-bond)
    ti, tj = h["types"][pairs & 0xFF], h["types"][(pairs >> 8) & 0xFF]
    assert np.array_equal(h["nrs"], (-(RADIUS[ti] + RADIUS[tj])).astype(np.float32))
    cls = _pair_class(ti, tj)
    P = h["n_pairs"]
    assert 0 <= h["hyd_begin"] <= h["hb_begin"] <= P
    assert np.array_equal(cls, np.repeat([0, 1, 2], [h["hyd_begin"], h["hb_begin"] - h["hyd_begin"], P - h["hb_begin"]]))
    _check_steps(h, pairs, steps)
    # bodies: depth-first order, subtree atom ranges contiguous and nested
    parent = brec[:, 3]
    begin, end = brec[:, 8], brec[:, 9]
    assert parent[0] == -1 and all(parent[b] < b for b in range(1, h["n_bodies"]))
    for b in range(h["n_bodies"]):
        sub = {b}
        for c in range(b + 1, h["n_bodies"]):
            if parent[c] in sub:
                sub.add(c)
        atoms = [i for i in range(n) if body[i] in sub]
        assert atoms == list(range(begin[b], end[b]))
    assert (1 << h["rounds"]) >= int(brec[:, 10].max()) + 1


@pytest.mark.parametrize("bad", ["n_da_type", "ring_rotatable", "too_many_atoms", "disconnected", "bad_bond"])
def test_ligand_pack_rejects_invalid_input(bad):
    lig = synth.ligand(12, 3, 0)
    if bad == "n_da_type":
        lig.xs_type = lig.xs_type.copy()
        lig.xs_type[0] = 8
    elif bad == "ring_rotatable":
        lig.bonds = np.vstack([lig.bonds, [[0, 11]]]).astype(np.int32)
        lig.rotatable = np.append(lig.rotatable, 1).astype(np.uint8)
    elif bad == "too_many_atoms":
        lig = synth.ligand(12, 3, 0)
        lig.xyz = np.zeros((70, 3), np.float32)
        lig.xs_type = np.zeros(70, np.uint8)
    elif bad == "disconnected":
        lig.bonds = lig.bonds[:-1]
        lig.rotatable = lig.rotatable[:-1]
    elif bad == "bad_bond":
        lig.bonds = lig.bonds.copy()
        lig.bonds[0, 1] = 99
    with pytest.raises(dsdp.DSDPError) as ei:
        dsdp.dsdp_ligand_pack(lig)
    assert ei.value.status == dsdp.DSDP_ERR_INVALID_ARG
    assert dsdp.dsdp_last_error()


def test_grid_map_bytes():
    box = dsdp.make_box([0, 0, 0], [30, 30, 30], 0.375)
    assert dsdp.dsdp_grid_map_bytes(box, dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4) == 8 * 80 ** 3 * 16
    assert dsdp.dsdp_grid_map_bytes(box, dsdp.DSDP_MAP_BF16, dsdp.DSDP_GRID_EQ4) == 8 * 80 ** 3 * 8
    assert dsdp.dsdp_grid_map_bytes(box, dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ3) == 8 * 80 ** 3 * 4
    box20 = dsdp.make_box([0, 0, 0], [20, 20, 20], 0.375)
    assert dsdp.dsdp_grid_map_bytes(box20) == 8 * 54 ** 3 * 16
    assert dsdp.dsdp_grid_map_bytes(dsdp.make_box([0, 0, 0], [0.1, 1, 1], 0.375)) == 0


def test_create_without_a_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dsdp.DSDPError) as ei:
        dsdp.dsdp_create(0)
    assert ei.value.status == dsdp.DSDP_ERR_DEVICE


def test_submit_many_rejects_bad_arguments_without_a_gpu():
    """dsdp_dock_submit_many checks its arguments before touching a context."""
    import ctypes as C

    lib = dsdp._lib
    ids = (C.c_uint64 * 1)()
    assert lib.dsdp_dock_submit_many(None, 1, None, None, None, ids) == dsdp.DSDP_ERR_INVALID_ARG
    assert "NULL" in dsdp.dsdp_last_error()
    assert lib.dsdp_dock_submit_many(None, -1, None, None, None, ids) == dsdp.DSDP_ERR_INVALID_ARG
