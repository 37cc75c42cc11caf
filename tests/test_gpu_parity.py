"""GPU path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 device arithmetic against FP64), see gpu_util:
  energy   |dE| <= 1e-4 * max(sum_i |e_i|, 1)   (e_i: per-atom and per-pair terms)
  gradient ||dg||_inf <= 1e-4 * max(||g||_inf, 1e-2); map vertices use the sums
  of the absolute pair terms and slopes as their scales.
Where FP32 and FP64 may take different branches (a pair within 2e-4 A of the
cutoff or of a slope kink, an atom on a cell face in Eq. 3 mode) the input is
skipped and counted, never silently compared with a looser bound.
"""

import numpy as np
import pytest

import oracle
from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402

from gpu_util import E_REL, G_FP32, G_REL, Complex, vertex_ambiguity, vertex_scales  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = dsdp.dsdp_create(0)
    yield c
    dsdp.dsdp_destroy(c)


def _box(cx):
    return dsdp.make_box(cx.center, cx.size, cx.spacing)


# ---------------------------------------------------------------- grid maps
@pytest.fixture(scope="module")
def ragged():
    # 7.1 A at 0.375 A -> 19 vertices per axis: bricks of 8 x 8 x 4 leave ragged tails on every axis
    return Complex(2000, 7.1, 10, 2, seed=11)


def test_grid_build_f32_matches_oracle(ctx, ragged):
    cx = ragged
    grid = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4)
    try:
        info = dsdp.dsdp_grid_info(grid)
        og = cx.oracle_grid()
        assert info["n"] == list(og.n) == [19, 19, 19]
        assert np.allclose(info["origin"], og.origin, atol=1e-12)
        maps = dsdp.dsdp_grid_download(ctx, grid).astype(np.float64)
    finally:
        dsdp.dsdp_grid_free(ctx, grid)
    ref = og.maps
    amb = vertex_ambiguity(cx.rec_xyz64, cx.rec.xs_type, og.origin, og.n, og.h)
    ok = ~amb
    assert amb.mean() < 0.01, amb.mean()
    scale = vertex_scales(cx, og)  # (8, nz, ny, nx, 2): sum |f|, sum |f'| over the summed terms
    e_err = np.abs(maps[..., 0] - ref[..., 0])
    e_tol = E_REL * np.maximum(scale[..., 0], 1.0)
    assert np.all(e_err[ok] <= e_tol[ok]), (e_err / e_tol)[ok].max()
    g_err = np.abs(maps[..., 1:] - ref[..., 1:]).max(-1)
    g_tol = G_REL * np.maximum(scale[..., 1], 1e-2)
    assert np.all(g_err[ok] <= g_tol[ok]), (g_err / g_tol)[ok].max()
    # errors relative to the vertex values themselves: what the FP32 sums (with
    # the ex2.approx intrinsic) really use of the term-scale budget
    e_rel = (e_err / np.maximum(np.abs(ref[..., 0]), 1.0))[ok].max()
    g_rel = (g_err / np.maximum(np.abs(ref[..., 1:]).max(-1), 1e-2))[ok].max()
    print(f"grid vertices: max |dE| / sum|f| {(e_err / np.maximum(scale[..., 0], 1.0))[ok].max():.2e}, "
          f"|dE| / max(|E|, 1) {e_rel:.2e}, |dg|_inf / |g|_inf {g_rel:.2e}")
    assert e_rel <= E_REL, e_rel  # the gradient, a vector sum, may cancel: reported only


@pytest.mark.parametrize("dtype", [dsdp.DSDP_MAP_BF16, dsdp.DSDP_MAP_F16])
def test_grid_build_16bit_is_the_rounded_fp32_map(ctx, ragged, dtype):
    cx = ragged
    g32 = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4)
    g16 = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dtype, dsdp.DSDP_GRID_EQ4)
    try:
        m32 = dsdp.dsdp_grid_download(ctx, g32)
        m16 = dsdp.dsdp_grid_download(ctx, g16)
    finally:
        dsdp.dsdp_grid_free(ctx, g32)
        dsdp.dsdp_grid_free(ctx, g16)
    t = torch.from_numpy(m32)
    rounded = (t.to(torch.bfloat16) if dtype == dsdp.DSDP_MAP_BF16 else t.to(torch.float16)).float().numpy()
    assert np.array_equal(m16, rounded)


def test_grid_eq3_score_channel_matches_eq4(ctx, ragged):
    cx = ragged
    g4 = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4)
    g3 = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ3)
    try:
        m4 = dsdp.dsdp_grid_download(ctx, g4, dsdp.DSDP_GRID_EQ4)
        m3 = dsdp.dsdp_grid_download(ctx, g3, dsdp.DSDP_GRID_EQ3)
    finally:
        dsdp.dsdp_grid_free(ctx, g4)
        dsdp.dsdp_grid_free(ctx, g3)
    # same accumulation; the two instantiations may contract multiply-adds differently
    assert np.allclose(m3[..., 0], m4[..., 0], rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- scoring
@pytest.fixture(scope="module")
def scoring_complex():
    return Complex(2000, 16.0, 24, 6, seed=3)


def _compare_scores(cx, grid_o, mode, confs, e, g, flags=3, label=""):
    """Element-wise comparison with the oracle at the stated tolerances (term
    scale for energies, gradient norm for gradients).  Also reports, and bounds,
    the errors relative to the result itself: |dE| / max(|E|, 1) and
    ||dg||_inf / max(||g||_inf, 1e-2) -- how much of the budget the FP32
    arithmetic (with the ex2.approx and __sincosf intrinsics) really uses: on
    Eq. 4 maps the gradient stays within G_FP32, the size of the gradient probe
    the chain tests use."""
    skipped = 0
    worst_e = worst_er = worst_g = 0.0
    for i, c in enumerate(confs):
        if cx.conf_is_ambiguous(grid_o, mode, c):
            skipped += 1
            continue
        terms, gref = cx.olig.score_grid(grid_o, mode, c, flags)
        eref = (terms[0] if flags & 1 else 0.0) + (terms[1] if flags & 2 else 0.0)
        scale = max(cx.abs_terms(grid_o, mode, c), 1.0)
        de = abs(e[i] - eref)
        dg = np.abs(g[i] - gref).max()
        gs = max(np.abs(gref).max(), 1e-2)
        worst_e = max(worst_e, de / scale)
        worst_er = max(worst_er, de / max(abs(eref), 1.0))
        worst_g = max(worst_g, dg / gs)
        assert de <= E_REL * scale, (i, e[i], eref, scale)
        assert dg <= G_REL * gs, (i, g[i], gref)
    assert skipped <= len(confs) // 4, skipped
    print(f"score errors {label} mode {mode} flags {flags}: max |dE| / sum|e_i| {worst_e:.2e}, "
          f"|dE| / max(|E|, 1) {worst_er:.2e}, |dg|_inf / |g|_inf {worst_g:.2e} ({skipped} skipped)")
    assert worst_er <= E_REL, worst_er
    if mode == dsdp.DSDP_GRID_EQ4:
        assert worst_g <= G_FP32, worst_g
    return worst_e, worst_er, worst_g


@pytest.mark.parametrize("mode", [dsdp.DSDP_GRID_EQ4, dsdp.DSDP_GRID_EQ3])
def test_score_eval_on_oracle_maps(ctx, scoring_complex, mode):
    """(i) the scoring kernel alone, on the oracle's maps rounded to FP32."""
    cx = scoring_complex
    og = cx.oracle_grid()
    maps = og.maps if mode == dsdp.DSDP_GRID_EQ4 else og.maps[..., :1]
    grid = dsdp.dsdp_grid_from_maps(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, mode,
                                    maps.astype(np.float32))
    try:
        confs = cx.random_confs(96, seed=1 + mode)
        for flags in (dsdp.DSDP_TERM_ALL, dsdp.DSDP_TERM_INTER, dsdp.DSDP_TERM_INTRA):
            e, g = dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs, flags)
            _compare_scores(cx, og, mode, confs, e, g, flags)
    finally:
        dsdp.dsdp_grid_free(ctx, grid)


def test_score_eval_normalised(ctx, scoring_complex):
    """DSDP_TERM_NORMALISED divides the selected terms and their gradient by
    1 + 0.0585 T (the torsion normalisation of the reported scores); undone, the
    results match the oracle's FP64 terms within the FP32 tolerance."""
    cx = scoring_complex
    og = cx.oracle_grid()
    grid = dsdp.dsdp_grid_from_maps(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32,
                                    dsdp.DSDP_GRID_EQ4, og.maps.astype(np.float32))
    try:
        confs = cx.random_confs(48, seed=3)
        w = 1.0 + 0.0585 * cx.T
        for flags in (dsdp.DSDP_TERM_ALL, dsdp.DSDP_TERM_INTER):
            e, g = dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs, flags)
            en, gn = dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs, flags | dsdp.DSDP_TERM_NORMALISED)
            assert np.allclose(en, e / w, rtol=1e-6, atol=1e-6) and np.allclose(gn, g / w, rtol=1e-6, atol=1e-6)
            _compare_scores(cx, og, 0, confs, en * w, gn * w, flags)
        with pytest.raises(dsdp.DSDPError):
            dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs, dsdp.DSDP_TERM_NORMALISED)  # selects no term
    finally:
        dsdp.dsdp_grid_free(ctx, grid)


def test_score_eval_end_to_end_on_gpu_maps(ctx, scoring_complex):
    """(ii) GPU-built maps and the scoring kernel together."""
    cx = scoring_complex
    og = cx.oracle_grid()
    grid = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4)
    try:
        confs = cx.random_confs(64, seed=7)
        e, g = dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs)
        _compare_scores(cx, og, 0, confs, e, g)
    finally:
        dsdp.dsdp_grid_free(ctx, grid)


@pytest.mark.parametrize("n_atoms,T,seed", [(60, 15, 21), (33, 0, 22), (1, 0, 23), (2, 0, 24), (32, 9, 25)])
def test_score_eval_ligand_shapes(ctx, n_atoms, T, seed):
    """Edge shapes: two atoms per lane (> 32 atoms), rigid ligands, a single atom."""
    if n_atoms == 1:
        cx = Complex(800, 12.0, 2, 0, seed=seed)
        lig = synth.Ligand(cx.lig.xyz[:1].copy(), cx.lig.xs_type[:1].copy(), np.zeros((0, 2), np.int32),
                           np.zeros(0, np.uint8), 0)
        cx.lig = lig
        cx.olig = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    else:
        cx = Complex(800, 12.0, n_atoms, T, seed=seed)
    og = cx.oracle_grid()
    grid = dsdp.dsdp_grid_from_maps(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32,
                                    dsdp.DSDP_GRID_EQ4, og.maps.astype(np.float32))
    try:
        confs = cx.random_confs(40, seed=seed)
        e, g = dsdp.dsdp_score_eval(ctx, grid, cx.lig, confs)
        _compare_scores(cx, og, 0, confs, e, g)
    finally:
        dsdp.dsdp_grid_free(ctx, grid)


# ---------------------------------------------------------------- chains
@pytest.fixture(scope="module")
def chain_complex():
    return Complex(1500, 14.0, 16, 4, seed=5)


def _run_job(ctx, grid, lig, T, **kw):
    params = dsdp.make_params(**kw)
    jid = dsdp.dsdp_dock_submit(ctx, grid, lig, params)
    return dsdp.dsdp_dock_poll(ctx, jid, dsdp.result_buffers(lig.n_atoms, T, params), wait_ms=-1)


def test_adaptive_search_space_starts_match_the_oracle(ctx, chain_complex):
    """Adaptive search space (Sec. 2, third modification): with binding-site
    points the chains start in the box intersected with the union of 7 A balls.
    The first line search of every chain (one BFGS iteration) ends where the
    oracle's does from its own start -- so the GPU drew the same starts (the
    inside / outside decisions are FP32 on both sides).  The device-resident
    plan with d_site_points gives bitwise the handle API's chains."""
    cx = chain_complex
    og = cx.oracle_grid()
    sites = synth.site_points(cx.rec, 60, seed=4, spread=4.0)
    grid = dsdp.dsdp_grid_from_maps(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx), dsdp.DSDP_MAP_F32,
                                    dsdp.DSDP_GRID_EQ4, og.maps.astype(np.float32))
    nc, nx = 32, 7 + cx.T
    dp = oracle.dock_params_array(1, 0, 1.2, cx.box_lo(), cx.size, sites, 7.0)
    starts = np.array([oracle.chain_init(cx.olig, dp, 7, c) for c in range(nc)])
    d = np.linalg.norm(starts[:, None, :3] - sites[None].astype(np.float64), axis=2).min(1)
    assert np.all(d <= 7.0 + 1e-5)
    box_starts = np.array([oracle.chain_init(cx.olig, oracle.dock_params_array(1, 0, 1.2, cx.box_lo(), cx.size), 7, c)
                           for c in range(nc)])
    assert not np.array_equal(starts[:, :3], box_starts[:, :3])  # the region does restrict these starts
    try:
        res = _run_job(ctx, grid, cx.lig, cx.T, n_chains=nc, n_mc_steps=2, n_opt_iters=1, seed=7, trace=1, top_k=1,
                       site_points=sites)
        for c in range(nc):
            _, e_ref, _, _ = cx.olig.local_opt(og, 0, 0, starts[c], opt=dict(max_iters=1))
            pose = res["trace"][c, 0, :nx].astype(np.float64)
            tol = E_REL * max(cx.abs_terms(og, 0, pose), 1.0)
            assert abs(float(res["trace"][c, 0, nx + 1]) - e_ref) <= tol, c
        # the same jobs through the device-resident plan
        dev = torch.device("cuda", 0)
        stream = torch.cuda.current_stream().cuda_stream
        info = dsdp.dsdp_grid_info(grid)
        maps = torch.from_numpy(og.maps.astype(np.float32).ravel().copy()).to(dev)
        blob = dsdp.dsdp_ligand_pack(cx.lig)
        dblob = torch.from_numpy(blob.copy()).to(dev)
        dsites = torch.from_numpy(sites.copy()).to(dev)
        conf = torch.zeros((nc, nx), dtype=torch.float32, device=dev)
        e = torch.zeros(nc, dtype=torch.float32, device=dev)
        j = dsdp.dsdp_job_device()
        j.grid = dsdp.grid_view(maps.data_ptr(), info["n"], info["origin"], cx.spacing, dsdp.DSDP_MAP_F32)
        j.h_blob, j.d_blob = blob.ctypes.data, dblob.data_ptr()
        j.params = dsdp.make_params(n_chains=nc, n_mc_steps=2, n_opt_iters=1, seed=7, top_k=1, site_points=sites)
        j.d_site_points = dsites.data_ptr()
        for a in range(3):
            j.box_lo[a], j.box_size[a] = cx.box_lo()[a], cx.size[a]
        j.d_chain_best_conf, j.d_chain_best_e = conf.data_ptr(), e.data_ptr()
        plan = dsdp.dsdp_plan_create(None, [j], dsdp.DSDP_PLAN_NO_RESCORE, 1)
        try:
            dsdp.dsdp_plan_launch(plan, stream)
            torch.cuda.synchronize()
        finally:
            dsdp.dsdp_plan_destroy(None, plan)
        assert np.array_equal(e.cpu().numpy(), res["chain_best_e"])
        assert np.array_equal(conf.cpu().numpy(), res["chain_best_conf"])
    finally:
        dsdp.dsdp_grid_free(ctx, grid)


def test_rescore_topk_matches_oracle(ctx):
    cx = Complex(2000, 16.0, 20, 4, seed=9)
    grid = dsdp.dsdp_grid_build(ctx, cx.rec.xyz, cx.rec.xs_type, _box(cx))
    try:
        res = _run_job(ctx, grid, cx.lig, cx.T, n_chains=64, n_mc_steps=5, n_opt_iters=30, seed=3, top_k=9)
    finally:
        dsdp.dsdp_grid_free(ctx, grid)
    confs = res["chain_best_conf"].astype(np.float64)
    scores, idx, terms = oracle.rescore_topk(cx.olig, cx.rec_xyz64, cx.rec.xs_type, confs, k=9, rmsd_cut=1.0)
    assert list(res["chain"]) == list(idx)
    assert np.allclose(res["score"], terms[:, 0], rtol=1e-10, atol=1e-12)
    assert np.allclose(res["inter"], terms[:, 1], rtol=1e-10, atol=1e-12)
    assert np.allclose(res["intra"], terms[:, 2], rtol=1e-10, atol=1e-12)
    assert np.array_equal(res["conf"], confs[idx])
    for q, c in enumerate(idx):
        assert np.allclose(res["coords"][q], cx.olig.coords(confs[c]), atol=2e-5)


def test_determinism_and_batch_independence(ctx):
    """A job's results depend on (seed, chain) only: bitwise equal when rerun and
    when run together with other jobs on other grids."""
    a = Complex(1500, 14.0, 18, 5, seed=31)
    b = Complex(2500, 18.0, 40, 10, seed=32)
    ga = dsdp.dsdp_grid_build(ctx, a.rec.xyz, a.rec.xs_type, _box(a))
    gb = dsdp.dsdp_grid_build(ctx, b.rec.xyz, b.rec.xs_type, _box(b), dsdp.DSDP_MAP_BF16)
    try:
        kw = dict(n_chains=48, n_mc_steps=6, n_opt_iters=25, seed=5, top_k=6)
        r1 = _run_job(ctx, ga, a.lig, a.T, **kw)
        r2 = _run_job(ctx, ga, a.lig, a.T, **kw)
        # in the mix: other jobs submitted before and after, all in flight together
        pa = dsdp.make_params(**kw)
        pb = dsdp.make_params(n_chains=96, n_mc_steps=6, n_opt_iters=25, seed=9, top_k=6)
        j0 = dsdp.dsdp_dock_submit(ctx, gb, b.lig, pb)
        j1 = dsdp.dsdp_dock_submit(ctx, ga, a.lig, pa)
        j2 = dsdp.dsdp_dock_submit(ctx, gb, b.lig, pb)
        r3 = dsdp.dsdp_dock_poll(ctx, j1, dsdp.result_buffers(a.lig.n_atoms, a.T, pa), wait_ms=-1)
        for j in (j0, j2):
            dsdp.dsdp_dock_poll(ctx, j, dsdp.result_buffers(b.lig.n_atoms, b.T, pb), wait_ms=-1)
    finally:
        dsdp.dsdp_grid_free(ctx, ga)
        dsdp.dsdp_grid_free(ctx, gb)
    for r in (r2, r3):
        assert np.array_equal(r["chain_best_e"], r1["chain_best_e"])
        assert np.array_equal(r["chain_best_conf"], r1["chain_best_conf"])
        assert np.array_equal(r["score"], r1["score"]) and list(r["chain"]) == list(r1["chain"])


def test_submit_many_matches_single_submissions(ctx):
    """dsdp_dock_submit_many (ligands packed on several host threads, queued
    together) gives each job the results of its own dsdp_dock_submit, bitwise;
    a set with one invalid job queues nothing."""
    a = Complex(1500, 14.0, 18, 5, seed=41)
    b = Complex(2500, 18.0, 40, 10, seed=42)
    ga = dsdp.dsdp_grid_build(ctx, a.rec.xyz, a.rec.xs_type, _box(a))
    gb = dsdp.dsdp_grid_build(ctx, b.rec.xyz, b.rec.xs_type, _box(b))
    try:
        pa = dsdp.make_params(n_chains=48, n_mc_steps=6, n_opt_iters=25, seed=7, top_k=6)
        pb = dsdp.make_params(n_chains=64, n_mc_steps=6, n_opt_iters=25, seed=8, top_k=6)
        ref_a = _run_job(ctx, ga, a.lig, a.T, n_chains=48, n_mc_steps=6, n_opt_iters=25, seed=7, top_k=6)
        ref_b = _run_job(ctx, gb, b.lig, b.T, n_chains=64, n_mc_steps=6, n_opt_iters=25, seed=8, top_k=6)
        items = [(gb, b, pb, ref_b), (ga, a, pa, ref_a), (gb, b, pb, ref_b), (ga, a, pa, ref_a)] * 3
        ids = dsdp.dsdp_dock_submit_many(ctx, [g for g, *_ in items], [c.lig for _, c, *_ in items],
                                         [p for _, _, p, _ in items])
        assert len(set(ids)) == len(items)
        for jid, (_, c, p, ref) in zip(ids, items):
            r = dsdp.dsdp_dock_poll(ctx, jid, dsdp.result_buffers(c.lig.n_atoms, c.T, p), wait_ms=-1)
            assert np.array_equal(r["chain_best_e"], ref["chain_best_e"])
            assert np.array_equal(r["chain_best_conf"], ref["chain_best_conf"])
            assert np.array_equal(r["score"], ref["score"]) and list(r["chain"]) == list(ref["chain"])
        before = dsdp.dsdp_get_stats(ctx)["submitted"]
        bad = dsdp.make_params(n_chains=-3, n_mc_steps=6, n_opt_iters=25, seed=8, top_k=6)
        with pytest.raises(dsdp.DSDPError, match="job 1"):
            dsdp.dsdp_dock_submit_many(ctx, [ga, gb, ga], [a.lig, b.lig, a.lig], [pa, bad, pa])
        assert dsdp.dsdp_get_stats(ctx)["submitted"] == before
    finally:
        dsdp.dsdp_grid_free(ctx, ga)
        dsdp.dsdp_grid_free(ctx, gb)


def test_max_batch_chains_splits_batches_without_changing_results(ctx):
    """A context whose batches hold at most two jobs' chains runs six jobs queued
    together in at least three batches (dsdp_stats.batches), each job with the
    results it has in a context without the limit."""
    a = Complex(1500, 14.0, 18, 5, seed=51)
    kw = dict(n_chains=64, n_mc_steps=4, n_opt_iters=20, top_k=4)
    small = dsdp.dsdp_create(0, max_batch_chains=2 * kw["n_chains"], max_inflight_jobs=16)
    try:
        results = {}
        for c in (ctx, small):
            g = dsdp.dsdp_grid_build(c, a.rec.xyz, a.rec.xs_type, _box(a))
            try:
                params = [dsdp.make_params(seed=s, **kw) for s in range(6)]
                b0 = dsdp.dsdp_get_stats(c)["batches"]
                ids = dsdp.dsdp_dock_submit_many(c, [g] * 6, [a.lig] * 6, params)
                results[c] = [dsdp.dsdp_dock_poll(c, j, dsdp.result_buffers(a.lig.n_atoms, a.T, p), wait_ms=-1)
                              for j, p in zip(ids, params)]
                if c == small:
                    assert dsdp.dsdp_get_stats(c)["batches"] - b0 >= 3
            finally:
                dsdp.dsdp_grid_free(c, g)
        for r0, r1 in zip(results[ctx], results[small]):
            assert np.array_equal(r0["chain_best_e"], r1["chain_best_e"])
            assert np.array_equal(r0["score"], r1["score"]) and list(r0["chain"]) == list(r1["chain"])
    finally:
        dsdp.dsdp_destroy(small)


def test_plan_launch_configurations_agree(ctx):
    """One uneven batch (ligands of 10-60 atoms, 0-15 torsions, two map formats)
    through the device plan in every launch configuration the autotuner chooses
    from -- 128- or 96-register chain kernel, 1, 2 or 4 chains per CTA, with or
    without the persistent work queue -- gives bitwise the same chains, and the
    autotuner returns one of them.
    Each job run alone in a plan of its own gives bitwise what it gave in the
    batch (the batch mixes one- and two-atoms-per-lane ligands on one map format)."""
    dev = torch.device("cuda", 0)
    rec = synth.receptor(2000, 51)
    stream = torch.cuda.current_stream().cuda_stream
    keep, jobs = [], []
    for i, (n_atoms, T, dtype) in enumerate([(10, 0, 0), (24, 5, 0), (33, 9, 1), (60, 15, 0), (45, 12, 1)]):
        lig = synth.ligand(n_atoms, T, 60 + i, center=rec.pocket_center)
        box = dsdp.make_box(rec.pocket_center, 16.0, 0.375)
        nb = dsdp.dsdp_grid_map_bytes(box, dtype)
        maps = torch.empty(nb, dtype=torch.uint8, device=dev)
        xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
        ty = torch.from_numpy(rec.xs_type.copy()).to(dev)
        dsdp.dsdp_grid_build_device(len(ty), xyz.data_ptr(), ty.data_ptr(), box, dtype, 0, maps.data_ptr(), nb, stream)
        blob = dsdp.dsdp_ligand_pack(lig)
        nx = 7 + dsdp.dsdp_ligand_blob_info(blob)["n_torsions"]
        dblob = torch.from_numpy(blob.copy()).to(dev)
        conf = torch.zeros((48, nx), dtype=torch.float32, device=dev)
        e = torch.zeros(48, dtype=torch.float32, device=dev)
        n = [int(np.ceil(16.0 / 0.375))] * 3
        j = dsdp.dsdp_job_device()
        j.grid = dsdp.grid_view(maps.data_ptr(), n, [rec.pocket_center[a] - (n[a] - 1) * 0.375 / 2 for a in range(3)],
                                0.375, dtype)
        j.receptor = dsdp.dsdp_receptor(len(ty), xyz.data_ptr(), ty.data_ptr())
        j.h_blob, j.d_blob = blob.ctypes.data, dblob.data_ptr()
        j.params = dsdp.make_params(n_chains=48, n_mc_steps=3, n_opt_iters=15, seed=i)
        for a in range(3):
            j.box_lo[a] = rec.pocket_center[a] - 8.0
            j.box_size[a] = 16.0
        j.d_chain_best_conf, j.d_chain_best_e = conf.data_ptr(), e.data_ptr()
        jobs.append(j)
        keep.append((maps, xyz, ty, blob, dblob, conf, e))
    results = []
    for tile_config in range(1, 13):  # register budget (128, 96, 80, 72) x chains per CTA (1, 2, 4)
        for flags in (0, dsdp.DSDP_PLAN_PERSISTENT):
            plan = dsdp.dsdp_plan_create(None, jobs, flags | dsdp.DSDP_PLAN_NO_RESCORE, tile_config)
            try:
                dsdp.dsdp_plan_launch(plan, stream)
                torch.cuda.synchronize()
            finally:
                dsdp.dsdp_plan_destroy(None, plan)
            results.append([(k[5].cpu().numpy().copy(), k[6].cpu().numpy().copy()) for k in keep])
    for other in results[1:]:
        for (c0, e0), (c1, e1) in zip(results[0], other):
            assert np.array_equal(c0, c1) and np.array_equal(e0, e1)
    for k, j in enumerate(jobs):
        plan = dsdp.dsdp_plan_create(None, [j], dsdp.DSDP_PLAN_NO_RESCORE, 1)
        try:
            dsdp.dsdp_plan_launch(plan, stream)
            torch.cuda.synchronize()
        finally:
            dsdp.dsdp_plan_destroy(None, plan)
        assert np.array_equal(keep[k][5].cpu().numpy(), results[0][k][0]), k
        assert np.array_equal(keep[k][6].cpu().numpy(), results[0][k][1]), k
    plan = dsdp.dsdp_plan_create(None, jobs, dsdp.DSDP_PLAN_NO_RESCORE, 0)
    try:
        chosen = dsdp.dsdp_plan_autotune(plan, stream, 1)
    finally:
        dsdp.dsdp_plan_destroy(None, plan)
    assert 1 <= chosen <= 24


def test_plan_replayed_from_a_cuda_graph_matches_the_eager_launch(ctx):
    """A plan launch captured into a CUDA graph (persistent work queue included)
    replays with bitwise the eager results, twice in a row."""
    dev = torch.device("cuda", 0)
    rec = synth.receptor(1500, 71)
    stream = torch.cuda.current_stream().cuda_stream
    box = dsdp.make_box(rec.pocket_center, 14.0, 0.375)
    nb = dsdp.dsdp_grid_map_bytes(box)
    maps = torch.empty(nb, dtype=torch.uint8, device=dev)
    xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
    ty = torch.from_numpy(rec.xs_type.copy()).to(dev)
    dsdp.dsdp_grid_build_device(len(ty), xyz.data_ptr(), ty.data_ptr(), box, 0, 0, maps.data_ptr(), nb, stream)
    keep, jobs = [], []
    for i, (na, T) in enumerate([(14, 3), (37, 10), (22, 6)]):
        lig = synth.ligand(na, T, 80 + i, center=rec.pocket_center)
        blob = dsdp.dsdp_ligand_pack(lig)
        nx = 7 + dsdp.dsdp_ligand_blob_info(blob)["n_torsions"]
        d = dict(blob=blob, dblob=torch.from_numpy(blob.copy()).to(dev),
                 conf=torch.zeros((40, nx), dtype=torch.float32, device=dev),
                 e=torch.zeros(40, dtype=torch.float32, device=dev), n=torch.zeros(1, dtype=torch.int32, device=dev),
                 chain=torch.zeros(4, dtype=torch.int32, device=dev),
                 score=torch.zeros(4, dtype=torch.float64, device=dev))
        n = [int(np.ceil(14.0 / 0.375))] * 3
        j = dsdp.dsdp_job_device()
        j.grid = dsdp.grid_view(maps.data_ptr(), n, [rec.pocket_center[a] - (n[a] - 1) * 0.375 / 2 for a in range(3)],
                                0.375)
        j.receptor = dsdp.dsdp_receptor(len(ty), xyz.data_ptr(), ty.data_ptr())
        j.h_blob, j.d_blob = blob.ctypes.data, d["dblob"].data_ptr()
        j.params = dsdp.make_params(n_chains=40, n_mc_steps=3, n_opt_iters=15, seed=i, top_k=4)
        for a in range(3):
            j.box_lo[a] = rec.pocket_center[a] - 7.0
            j.box_size[a] = 14.0
        j.d_chain_best_conf, j.d_chain_best_e = d["conf"].data_ptr(), d["e"].data_ptr()
        j.d_out_n, j.d_out_chain, j.d_out_score = d["n"].data_ptr(), d["chain"].data_ptr(), d["score"].data_ptr()
        jobs.append(j)
        keep.append(d)
    plan = dsdp.dsdp_plan_create(None, jobs, dsdp.DSDP_PLAN_PERSISTENT, 1)
    try:
        dsdp.dsdp_plan_launch(plan, stream)
        torch.cuda.synchronize()
        eager = [{k: v.cpu().numpy().copy() for k, v in d.items() if torch.is_tensor(v)} for d in keep]
        for d in keep:
            for k in ("conf", "e", "score"):
                d[k].zero_()
        cap = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=cap):
            dsdp.dsdp_plan_launch(plan, cap.cuda_stream)
        for _ in range(2):
            graph.replay()
            torch.cuda.synchronize()
            for d, ref in zip(keep, eager):
                for k in ("conf", "e", "n", "chain", "score"):
                    assert np.array_equal(d[k].cpu().numpy(), ref[k]), k
    finally:
        dsdp.dsdp_plan_destroy(None, plan)


def test_plans_on_concurrent_streams_match_a_serial_launch(ctx):
    """Steps in flight on several streams, as the pipelined bench runs them: each
    stream builds its own maps and launches its own plan of the same jobs while
    the others run; every stream's results equal one serial launch's, bitwise."""
    dev = torch.device("cuda", 0)
    rec = synth.receptor(1500, 73)
    box = dsdp.make_box(rec.pocket_center, 14.0, 0.375)
    nb = dsdp.dsdp_grid_map_bytes(box)
    xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
    ty = torch.from_numpy(rec.xs_type.copy()).to(dev)
    ligs = [synth.ligand(na, T, 90 + i, center=rec.pocket_center) for i, (na, T) in enumerate([(18, 4), (30, 8), (41, 11)])]
    blobs = [dsdp.dsdp_ligand_pack(lig) for lig in ligs]
    dblobs = [torch.from_numpy(b.copy()).to(dev) for b in blobs]
    n = [int(np.ceil(14.0 / 0.375))] * 3
    origin = [rec.pocket_center[a] - (n[a] - 1) * 0.375 / 2 for a in range(3)]

    def make_slot():
        maps = torch.empty(nb, dtype=torch.uint8, device=dev)
        keep, jobs = [], []
        for i, (blob, dblob) in enumerate(zip(blobs, dblobs)):
            nx = 7 + dsdp.dsdp_ligand_blob_info(blob)["n_torsions"]
            d = dict(conf=torch.zeros((48, nx), dtype=torch.float32, device=dev),
                     e=torch.zeros(48, dtype=torch.float32, device=dev),
                     n=torch.zeros(1, dtype=torch.int32, device=dev),
                     chain=torch.zeros(4, dtype=torch.int32, device=dev),
                     score=torch.zeros(4, dtype=torch.float64, device=dev))
            j = dsdp.dsdp_job_device()
            j.grid = dsdp.grid_view(maps.data_ptr(), n, origin, 0.375)
            j.receptor = dsdp.dsdp_receptor(len(ty), xyz.data_ptr(), ty.data_ptr())
            j.h_blob, j.d_blob = blob.ctypes.data, dblob.data_ptr()
            j.params = dsdp.make_params(n_chains=48, n_mc_steps=3, n_opt_iters=15, seed=20 + i, top_k=4)
            for a in range(3):
                j.box_lo[a] = rec.pocket_center[a] - 7.0
                j.box_size[a] = 14.0
            j.d_chain_best_conf, j.d_chain_best_e = d["conf"].data_ptr(), d["e"].data_ptr()
            j.d_out_n, j.d_out_chain, j.d_out_score = d["n"].data_ptr(), d["chain"].data_ptr(), d["score"].data_ptr()
            jobs.append(j)
            keep.append(d)
        return dict(maps=maps, jobs=jobs, keep=keep, plan=dsdp.dsdp_plan_create(None, jobs, dsdp.DSDP_PLAN_PERSISTENT, 0))

    def step(slot, st):
        dsdp.dsdp_grid_build_device(len(ty), xyz.data_ptr(), ty.data_ptr(), box, 0, 0, slot["maps"].data_ptr(), nb, st)
        dsdp.dsdp_plan_launch(slot["plan"], st)

    slots = [make_slot() for _ in range(3)]
    try:
        step(slots[0], torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref = [{k: v.cpu().numpy().copy() for k, v in d.items()} for d in slots[0]["keep"]]
        streams = [torch.cuda.Stream() for _ in slots]
        for d in (d for sl in slots for d in sl["keep"]):
            for v in d.values():
                v.zero_()
        torch.cuda.synchronize()
        for k in range(6):  # two rounds over the three streams, all in flight together
            step(slots[k % 3], streams[k % 3].cuda_stream)
        torch.cuda.synchronize()
        for sl in slots:
            for d, r in zip(sl["keep"], ref):
                for key in ("conf", "e", "n", "chain", "score"):
                    assert np.array_equal(d[key].cpu().numpy(), r[key]), key
    finally:
        for sl in slots:
            dsdp.dsdp_plan_destroy(None, sl["plan"])
