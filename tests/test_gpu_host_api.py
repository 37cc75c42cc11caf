"""The handle API on a GPU: the job lifecycle and status codes (a queued job
polled without waiting is pending, a timed wait that expires is a TIMEOUT,
cancelling a queued or a running job drops it -- its one poll reports
CANCELLED, the next NOT_FOUND --, a finished job is released by its poll, a
grid larger than the context's budget is refused with OUT_OF_MEMORY), and a
context working on the caller's stream."""
import numpy as np
import pytest

from paper_2303_09916_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_09916_gb300 import dsdp  # noqa: E402


def test_job_lifecycle_pending_cancel_release():
    # one stream and one job in flight: the second job waits in the queue
    ctx = dsdp.dsdp_create(0, n_streams=1, max_inflight_jobs=1)
    rec = synth.receptor(2000, 5)
    lig = synth.ligand(20, 4, 5, center=rec.pocket_center)
    grid = dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(rec.pocket_center, 20.0, 0.375))
    try:
        long_p = dsdp.make_params(n_chains=2048, n_mc_steps=600, n_opt_iters=100, seed=1, top_k=3)
        short_p = dsdp.make_params(n_chains=64, n_mc_steps=5, n_opt_iters=20, seed=2, top_k=3)
        long_bufs = dsdp.result_buffers(lig.n_atoms, lig.n_torsions, long_p)
        a = dsdp.dsdp_dock_submit(ctx, grid, lig, long_p)
        b = dsdp.dsdp_dock_submit(ctx, grid, lig, short_p)
        bufs_b = dsdp.result_buffers(lig.n_atoms, lig.n_torsions, short_p)
        assert dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=0) is None  # queued behind a
        with pytest.raises(dsdp.DSDPError) as ei:  # a timed wait that expires
            dsdp.dsdp_dock_poll(ctx, a, long_bufs, wait_ms=1)
        assert ei.value.status == dsdp.DSDP_ERR_TIMEOUT
        s = dsdp.dsdp_get_stats(ctx)
        assert s["queued"] + s["running"] == 2
        assert dsdp.dsdp_dock_cancel(ctx, b) == dsdp.DSDP_OK  # still queued: dropped at once
        with pytest.raises(dsdp.DSDPError) as ei:
            dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=-1)
        assert ei.value.status == dsdp.DSDP_ERR_CANCELLED
        with pytest.raises(dsdp.DSDPError) as ei:
            dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=0)
        assert ei.value.status == dsdp.DSDP_ERR_NOT_FOUND
        assert dsdp.dsdp_get_stats(ctx)["running"] == 1
        assert dsdp.dsdp_dock_cancel(ctx, a) == dsdp.DSDP_OK  # running: dropped when its batch retires
        with pytest.raises(dsdp.DSDPError) as ei:
            dsdp.dsdp_dock_poll(ctx, a, long_bufs, wait_ms=-1)
        assert ei.value.status == dsdp.DSDP_ERR_CANCELLED
        c = dsdp.dsdp_dock_submit(ctx, grid, lig, short_p)
        r = dsdp.dsdp_dock_poll(ctx, c, bufs_b, wait_ms=-1)
        assert r is not None and r["n_out"] >= 1 and np.isfinite(r["score"][: r["n_out"]]).all()
        with pytest.raises(dsdp.DSDPError) as ei:  # released by its poll
            dsdp.dsdp_dock_poll(ctx, c, bufs_b, wait_ms=0)
        assert ei.value.status == dsdp.DSDP_ERR_NOT_FOUND
        s = dsdp.dsdp_get_stats(ctx)
        assert s["cancelled"] == 2 and s["completed"] >= 1 and s["queued"] == 0 and s["running"] == 0
        assert s["bytes_in_use"] <= dsdp.dsdp_grid_info(grid)["map_bytes"] + (16 << 20)  # the jobs' memory is back
    finally:
        dsdp.dsdp_grid_free(ctx, grid)
        dsdp.dsdp_destroy(ctx)


def test_grid_over_the_budget_is_refused():
    ctx = dsdp.dsdp_create(0, mem_budget_bytes=32 << 20)
    try:
        rec = synth.receptor(2000, 6)
        with pytest.raises(dsdp.DSDPError) as ei:  # 80^3 x 8 FP32 score + gradient maps: 65.5 MB
            dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(rec.pocket_center, 30.0, 0.375))
        assert ei.value.status == dsdp.DSDP_ERR_OUT_OF_MEMORY
        # a grid that fits is built in the same context
        g = dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(rec.pocket_center, 12.0, 0.375))
        dsdp.dsdp_grid_free(ctx, g)
    finally:
        dsdp.dsdp_destroy(ctx)


def test_context_on_the_callers_stream():
    """A context given the caller's stream runs its grid builds and scoring on it
    (same results as a context of its own) and leaves the stream alive."""
    rec = synth.receptor(1500, 8)
    lig = synth.ligand(14, 3, 8, center=rec.pocket_center)
    box = dsdp.make_box(rec.pocket_center, 14.0, 0.375)
    rng = np.random.default_rng(0)
    confs = np.zeros((16, 7 + lig.n_torsions))
    confs[:, :3] = rec.pocket_center + rng.uniform(-2, 2, (16, 3))
    q = rng.normal(size=(16, 4))
    confs[:, 3:7] = q / np.linalg.norm(q, axis=1, keepdims=True)
    confs[:, 7:] = rng.uniform(-3, 3, (16, lig.n_torsions))
    out = []
    user = torch.cuda.Stream()
    for stream in (None, user.cuda_stream):
        ctx = dsdp.dsdp_create(0, stream=stream)
        try:
            g = dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, box)
            out.append(dsdp.dsdp_score_eval(ctx, g, lig, confs))
            dsdp.dsdp_grid_free(ctx, g)
        finally:
            dsdp.dsdp_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    with torch.cuda.stream(user):  # still a valid stream after dsdp_destroy
        x = torch.ones(8, device="cuda") * 2
    user.synchronize()
    assert float(x.sum()) == 16.0
