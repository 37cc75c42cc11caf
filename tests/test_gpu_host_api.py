"""The handle API's job lifecycle and status codes on a GPU: a queued job
polled without waiting is pending, cancelling it frees it (its one poll
reports CANCELLED, the next NOT_FOUND), a finished job is released by its poll,
and a grid larger than the context's budget is refused with OUT_OF_MEMORY."""
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
        long_p = dsdp.make_params(n_chains=2048, n_mc_steps=200, n_opt_iters=100, seed=1, top_k=3)
        short_p = dsdp.make_params(n_chains=64, n_mc_steps=5, n_opt_iters=20, seed=2, top_k=3)
        a = dsdp.dsdp_dock_submit(ctx, grid, lig, long_p)
        b = dsdp.dsdp_dock_submit(ctx, grid, lig, short_p)
        bufs_b = dsdp.result_buffers(lig.n_atoms, lig.n_torsions, short_p)
        assert dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=0) is None  # queued behind a
        assert dsdp.dsdp_dock_poll(ctx, a, dsdp.result_buffers(lig.n_atoms, lig.n_torsions, long_p),
                                   wait_ms=1) is None  # still running after 1 ms
        s = dsdp.dsdp_get_stats(ctx)
        assert s["queued"] + s["running"] == 2
        assert dsdp.dsdp_dock_cancel(ctx, b) == dsdp.DSDP_OK  # still queued: cancelled
        with pytest.raises(dsdp.DSDPError) as ei:
            dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=-1)
        assert ei.value.status == dsdp.DSDP_ERR_CANCELLED
        with pytest.raises(dsdp.DSDPError) as ei:
            dsdp.dsdp_dock_poll(ctx, b, bufs_b, wait_ms=0)
        assert ei.value.status == dsdp.DSDP_ERR_NOT_FOUND
        r = dsdp.dsdp_dock_poll(ctx, a, dsdp.result_buffers(lig.n_atoms, lig.n_torsions, long_p), wait_ms=-1)
        assert r is not None and r["n_out"] >= 1 and np.isfinite(r["score"][: r["n_out"]]).all()
        with pytest.raises(dsdp.DSDPError) as ei:  # released by its poll
            dsdp.dsdp_dock_poll(ctx, a, dsdp.result_buffers(lig.n_atoms, lig.n_torsions, long_p), wait_ms=0)
        assert ei.value.status == dsdp.DSDP_ERR_NOT_FOUND
        s = dsdp.dsdp_get_stats(ctx)
        assert s["cancelled"] == 1 and s["completed"] >= 1 and s["queued"] == 0 and s["running"] == 0
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
