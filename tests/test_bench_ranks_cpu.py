"""The multi-GPU bench path (independent replicas, one per GPU: the docking
jobs shard with no exchange step) on two CPU ranks over gloo: replicas dock
disjoint systems, the timing is the slowest rank's, rates add up."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 95.5][rank]  # ms: rank 0 is the slower one
        e2e = [10.0, 12.5][rank]  # systems/s
        slowest = bench.max_over_ranks(dist, elapsed, "cpu")
        total = bench.sum_over_ranks(dist, e2e, "cpu")
        out[rank] = (slowest, total, bench.replica_seeds(rank, 16),
                     bench.job_throughput(world, 16, 10, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        slowest, total, seeds, value = res[r]
        assert slowest == 120.0  # max over ranks, on every rank
        assert total == 22.5  # e2e rates add up
        assert value == pytest.approx(2 * 16 * 10 / 0.120)  # all ranks' systems over the slowest time
    assert not set(res[0][2]) & set(res[1][2])  # replicas dock disjoint systems
    assert len(set(res[0][2])) == 16


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(None, 7.0, "cpu") == 7.0
    assert bench.sum_over_ranks(None, 3.0, "cpu") == 3.0
    assert bench.job_throughput(1, 16, 10, 500.0) == pytest.approx(320.0)


def test_fixed_tile_config_numbering():
    """bench.py --tile-config takes the autotuner's numbering (1 + variant + 4
    log2 W + 12 work queue); each maps back to the plan's tile_config (1 +
    variant + 4 log2 W) and flags, and to its description."""

    class Flags:
        DSDP_PLAN_PERSISTENT = 1

    seen = set()
    for chosen in range(1, 25):
        var, w, queue = (chosen - 1) % 4, 1 << (((chosen - 1) % 12) // 4), chosen > 12
        tc = bench.plan_tile_config(chosen)
        assert 1 <= tc <= 12 and (tc - 1) % 4 == var and 1 << ((tc - 1) // 4) == w
        assert bench.plan_flags(Flags, chosen) == (1 if queue else 0)
        text = bench.describe_tile_config(chosen)
        assert text.startswith(f"{(128, 96, 80, 72)[var]} regs, {w} chain") and text.endswith("work queue") == queue
        seen.add((tc, queue))
    assert len(seen) == 24


def test_committed_chain_kernel_capture_is_consistent():
    """The committed ncu record of the chain kernel: each captured launch
    configuration internally consistent (DRAM bytes = read + write, instructions
    per evaluation = instructions / evaluations of the capture they came from),
    described as bench.py describes the configuration."""
    import json

    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "dock_chains_kernel_traffic.json")) as f:
        rec = json.load(f)
    caps = {c["tile_config"]: c for c in rec["captures"]}
    assert caps and all(1 <= k <= 24 for k in caps)
    for k, c in caps.items():
        assert c["chain_kernel"] == bench.describe_tile_config(k)
        assert c["dram_bytes_per_launch"] == c["dram_read_bytes"] + c["dram_write_bytes"]
        ins = c.get("instructions_small_case", c)
        assert abs(ins["warp_instructions_per_eval"] - ins["warp_instructions"] / ins["evaluations"]) < 0.1
        assert c["warp_instructions_per_eval"] == ins["warp_instructions_per_eval"]
    assert rec["systems_per_launch"] == 32 and len(rec["sources_sha256"]) == 64
