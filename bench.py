#!/usr/bin/env python3
"""Throughput of the docking hot path on GB300 (one JSON line on rank 0).

Workload "typical-4k": each docked system is a 4,000-atom synthetic receptor
with a 30 A box at 0.375 A (80^3 x 8 FP32 score+gradient maps) and a 30-atom
ligand with 8 torsions, docked by 384 Monte Carlo chains x 40 steps of BFGS
(100 iterations) and rescored in FP64 (top 9).  One step = `--batch` such
systems, each with its own receptor, end to end: grid build, chains, FP64
rescoring and top-k.

  value  systems/s with inputs resident on the device (device-pointer API,
         caller-owned memory), timed with CUDA events over exactly K steps;
         consecutive steps rotate over four streams (--pipeline-depth), each with its own
         maps, outputs and plan, so that a step's grid builds and chains fill
         the SMs the previous step's last wave of chains leaves idle
         (--no-pipeline: one stream).  `serial` is the same K steps on one
         stream; the stage times and rooflines come from that pass
  e2e    systems/s through the host API (dsdp_grid_build / dsdp_dock_submit_many
         / dsdp_dock_poll) with host arrays, copies included; three steps
         in flight (--e2e-window: the next steps' requests go in before this
         step's results are read back)
  roofline  dock_chains_kernel against the maximum of its three bounds per
         launch: corner-gather bytes at the measured HBM copy peak, FP32 FMA
         work at the FP32 peak, special-function work at the MUFU peak; the
         binding one gives `bound`, `achieved` and `frac` (also the fraction of
         the L2-gather microbenchmark, --gather-bench alone)
  the same line also carries the other workloads of the method: one job per
  launch, the uneven batch under a CUDA graph, BF16 / FP16 maps with their
  error, Barzilai-Borwein, the plain-2k workload, receptor voxel features
  and grid maps at 4,000 and 8,000 atoms, the atoms-per-lane boundary, a
  short Poisson serving run, the search-region
  and grid-mode variants, and the autotuner's time for every configuration
  --impl reference   the FP64 CPU oracle on the host cores (whole systems)

N > 1 (torchrun): independent replicas, one per GPU; value sums all ranks'
systems over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_REC, BOX, SPACING, N_LIG, T_LIG = 4000, 30.0, 0.375, 30, 8
N_CHAINS, N_STEPS, N_ITERS, TOP_K = 384, 40, 100, 9


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=32, help="systems per step")
    p.add_argument("--optimizer", default="bfgs", choices=["bfgs", "bb"])
    p.add_argument("--map-dtype", default="f32", choices=["f32", "bf16", "f16"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=9)
    p.add_argument("--e2e-batch-chains", type=int, default=-1,
                   help="the host API's largest batch in chains (dsdp_create_params.max_batch_chains): -1 = one "
                        "step's chains (default), 0 = the library's default")
    p.add_argument("--serve", action="store_true",
                   help="run the serving workload (Poisson arrivals, 8 receptors) and print its JSON line instead")
    p.add_argument("--serve-requests", type=int, default=4000)
    p.add_argument("--serve-streams", type=int, default=8, help="batches in flight (one per stream)")
    p.add_argument("--no-forms", dest="forms", action="store_false",
                   help="skip the one-job-per-launch and uneven-batch (CUDA graph) measurements")
    p.add_argument("--gather-bench", action="store_true",
                   help="run the L2-gather microbenchmark alone on one typical-4k system's maps and print its JSON line")
    p.add_argument("--sweep", action="store_true",
                   help="copies x steps sweep of the typical-4k system (the paper's Table 1 grid) and print its JSON line")
    p.add_argument("--no-pipeline", dest="pipeline", action="store_false",
                   help="time the device-resident steps on one stream only (no overlap of consecutive steps)")
    p.add_argument("--pipeline-depth", type=int, default=4, help="streams (steps in flight) of the pipelined pass")
    p.add_argument("--e2e-window", type=int, default=3,
                   help="steps in flight through the host API (the end-to-end pass; 1 with --no-pipeline)")
    p.add_argument("--tile-config", type=int, default=-1,
                   help="chain kernel launch configuration: -1 autotune (default); 1..24 fixed, numbered as the "
                        "autotuner reports them: 1 + variant (0: 128 registers, 1: 96, 2: 80, 3: 72) + 4 log2(chains "
                        "per CTA) + 12 work queue")
    args = p.parse_args()
    if args.pipeline_depth < 1:
        p.error("--pipeline-depth must be at least 1")
    if args.e2e_window < 1:
        p.error("--e2e-window must be at least 1")
    return args


def replica_seeds(rank, batch):
    """Seeds of the systems rank `rank` docks: the replicas share no system."""
    return [1000 * rank + b for b in range(batch)]


def max_over_ranks(dist, value, device):
    """The slowest rank's time (every rank gets it)."""
    import torch

    if not dist:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device):
    """A per-rank rate summed over the ranks (every rank gets it)."""
    import torch

    if not dist:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def job_throughput(world, systems_per_rank_step, steps, slowest_ms):
    """Whole-job systems/s: every rank's systems over the slowest rank's time."""
    return world * systems_per_rank_step * steps / (slowest_ms * 1e-3)


def systems(rank, batch):
    from paper_2303_09916_gb300 import synth

    out = []
    for seed in replica_seeds(rank, batch):
        rec = synth.receptor(N_REC, seed)
        lig = synth.ligand(N_LIG, T_LIG, seed, center=rec.pocket_center)
        out.append((seed, rec, lig))
    return out


def plan_tile_config(chosen):
    """dsdp_plan_create's tile_config (1 + variant + 4 log2 W) of an autotuner choice."""
    return 1 + (chosen - 1) % 12


def plan_flags(dsdp, chosen):
    """The plan flags of an autotuner choice: the persistent work queue or none."""
    return dsdp.DSDP_PLAN_PERSISTENT if chosen > 12 else 0


def describe_tile_config(chosen):
    """The autotuner's choice (1 + variant + 4 log2 W + 12 persistent) in words."""
    if not 1 <= chosen <= 24:
        return "?"
    c = chosen - 1
    regs, warps, queue = (128, 96, 80, 72)[c % 4], 1 << ((c % 12) // 4), c >= 12
    return f"{regs} regs, {warps} chain{'s' if warps > 1 else ''}/CTA" + (", work queue" if queue else "")


def flops_per_eval(n_atoms, n_pairs, n_bodies):
    # algorithmic work of one score+gradient evaluation: trilinear gather and
    # weights 45 FMA per atom, kinematics + back-propagation 30 flop per atom and
    # 40 per body, 40 flop per intra pair
    return n_atoms * (2 * 45 + 30) + n_pairs * 40 + n_bodies * 40


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(power))}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Sources that define the chain kernel; the committed ncu traffic figure is used
# only while their hash matches the one recorded with it.
CHAIN_SOURCES = ["chain_device.cuh", "device_common.cuh", "dock_kernels.cuh", "dsdp_internal.h", "launch.cu",
                 "launch.h", "ligand_pack.cpp"]


def chain_kernel_capture(batch, map_dtype, chain_kernel):
    """The committed ncu figures of the chain kernel (DRAM bytes per launch of the
    bench's workload, warp instructions per evaluation), or None when the kernel
    sources changed since they were taken, the workload differs or this run's
    launch configuration (register budget, chains per CTA, work queue) is not
    the captured one."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "dock_chains_kernel_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    for name in CHAIN_SOURCES:
        with open(os.path.join(ROOT, "paper_2303_09916_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec.get("sources_sha256") or batch != rec.get("systems_per_launch") or map_dtype != "f32":
        return None
    for cap in rec.get("captures", []):
        if cap.get("chain_kernel") == chain_kernel:
            return cap
    return None


def mufu_per_eval(n_pairs, n_bodies):
    # special-function (MUFU) operations of one evaluation: per intra pair a
    # reciprocal square root and two exp2; per torsion body sin and cos of the
    # half angle; one reciprocal square root normalising the orientation
    return 3 * n_pairs + 2 * (n_bodies - 1) + 1


def mufu_peak_per_s(sm_mhz):
    # 152 SMs x 16 special-function results per clock (4 per SM sub-partition)
    return 152 * 16 * sm_mhz * 1e6


def chain_roofline(gather_bytes, flops, mufu_ops, chain_s, gather_gbs, peaks, peaks_src, sm_mhz, capture):
    """The chain kernel's roofline as the maximum of its three bounds -- corner
    gathers at the measured HBM copy bandwidth, FP32 FMA work at the FP32 peak,
    special-function work at the MUFU peak -- per launch: `bound` names the
    binding one, `achieved` its algorithmic work / the launch's event-timed
    duration, `frac` = achieved / peak.  The gather bound is also given against
    the L2-gather microbenchmark (the same random 8-corner reads, no arithmetic)."""
    hbm = float(peaks["hbm_gbs"]) * 1e9
    bounds = {"gather_hbm": gather_bytes / hbm, "fp32_fma": flops / (fp32_peak_tflops(sm_mhz) * 1e12),
              "mufu": mufu_ops / mufu_peak_per_s(sm_mhz)}
    binding = max(bounds, key=bounds.get)
    if binding == "gather_hbm":
        out = {"bound": "hbm", "achieved": gather_bytes / chain_s / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
               "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peaks_src})"}
    elif binding == "fp32_fma":
        out = {"bound": "alu", "achieved": flops / chain_s / 1e12, "peak": fp32_peak_tflops(sm_mhz),
               "unit": "TFLOP/s", "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"}
    else:
        out = {"bound": "alu", "achieved": mufu_ops / chain_s / 1e12, "peak": mufu_peak_per_s(sm_mhz) / 1e12,
               "unit": "Tops/s (MUFU)", "peak_source": f"derived: 152 SMs x 16 MUFU x {sm_mhz:.0f} MHz"}
    out["frac"] = out["achieved"] / out["peak"]
    out.update({"kernel": "dock_chains_kernel", "binding": binding,
                "traffic": capture["dram_bytes_per_launch"] if capture else None,
                "traffic_unit": "DRAM bytes per launch (ncu)",
                "algorithmic": {"gather_bytes": gather_bytes, "fp32_flop": flops, "mufu_ops": mufu_ops},
                "bounds_ms": {k: 1e3 * v for k, v in bounds.items()}, "launch_ms": 1e3 * chain_s,
                "frac_of_gather_microbench": gather_bytes / chain_s / 1e9 / gather_gbs,
                "gather_microbench_gbs": gather_gbs})
    return out


def issue_peak_per_s(sm_mhz):
    # 152 SMs x 4 schedulers x one warp instruction per cycle
    return 152 * 4 * sm_mhz * 1e6


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def gather_microbench(dsdp, torch, dev, g_view, dtype, stream, npts=1 << 20, reps=16):
    """The L2-gather roofline: 1 M threads x 16 random 8-corner gathers (one map
    type each) over the maps of one system, no arithmetic; algorithmic bytes /
    event-timed duration (GB/s), 5 launches after 3 untimed."""
    sptr = stream.cuda_stream
    rng = np.random.default_rng(0)
    pts = (np.array(g_view.origin) + rng.uniform(0, (np.array(g_view.n) - 1) * g_view.spacing, size=(npts, 3))).astype(
        np.float32)
    d_pts = torch.from_numpy(pts).to(dev)
    d_ty = torch.from_numpy(rng.integers(0, 8, npts).astype(np.uint8)).to(dev)
    d_out = torch.empty(npts, dtype=torch.float32, device=dev)
    for _ in range(3):
        dsdp.dsdp_gather_bench_device(g_view, d_pts.data_ptr(), d_ty.data_ptr(), npts, reps, d_out.data_ptr(), sptr)
    ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ga.record(stream)
    for _ in range(5):
        dsdp.dsdp_gather_bench_device(g_view, d_pts.data_ptr(), d_ty.data_ptr(), npts, reps, d_out.data_ptr(), sptr)
    gb.record(stream)
    torch.cuda.synchronize()
    return 5 * npts * reps * (128 if dtype == 0 else 64) / (ga.elapsed_time(gb) * 1e-3) / 1e9


def run_gather_bench(args):
    """The gather microbenchmark alone on the first typical-4k system's maps
    (the command the committed ncu capture of gather_bench_kernel runs)."""
    import torch
    from paper_2303_09916_gb300 import dsdp

    dev = 0
    torch.cuda.set_device(dev)
    (seed, rec, lig), = systems(0, 1)
    dtype = {"f32": dsdp.DSDP_MAP_F32, "bf16": dsdp.DSDP_MAP_BF16, "f16": dsdp.DSDP_MAP_F16}[args.map_dtype]
    j, keep = make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dtype, N_CHAINS, N_STEPS, N_ITERS,
                              TOP_K)
    stream = torch.cuda.current_stream()
    build_grid(dsdp, keep["grid"], dtype, stream.cuda_stream)
    gbs = gather_microbench(dsdp, torch, dev, j.grid, dtype, stream)
    return {"metric": "random 8-corner map gathers, algorithmic GB/s", "value": gbs, "unit": "GB/s",
            "map_dtype": args.map_dtype, "maps_bytes": int(keep["grid"]["maps"].numel()),
            "points": 1 << 20, "repeats": 16}


# ---------------------------------------------------------------- device-resident path
def run_device(args, rank, world, dev, dist):
    """The device-resident step (grid builds, chains, FP64 rescoring + top-k of
    args.batch systems), timed twice: serially on one stream (stage times and the
    kernel rooflines come from this pass) and pipelined, consecutive steps
    rotating over --pipeline-depth streams with their own maps and outputs so that a
    step's grid builds and chains fill the SMs the previous step's last wave of
    chains leaves idle (the headline throughput; each step still does all of its
    work)."""
    import torch
    from paper_2303_09916_gb300 import dsdp

    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    dtype = {"f32": dsdp.DSDP_MAP_F32, "bf16": dsdp.DSDP_MAP_BF16, "f16": dsdp.DSDP_MAP_F16}[args.map_dtype]
    opt = dsdp.DSDP_OPT_BFGS if args.optimizer == "bfgs" else dsdp.DSDP_OPT_BB
    sysl = systems(rank, args.batch)
    shared = []  # per system: receptor, ligand blob, box and grid geometry (read-only, shared by the slots)
    for seed, rec, lig in sysl:
        box = dsdp.make_box(rec.pocket_center, BOX, SPACING)
        blob = dsdp.dsdp_ligand_pack(lig)
        n = [int(np.ceil(BOX / SPACING))] * 3
        shared.append(dict(seed=seed, rec=rec, box=box, blob=blob, info=dsdp.dsdp_ligand_blob_info(blob),
                           d_xyz=torch.from_numpy(rec.xyz.copy()).to(dev),
                           d_type=torch.from_numpy(rec.xs_type.copy()).to(dev),
                           d_blob=torch.from_numpy(blob.copy()).to(dev), n=n,
                           origin=[rec.pocket_center[a] - (n[a] - 1) * SPACING / 2 for a in range(3)],
                           nbytes=dsdp.dsdp_grid_map_bytes(box, dtype, dsdp.DSDP_GRID_EQ4)))
    lig_info = [sh["info"] for sh in shared]

    def make_slot():
        """Maps, outputs and job descriptors of one in-flight step."""
        jobs, maps, outs_l = [], [], []
        for sh in shared:
            rec = sh["rec"]
            d_maps = torch.empty(sh["nbytes"], dtype=torch.uint8, device=dev)
            nx = 7 + sh["info"]["n_torsions"]
            outs = dict(conf=torch.empty((N_CHAINS, nx), dtype=torch.float32, device=dev),
                        e=torch.empty(N_CHAINS, dtype=torch.float32, device=dev),
                        evals=torch.zeros(N_CHAINS, dtype=torch.int32, device=dev),
                        n=torch.zeros(1, dtype=torch.int32, device=dev),
                        chain=torch.zeros(TOP_K, dtype=torch.int32, device=dev),
                        score=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                        inter=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                        intra=torch.zeros(TOP_K, dtype=torch.float64, device=dev),
                        oconf=torch.zeros((TOP_K, nx), dtype=torch.float64, device=dev),
                        coords=torch.zeros((TOP_K, N_LIG, 3), dtype=torch.float32, device=dev))
            j = dsdp.dsdp_job_device()
            j.grid = dsdp.grid_view(d_maps.data_ptr(), sh["n"], sh["origin"], SPACING, dtype, dsdp.DSDP_GRID_EQ4)
            j.receptor = dsdp.dsdp_receptor(N_REC, sh["d_xyz"].data_ptr(), sh["d_type"].data_ptr())
            j.h_blob = sh["blob"].ctypes.data
            j.d_blob = sh["d_blob"].data_ptr()
            j.params = dsdp.make_params(n_chains=N_CHAINS, n_mc_steps=N_STEPS, n_opt_iters=N_ITERS, optimizer=opt,
                                        seed=sh["seed"], top_k=TOP_K)
            for a in range(3):
                j.box_lo[a] = rec.pocket_center[a] - BOX / 2
                j.box_size[a] = BOX
            j.d_chain_best_conf = outs["conf"].data_ptr()
            j.d_chain_best_e = outs["e"].data_ptr()
            j.d_chain_evals = outs["evals"].data_ptr()
            j.d_out_n = outs["n"].data_ptr()
            j.d_out_chain = outs["chain"].data_ptr()
            j.d_out_score = outs["score"].data_ptr()
            j.d_out_inter = outs["inter"].data_ptr()
            j.d_out_intra = outs["intra"].data_ptr()
            j.d_out_conf = outs["oconf"].data_ptr()
            j.d_out_coords = outs["coords"].data_ptr()
            jobs.append(j)
            maps.append(d_maps)
            outs_l.append(outs)
        return dict(jobs=jobs, maps=maps, outs=outs_l)

    def build_grids(slot, st):
        for sh, d_maps in zip(shared, slot["maps"]):
            dsdp.dsdp_grid_build_device(N_REC, sh["d_xyz"].data_ptr(), sh["d_type"].data_ptr(), sh["box"], dtype,
                                        dsdp.DSDP_GRID_EQ4, d_maps.data_ptr(), d_maps.numel(), st)

    slots = [make_slot() for _ in range(args.pipeline_depth if args.pipeline else 1)]
    plan = dsdp.dsdp_plan_create(None, slots[0]["jobs"], 0, 0)
    build_grids(slots[0], sptr)
    autotune_ms = None
    if args.tile_config < 0:  # register budget, chains per CTA, work queue
        tile_config, autotune_ms = dsdp.dsdp_plan_autotune(plan, sptr, 2, with_times=True)
    else:
        dsdp.dsdp_plan_destroy(None, plan)
        plan = dsdp.dsdp_plan_create(None, slots[0]["jobs"], plan_flags(dsdp, args.tile_config),
                                     plan_tile_config(args.tile_config))
        tile_config = args.tile_config
    plans = [plan] + [dsdp.dsdp_plan_create(None, sl["jobs"], plan_flags(dsdp, tile_config), plan_tile_config(tile_config))
                      for sl in slots[1:]]
    n_plan_kernels = dsdp.dsdp_plan_kernel_count(plan)
    flushes = [torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev) for _ in slots]  # > 129 MB L2

    def step(i, st, evs=None):
        if evs:
            evs[0].record(torch.cuda.current_stream())
        build_grids(slots[i], st)
        if evs:
            evs[1].record(torch.cuda.current_stream())
        dsdp.dsdp_plan_launch_stage(plans[i], dsdp.DSDP_STAGE_CHAINS, st)
        if evs:
            evs[2].record(torch.cuda.current_stream())
        dsdp.dsdp_plan_launch_stage(plans[i], dsdp.DSDP_STAGE_RESCORE, st)
        if evs:
            evs[3].record(torch.cuda.current_stream())

    for _ in range(args.warmup):
        flushes[0].zero_()
        step(0, sptr)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    # serial pass: one stream, stage events
    t0.record(stream)
    for k in range(args.steps):
        flushes[0].zero_()
        step(0, sptr, evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    serial_ms = max_over_ranks(dist, t0.elapsed_time(t1), dev)
    elapsed_ms = serial_ms
    if args.pipeline:
        # pipelined pass: step k on stream k % depth with slot k % depth
        streams = [torch.cuda.Stream(device=dev) for _ in slots]
        for k in range(len(slots)):  # untimed: one step per slot and stream
            with torch.cuda.stream(streams[k]):
                flushes[k].zero_()
                step(k, streams[k].cuda_stream)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        p0.record(stream)
        for s in streams:
            s.wait_event(p0)
        for k in range(args.steps):
            i = k % len(slots)
            with torch.cuda.stream(streams[i]):
                flushes[i].zero_()
                step(i, streams[i].cuda_stream)
        for s in streams:
            stream.wait_stream(s)
        p1.record(stream)
        torch.cuda.synchronize()
        elapsed_ms = max_over_ranks(dist, p0.elapsed_time(p1), dev)
    clk = clocks.stop()
    grid_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    chain_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    rescore_ms = float(np.mean([e[2].elapsed_time(e[3]) for e in evs]))
    evals = [int(o["evals"].sum().item()) for o in slots[0]["outs"]]
    total_evals = sum(evals)
    # every slot docked the same systems with the same seeds: the same evaluations
    same = all([int(o["evals"].sum().item()) for o in sl["outs"]] == evals for sl in slots[1:])
    flops = sum(ev * flops_per_eval(li["n_atoms"], li["n_pairs"], li["n_bodies"]) for ev, li in zip(evals, lig_info))
    mufu = sum(ev * mufu_per_eval(li["n_pairs"], li["n_bodies"]) for ev, li in zip(evals, lig_info))
    gather_bytes = sum(ev * li["n_atoms"] * (128 if dtype == 0 else 64) for ev, li in zip(evals, lig_info))
    results_ok = same and all(int(o["n"].item()) >= 1 and bool(torch.isfinite(o["score"][: int(o["n"].item())]).all())
                              for sl in slots for o in sl["outs"])
    jobs = slots[0]["jobs"]
    gather_gbs = gather_microbench(dsdp, torch, dev, jobs[0].grid, dtype, stream)  # the first system's maps
    for pl in plans:
        dsdp.dsdp_plan_destroy(None, pl)
    return dict(tile_config=tile_config, autotune_ms=autotune_ms, elapsed_ms=elapsed_ms, serial_ms=serial_ms,
                grid_ms=grid_ms, chain_ms=chain_ms,
                rescore_ms=rescore_ms,
                total_evals=total_evals, flops=flops, mufu=mufu, gather_bytes=gather_bytes, clocks=clk,
                launches_per_step=args.batch + n_plan_kernels, results_ok=results_ok, gather_gbs=gather_gbs)


# ---------------------------------------------------------------- other forms of the same work
def make_device_job(dsdp, torch, dev, rec, lig, seed, box_size, spacing, dtype, n_chains, n_steps, n_iters, top_k,
                    grid=None, sites=None, mode=0, coords=False, center=None, optimizer=0):
    """Device buffers and a dsdp_job_device for one docking job (caller-owned memory);
    box_size: edge length(s) of the box (scalar or per axis) around `center`
    (default: the receptor's pocket centre);
    sites: binding-site points of the adaptive search space (None: the whole box);
    mode: DSDP_GRID_EQ4 (score + gradient maps) or DSDP_GRID_EQ3 (score maps);
    coords: also return the top poses' heavy-atom coordinates (input atom order)."""
    size = np.broadcast_to(np.asarray(box_size, dtype=np.float64), (3,))
    c = np.asarray(rec.pocket_center if center is None else center, dtype=np.float64)
    box = dsdp.make_box(c, size, spacing)
    if grid is None:
        nbytes = dsdp.dsdp_grid_map_bytes(box, dtype, mode)
        grid = dict(box=box, mode=mode, maps=torch.empty(nbytes, dtype=torch.uint8, device=dev),
                    xyz=torch.from_numpy(rec.xyz.copy()).to(dev), type=torch.from_numpy(rec.xs_type.copy()).to(dev))
    blob = dsdp.dsdp_ligand_pack(lig)
    info = dsdp.dsdp_ligand_blob_info(blob)
    nx = 7 + info["n_torsions"]
    keep = dict(grid=grid, blob=blob, d_blob=torch.from_numpy(blob.copy()).to(dev), info=info,
                conf=torch.empty((n_chains, nx), dtype=torch.float32, device=dev),
                e=torch.empty(n_chains, dtype=torch.float32, device=dev),
                evals=torch.zeros(n_chains, dtype=torch.int32, device=dev),
                n=torch.zeros(1, dtype=torch.int32, device=dev),
                chain=torch.zeros(top_k, dtype=torch.int32, device=dev),
                score=torch.zeros(top_k, dtype=torch.float64, device=dev))
    n = [int(np.ceil(size[a] / spacing)) for a in range(3)]
    j = dsdp.dsdp_job_device()
    j.grid = dsdp.grid_view(grid["maps"].data_ptr(), n, [c[a] - (n[a] - 1) * spacing / 2 for a in range(3)], spacing,
                            dtype, grid.get("mode", 0))
    j.receptor = dsdp.dsdp_receptor(len(rec.xs_type), grid["xyz"].data_ptr(), grid["type"].data_ptr())
    j.h_blob = blob.ctypes.data
    j.d_blob = keep["d_blob"].data_ptr()
    j.params = dsdp.make_params(n_chains=n_chains, n_mc_steps=n_steps, n_opt_iters=n_iters, seed=seed, top_k=top_k,
                                site_points=sites, optimizer=optimizer)
    if sites is not None:
        keep["sites"] = torch.from_numpy(np.ascontiguousarray(sites, dtype=np.float32)).to(dev)
        j.d_site_points = keep["sites"].data_ptr()
    for a in range(3):
        j.box_lo[a] = c[a] - size[a] / 2
        j.box_size[a] = size[a]
    j.d_chain_best_conf, j.d_chain_best_e = keep["conf"].data_ptr(), keep["e"].data_ptr()
    j.d_chain_evals = keep["evals"].data_ptr()
    j.d_out_n, j.d_out_chain, j.d_out_score = keep["n"].data_ptr(), keep["chain"].data_ptr(), keep["score"].data_ptr()
    if coords:
        keep["coords"] = torch.zeros((top_k, info["n_atoms"], 3), dtype=torch.float32, device=dev)
        j.d_out_coords = keep["coords"].data_ptr()
    return j, keep


def build_grid(dsdp, grid, dtype, sptr):
    dsdp.dsdp_grid_build_device(len(grid["type"]), grid["xyz"].data_ptr(), grid["type"].data_ptr(), grid["box"],
                                dtype, grid.get("mode", 0), grid["maps"].data_ptr(), grid["maps"].numel(), sptr)


def run_one_job_per_launch(args, rank, dev, steps):
    """The plain form: each system alone -- its grid, then a one-job plan -- one after another."""
    import torch
    from paper_2303_09916_gb300 import dsdp

    sptr = torch.cuda.current_stream().cuda_stream
    dtype = {"f32": dsdp.DSDP_MAP_F32, "bf16": dsdp.DSDP_MAP_BF16, "f16": dsdp.DSDP_MAP_F16}[args.map_dtype]
    items = []
    for seed, rec, lig in systems(rank, args.batch):
        j, keep = make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dtype, N_CHAINS, N_STEPS, N_ITERS,
                                  TOP_K)
        items.append((dsdp.dsdp_plan_create(None, [j], 0, 1), keep))
    lat = []

    def one_pass(record):
        for plan, keep in items:
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            build_grid(dsdp, keep["grid"], dtype, sptr)
            dsdp.dsdp_plan_launch(plan, sptr)
            b.record()
            if record:
                lat.append((a, b))

    one_pass(False)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(True), torch.cuda.Event(True)
    t0.record()
    for _ in range(steps):
        one_pass(True)
    t1.record()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in lat]
    for plan, _ in items:
        dsdp.dsdp_plan_destroy(None, plan)
    return dict(systems_per_s=steps * len(items) / (t0.elapsed_time(t1) * 1e-3),
                latency_p50_ms=float(np.percentile(ms, 50)), latency_p99_ms=float(np.percentile(ms, 99)))


def run_variants(args, rank, dev, steps=2):
    """The typical-4k batch docked in variants of the method, each reporting the
    systems/s of the chain + rescoring stages and the mean top-1 FP64 score
    (lower is better):
      search_region: initial positions from the whole 30 A box (cube) or from
        the box intersected with 7 A balls around 100 synthetic binding-site
        points in the pocket (shape; Sec. 2 third modification);
      grid_mode: score + gradient maps interpolated (Eq. 4, 128 B gathered per
        atom) or score maps only with the gradient of the interpolant (Eq. 3,
        32 B per atom).
    Each variant also redocks the 18 open synthetic pockets of redock_success
    (cube: 30 A boxes; shape: with site points; grid modes: known-site box and
    30 A boxes with site points)."""
    import torch
    from paper_2303_09916_gb300 import dsdp, synth

    sptr = torch.cuda.current_stream().cuda_stream
    dtype = {"f32": dsdp.DSDP_MAP_F32, "bf16": dsdp.DSDP_MAP_BF16, "f16": dsdp.DSDP_MAP_F16}[args.map_dtype]
    variants = [("search_region", "cube", False, dsdp.DSDP_GRID_EQ4), ("search_region", "shape", True, dsdp.DSDP_GRID_EQ4),
                ("grid_mode", "eq4", False, dsdp.DSDP_GRID_EQ4), ("grid_mode", "eq3", False, dsdp.DSDP_GRID_EQ3)]
    out = {"search_region": {"site_points": "100 per system, uniform within 6 A of the pocket centre; 7 A balls"},
           "grid_mode": {}}
    for group, name, use_sites, mode in variants:
        jobs, keeps = [], []
        for seed, rec, lig in systems(rank, args.batch):
            sites = synth.site_points(rec, 100, seed) if use_sites else None
            j, keep = make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dtype, N_CHAINS, N_STEPS,
                                      N_ITERS, TOP_K, sites=sites, mode=mode)
            build_grid(dsdp, keep["grid"], dtype, sptr)
            jobs.append(j)
            keeps.append(keep)
        plan = dsdp.dsdp_plan_create(None, jobs, 0, 0)
        dsdp.dsdp_plan_launch(plan, sptr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(steps):
            dsdp.dsdp_plan_launch(plan, sptr)
        b.record()
        torch.cuda.synchronize()
        dsdp.dsdp_plan_destroy(None, plan)
        top1 = [float(k["score"][0].item()) for k in keeps]
        evals = sum(int(k["evals"].sum().item()) for k in keeps)
        sec = a.elapsed_time(b) * 1e-3 / steps
        out[group][name] = dict(systems_per_s=len(jobs) / sec, evals_per_s=evals / sec,
                                evals_per_system=evals / len(jobs), mean_top1_score=float(np.mean(top1)))
        # redocking accuracy of the variant (open synthetic pockets, 384 x 40)
        regions = {"cube": ("box30",), "shape": ("box30_sites",)}.get(name, ("site", "box30_sites"))
        out[group][name].update(redock_success(dsdp, torch, dev, sptr, N_CHAINS, N_STEPS, regions=regions, mode=mode))
        if group == "grid_mode":  # the paper pairs its Eq. 4 maps with Barzilai-Borwein
            bb = redock_success(dsdp, torch, dev, sptr, N_CHAINS, N_STEPS, regions=regions, mode=mode,
                                optimizer=dsdp.DSDP_OPT_BB)
            out[group][name].update({k + "_bb": v for k, v in bb.items()})
    return out


def run_uneven_graph(args, dev, steps=3):
    """Batched uneven launch: one 5,000-atom receptor, 256 ligands of 10-60 atoms and
    0-15 torsions, 128 chains each, all in one plan replayed from a captured CUDA graph."""
    import torch
    from paper_2303_09916_gb300 import dsdp, synth

    cfg = synth.config("uneven-5k", seed=0)
    rec = cfg.receptor
    sptr = torch.cuda.current_stream().cuda_stream
    jobs, keeps, grid = [], [], None
    for i, lig in enumerate(cfg.ligands):
        j, keep = make_device_job(dsdp, torch, dev, rec, lig, i, 26.0, SPACING, dsdp.DSDP_MAP_F32, cfg.n_chains,
                                  cfg.n_mc_steps, N_ITERS, TOP_K, grid=grid)
        grid = keep["grid"]
        jobs.append(j)
        keeps.append(keep)
    build_grid(dsdp, grid, dsdp.DSDP_MAP_F32, sptr)
    plan = dsdp.dsdp_plan_create(None, jobs, 0, 0)
    chosen, tune_ms = dsdp.dsdp_plan_autotune(plan, sptr, 2, with_times=True)
    cap = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=cap):
        dsdp.dsdp_plan_launch(plan, cap.cuda_stream)
    graph.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(True), torch.cuda.Event(True)
    a.record()
    for _ in range(steps):
        graph.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    evals = sum(int(k["evals"].sum().item()) for k in keeps)
    ok = all(int(k["n"].item()) >= 1 for k in keeps)
    dsdp.dsdp_plan_destroy(None, plan)
    atoms = [lig.n_atoms for lig in cfg.ligands]
    return dict(ligands_per_s=len(jobs) / (ms * 1e-3), ms_per_launch=ms, evals_per_s=evals / (ms * 1e-3),
                ligand_atoms=f"{min(atoms)}-{max(atoms)}", chains_per_ligand=cfg.n_chains,
                chain_kernel=describe_tile_config(chosen), launch="captured CUDA graph",
                autotune_ms_per_launch={describe_tile_config(k): round(v, 3) for k, v in sorted(tune_ms.items())},
                results_ok=ok)


def _timed_plan(dsdp, torch, items, dtype, sptr, steps, optimizer=0, tuned=None):
    """Grid builds + one plan launch (chains, FP64 rescoring, top-k) of all the
    items, timed over `steps` repetitions after one untimed run: seconds per step.
    tuned: a dict that receives the launch configuration the autotuner picks
    (the plan is autotuned first), or None (the plan's default configuration)."""
    plan = dsdp.dsdp_plan_create(None, [j for j, _ in items], 0, 0)
    try:
        for _, keep in items:
            build_grid(dsdp, keep["grid"], dtype, sptr)
        if tuned is not None:
            tuned["chain_kernel"] = describe_tile_config(dsdp.dsdp_plan_autotune(plan, sptr, 1))
        dsdp.dsdp_plan_launch(plan, sptr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(steps):
            for _, keep in items:
                build_grid(dsdp, keep["grid"], dtype, sptr)
            dsdp.dsdp_plan_launch(plan, sptr)
        b.record()
        torch.cuda.synchronize()
    finally:
        dsdp.dsdp_plan_destroy(None, plan)
    return a.elapsed_time(b) * 1e-3 / steps


def run_voxel_features(dsdp, torch, synth, dev, sptr, reps=20):
    """Receptor voxel features (36^3 x 18, the binding-site network's input) of
    4,000- and 8,000-atom receptors: ms per receptor (CUDA events, `reps`
    launches after one untimed); the work is the surface test, n x 98 points
    against each atom's neighbours."""
    out = {}
    work = torch.empty(dsdp.dsdp_voxel_work_bytes(), dtype=torch.uint8, device=dev)
    vox = torch.empty((36, 36, 36, 18), dtype=torch.float32, device=dev)
    for n in (4000, 8000):
        rec = synth.receptor(n, 7)
        radius, feats = synth.receptor_voxel_inputs(rec)
        c = synth.protein_center(rec)
        d = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (rec.xyz, radius, feats)]

        def launch():
            dsdp.dsdp_voxelize_device(n, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(), c, vox.data_ptr(),
                                      work.data_ptr(), work.numel(), sptr)

        launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            launch()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out[f"atoms_{n}"] = dict(ms_per_receptor=ms, receptors_per_s=1e3 / ms,
                                 surface_atoms=int(vox[..., 17].sum().item()))
    return out


def run_grid_build(dsdp, torch, synth, dev, sptr, reps=10):
    """Receptor grid maps (Eq. 1, Eq. 4 maps; 80^3 x 8 FP32 nodes of (E, grad E)
    around the pocket) of 4,000- and 8,000-atom receptors: ms per receptor
    (CUDA events, `reps` launches after one untimed).  Each 8 x 8 x 4 brick of
    vertices scans every receptor atom for those within the cutoff of the
    brick, then sums the pair terms of the ones it kept: the scan grows with
    the receptor, the pair work with the atom density around the box."""
    out = {}
    for n in (4000, 8000):
        rec = synth.receptor(n, 7)
        box = dsdp.make_box(np.asarray(rec.pocket_center, dtype=np.float64), np.array([BOX] * 3), SPACING)
        maps = torch.empty(dsdp.dsdp_grid_map_bytes(box, dsdp.DSDP_MAP_F32, dsdp.DSDP_GRID_EQ4), dtype=torch.uint8,
                           device=dev)
        xyz = torch.from_numpy(rec.xyz.copy()).to(dev)
        typ = torch.from_numpy(rec.xs_type.copy()).to(dev)

        def launch():
            dsdp.dsdp_grid_build_device(n, xyz.data_ptr(), typ.data_ptr(), box, dsdp.DSDP_MAP_F32,
                                        dsdp.DSDP_GRID_EQ4, maps.data_ptr(), maps.numel(), sptr)

        launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _ in range(reps):
            launch()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        vertices = maps.numel() // (8 * 16)  # 8 map types x (E, grad E) FP32 per vertex
        out[f"atoms_{n}"] = dict(ms_per_receptor=ms, receptors_per_s=1e3 / ms, vertices=vertices,
                                 vertices_per_s=vertices * 1e3 / ms)
    return out


def run_configs(args, rank, dev, steps=2):
    """The other workloads of the method, each timed as grid builds + one plan
    launch (chains, FP64 rescoring, top-k) on one stream:
      map_dtype: the typical-4k batch with FP32, BF16 and FP16 maps (FP32
        accumulation), each plan autotuned first.  Error stated per dtype: each chain's best search energy
        against the same pose scored on FP32 maps by the FP32 score kernel (which
        matches the FP64 oracle within 1e-4 of the term scale), relative to
        max(|E|, 1), median / p95 / max over all chains; and the top-1 FP64
        score against the FP32-map run's (median |difference| over systems);
      optimizer_bb: the typical-4k batch with Barzilai-Borwein local
        optimisation (the paper's, Sec. 2 second modification; 100 iterations);
      plain_2k: the plain-method workload (2,000-atom receptor, 20 A box -> 54^3
        maps, 20-atom ligand with 4 torsions, 64 chains x 100 steps): one system
        per launch (its latency) and `--batch` systems per launch."""
    import torch
    from paper_2303_09916_gb300 import dsdp, synth

    sptr = torch.cuda.current_stream().cuda_stream
    sysl = systems(rank, args.batch)
    out = {}
    # ---- map storage precision
    runs = {}
    for name, dtype in (("f32", dsdp.DSDP_MAP_F32), ("bf16", dsdp.DSDP_MAP_BF16), ("f16", dsdp.DSDP_MAP_F16)):
        items = [make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dtype, N_CHAINS, N_STEPS, N_ITERS,
                                 TOP_K) for seed, rec, lig in sysl]
        tuned = {}
        sec = _timed_plan(dsdp, torch, items, dtype, sptr, steps, tuned=tuned)
        evals = sum(int(k["evals"].sum().item()) for _, k in items)
        runs[name] = (items, dict(systems_per_s=len(items) / sec, evals_per_s=evals / sec, **tuned))
    f32_items = runs["f32"][0]
    for name in ("bf16", "f16"):
        items, row = runs[name]
        rel, top1 = [], []
        for (j32, k32), (j, k) in zip(f32_items, items):
            e32 = torch.empty(N_CHAINS, dtype=torch.float32, device=dev)
            dsdp.dsdp_score_eval_device(j32.grid, k["blob"], k["d_blob"].data_ptr(), k["conf"].data_ptr(), N_CHAINS,
                                        e32.data_ptr(), 0, dsdp.DSDP_TERM_ALL, sptr)
            torch.cuda.synchronize()
            e_red = k["e"].cpu().numpy().astype(np.float64)
            e_ref = e32.cpu().numpy().astype(np.float64)
            rel.extend((np.abs(e_red - e_ref) / np.maximum(np.abs(e_ref), 1.0)).tolist())
            top1.append(abs(float(k["score"][0].item()) - float(k32["score"][0].item())))
        row["search_energy_rel_err_vs_f32_maps"] = dict(median=float(np.median(rel)),
                                                        p95=float(np.percentile(rel, 95)), max=float(np.max(rel)))
        row["top1_fp64_score_abs_diff_vs_f32_run_median"] = float(np.median(top1))
        row["rescoring"] = "FP64 gridless (exact for the reported poses)"
        out.setdefault("map_dtype", {})[name] = row
    out["map_dtype"]["f32"] = runs["f32"][1]
    del runs, f32_items
    # ---- Barzilai-Borwein (the paper's local optimiser)
    items = [make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dsdp.DSDP_MAP_F32, N_CHAINS, N_STEPS,
                             N_ITERS, TOP_K, optimizer=dsdp.DSDP_OPT_BB) for seed, rec, lig in sysl]
    sec = _timed_plan(dsdp, torch, items, dsdp.DSDP_MAP_F32, sptr, steps)
    evals = sum(int(k["evals"].sum().item()) for _, k in items)
    out["optimizer_bb"] = dict(systems_per_s=len(items) / sec, evals_per_s=evals / sec,
                               evals_per_system=evals / len(items),
                               mean_top1_score=float(np.mean([float(k["score"][0].item()) for _, k in items])))
    del items
    # ---- plain method, one system (2,000 atoms, 54^3 maps, 20 atoms / 4 torsions, 64 x 100)
    plain = []
    for b in range(args.batch):
        seed = 2000 + 1000 * rank + b
        rec = synth.receptor(2000, seed)
        plain.append((seed, rec, synth.ligand(20, 4, seed, center=rec.pocket_center)))
    items = [make_device_job(dsdp, torch, dev, rec, lig, seed, 20.0, SPACING, dsdp.DSDP_MAP_F32, 64, 100, N_ITERS,
                             TOP_K) for seed, rec, lig in plain]
    one = _timed_plan(dsdp, torch, items[:1], dsdp.DSDP_MAP_F32, sptr, 3)
    sec = _timed_plan(dsdp, torch, items, dsdp.DSDP_MAP_F32, sptr, steps)
    evals = sum(int(k["evals"].sum().item()) for _, k in items)
    out["voxel_features"] = run_voxel_features(dsdp, torch, synth, dev, sptr)
    out["grid_build"] = run_grid_build(dsdp, torch, synth, dev, sptr)
    out["plain_2k"] = dict(one_system_ms=1e3 * one, batched_systems_per_s=len(items) / sec,
                           evals_per_s=evals / sec, systems_per_launch=len(items),
                           workload="2,000-atom receptor, 20 A box (54^3 x 8 FP32 maps), 20-atom ligand / 4 "
                                    "torsions, 64 chains x 100 steps, top-9 FP64 rescoring")
    # ---- atoms per lane: ligands of 32 atoms run one atom per lane, 33 atoms two
    apl = {}
    for n_lig in (32, 33):
        items = []
        for seed, rec, _ in sysl[:16]:
            lig = synth.ligand(n_lig, T_LIG, seed, center=rec.pocket_center)
            items.append(make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dsdp.DSDP_MAP_F32,
                                         N_CHAINS, N_STEPS, N_ITERS, TOP_K))
        plan = dsdp.dsdp_plan_create(None, [j for j, _ in items], dsdp.DSDP_PLAN_NO_RESCORE, 0)
        try:
            for _, keep in items:
                build_grid(dsdp, keep["grid"], dsdp.DSDP_MAP_F32, sptr)
            chosen = dsdp.dsdp_plan_autotune(plan, sptr, 1)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            dsdp.dsdp_plan_launch(plan, sptr)
            b.record()
            torch.cuda.synchronize()
        finally:
            dsdp.dsdp_plan_destroy(None, plan)
        evals = sum(int(k["evals"].sum().item()) for _, k in items)
        pairs = sum(k["info"]["n_pairs"] for _, k in items) / len(items)
        sec = a.elapsed_time(b) * 1e-3
        apl[f"atoms_{n_lig}"] = dict(atoms_per_lane=1 if n_lig <= 32 else 2, evals_per_s=evals / sec,
                                     ns_per_eval=1e9 * sec / evals,
                                     mean_intra_pairs=pairs, chain_kernel=describe_tile_config(chosen))
    out["atoms_per_lane"] = dict(apl, note="16 typical-4k receptors; the same 8-torsion ligand shape at 32 atoms "
                                          "(one atom per lane) and 33 (two per lane); chain stage only")
    return out


# ---------------------------------------------------------------- copies x steps sweep
SWEEP = [(128, 20), (384, 40), (512, 40), (512, 200), (1024, 200), (2048, 200)]


def run_sweep(args, dev=0):
    """Typical-4k systems docked with the copies x MC-steps combinations of the
    paper's Table 1 (128 x 20 ... 2048 x 200): one system per launch (grid build,
    chains, rescoring: its latency) and `--batch` systems per launch (throughput)."""
    import torch
    from paper_2303_09916_gb300 import dsdp

    torch.cuda.set_device(dev)
    sptr = torch.cuda.current_stream().cuda_stream
    sysl = systems(0, args.batch)
    rows = []
    for chains, steps in SWEEP:
        items = [make_device_job(dsdp, torch, dev, rec, lig, seed, BOX, SPACING, dsdp.DSDP_MAP_F32, chains, steps,
                                 N_ITERS, TOP_K) for seed, rec, lig in sysl]
        for _, keep in items:
            build_grid(dsdp, keep["grid"], dsdp.DSDP_MAP_F32, sptr)
        # one system per launch: grid build + chains + rescoring, CUDA events
        j0, k0 = items[0]
        plan = dsdp.dsdp_plan_create(None, [j0], 0, 0)
        lat = []
        for r in range(3):
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            build_grid(dsdp, k0["grid"], dsdp.DSDP_MAP_F32, sptr)
            dsdp.dsdp_plan_launch(plan, sptr)
            b.record()
            torch.cuda.synchronize()
            if r:
                lat.append(a.elapsed_time(b))
        dsdp.dsdp_plan_destroy(None, plan)
        # the batch in one launch
        plan = dsdp.dsdp_plan_create(None, [j for j, _ in items], 0, 0)
        dsdp.dsdp_plan_launch(plan, sptr)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        for _, keep in items:
            build_grid(dsdp, keep["grid"], dsdp.DSDP_MAP_F32, sptr)
        dsdp.dsdp_plan_launch(plan, sptr)
        b.record()
        torch.cuda.synchronize()
        dsdp.dsdp_plan_destroy(None, plan)
        evals = sum(int(k["evals"].sum().item()) for _, k in items)
        row = dict(copies=chains, steps=steps, one_system_ms=float(np.mean(lat)),
                   batch_systems_per_s=len(items) / (a.elapsed_time(b) * 1e-3),
                   evals_per_system=evals / len(items),
                   mean_top1_score=float(np.mean([float(k["score"][0].item()) for _, k in items])))
        row.update(redock_success(dsdp, torch, dev, sptr, chains, steps))
        rows.append(row)
    return rows


REDOCK = [(12, 2), (16, 3), (20, 4), (24, 6), (28, 7), (30, 8)]


def redock_success(dsdp, torch, dev, sptr, chains, steps, n_ligands=18, regions=("box30", "box30_sites", "site"),
                   mode=0, optimizer=0):
    """Redocking with one copies x steps setting (the accuracy side of the paper's
    Table 1): ligands of 12-30 atoms in receptor shells built around their own
    poses and open on one side (synth.shell_receptor, a 60 degree mouth), all in
    one launch, in three search regions: 30 A cubes (chains starting anywhere
    must find the pocket and enter it), the same cubes intersected with 7 A
    balls around 100 binding-site points within 3 A of the pocket centre (the
    adaptive search space; stand-ins for the site network's points), and the
    paper's known-site box (the ligand's extent plus 4 A on every side).
    Reported per region: the fraction whose top
    pose lies within 2 A (and 5 A) heavy-atom RMSD of the pose the shell was
    built around, and the launch time.  mode: the grid maps (Eq. 4 or Eq. 3);
    optimizer: BFGS or Barzilai-Borwein."""
    from paper_2303_09916_gb300 import synth

    cases = []
    for i in range(n_ligands):
        na, t = REDOCK[i % len(REDOCK)]
        lig = synth.ligand(na, t, 200 + i)
        cases.append((lig, synth.shell_receptor(lig, 200 + i, mouth_deg=60.0), 200 + i))
    out = {}
    for tag in regions:
        items = []
        for lig, rec, seed in cases:
            sites = None
            if tag == "site":
                lo, hi = lig.xyz.min(axis=0) - 4.0, lig.xyz.max(axis=0) + 4.0
                size, center = hi - lo, (lo + hi) / 2
            else:
                size, center = BOX, None
                if tag == "box30_sites":  # the adaptive search space: 7 A balls around predicted points
                    sites = synth.site_points(rec, 100, seed, spread=3.0)
            items.append(make_device_job(dsdp, torch, dev, rec, lig, seed, size, SPACING, dsdp.DSDP_MAP_F32, chains,
                                         steps, N_ITERS, 1, coords=True, center=center, sites=sites, mode=mode,
                                         optimizer=optimizer))
        for _, keep in items:
            build_grid(dsdp, keep["grid"], dsdp.DSDP_MAP_F32, sptr)
        plan = dsdp.dsdp_plan_create(None, [j for j, _ in items], 0, 0)
        a, b = torch.cuda.Event(True), torch.cuda.Event(True)
        a.record()
        dsdp.dsdp_plan_launch(plan, sptr)
        b.record()
        torch.cuda.synchronize()
        dsdp.dsdp_plan_destroy(None, plan)
        rmsd = [float(np.sqrt(((k["coords"][0].cpu().numpy().astype(np.float64) - lig.xyz) ** 2).sum(-1).mean()))
                for (_, k), (lig, _, _) in zip(items, cases)]
        out[f"redock_{tag}"] = dict(success_2A=float(np.mean([r < 2.0 for r in rmsd])),
                                    success_5A=float(np.mean([r < 5.0 for r in rmsd])),
                                    median_rmsd=float(np.median(rmsd)), ms=a.elapsed_time(b), ligands=n_ligands)
    return out


# ---------------------------------------------------------------- serving (continuous batching)
def run_serving(args, n_requests=None, loads=(0.5, 0.8, 0.95)):
    """Poisson arrivals of docking requests over 8 resident receptors (2,000-8,000
    atoms, boxes 20-40 A, BF16 maps), ligands of 10-60 atoms and 0-15 torsions,
    64-384 chains x 40 steps each, admitted by a device-memory budget while other
    jobs run.  First the saturated throughput (everything queued at once), then
    offered loads of 0.5 / 0.8 / 0.95 of it; p50/p99 latency from submission to
    completion as the library measures it."""
    import torch
    from paper_2303_09916_gb300 import dsdp, synth

    rng = np.random.default_rng(0)
    recs = []
    for r in range(8):
        n = int(rng.integers(2000, 8001))
        rec = synth.receptor(n, 100 + r)
        recs.append((rec, float(rng.uniform(20.0, 40.0))))
    pool = []
    for i in range(64):
        pool.append(synth.ligand(int(rng.integers(10, 61)), int(rng.integers(0, 16)), 500 + i))
    n_req = n_requests or args.serve_requests
    reqs = [(int(rng.integers(0, 8)), int(rng.integers(0, len(pool))), int(rng.integers(64, 385))) for _ in range(n_req)]
    map_bytes = sum(dsdp.dsdp_grid_map_bytes(dsdp.make_box([0, 0, 0], b, SPACING), dsdp.DSDP_MAP_BF16) for _, b in recs)
    # grids (+ receptor copies) plus 48 MB for jobs: admission has to wait for memory as well as for slots
    budget = map_bytes + 8 * (1 << 20) + (48 << 20)
    ctx = dsdp.dsdp_create(0, mem_budget_bytes=budget, n_streams=args.serve_streams, max_inflight_jobs=64)
    out = {}
    try:
        grids = []
        for rec, b in recs:
            lig_center = rec.pocket_center
            grids.append(dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, dsdp.make_box(lig_center, b, SPACING),
                                              dsdp.DSDP_MAP_BF16))

        def run(rate):
            pend = []
            t0 = time.perf_counter()
            t_next = t0
            for k, (ri, li, nc) in enumerate(reqs):
                if rate:
                    t_next += rng.exponential(1.0 / rate)
                    while time.perf_counter() < t_next:
                        time.sleep(0.0002)
                params = dsdp.make_params(n_chains=nc, n_mc_steps=40, n_opt_iters=N_ITERS, seed=k, top_k=TOP_K)
                lig = pool[li]
                jid = dsdp.dsdp_dock_submit(ctx, grids[ri], lig, params)
                pend.append((jid, lig, params))
            lat, evals = [], 0
            for jid, lig, params in pend:
                bufs = dsdp.result_buffers(lig.n_atoms, lig.n_torsions, params, chains=False)
                r = dsdp.dsdp_dock_poll(ctx, jid, bufs, wait_ms=-1)
                lat.append(r["latency_ms"])
                evals += r["n_evals"]
            dt = time.perf_counter() - t0
            return dict(offered_per_s=rate, systems_per_s=len(reqs) / dt, evals_per_s=evals / dt,
                        latency_p50_ms=float(np.percentile(lat, 50)), latency_p99_ms=float(np.percentile(lat, 99)))

        sat = run(None)
        out["saturated"] = sat
        for f in loads:
            out[f"load_{f}"] = run(f * sat["systems_per_s"])
        st = dsdp.dsdp_get_stats(ctx)
        out["admission"] = {"budget_bytes": budget, "grid_bytes": map_bytes, "completed": st["completed"],
                            "failed": st["failed"]}
        for g in grids:
            dsdp.dsdp_grid_free(ctx, g)
    finally:
        dsdp.dsdp_destroy(ctx)
    torch.cuda.synchronize()
    return out


# ---------------------------------------------------------------- host API (end to end)
def run_e2e(args, rank, dev):
    import torch
    from paper_2303_09916_gb300 import dsdp

    dtype = {"f32": dsdp.DSDP_MAP_F32, "bf16": dsdp.DSDP_MAP_BF16, "f16": dsdp.DSDP_MAP_F16}[args.map_dtype]
    opt = dsdp.DSDP_OPT_BFGS if args.optimizer == "bfgs" else dsdp.DSDP_OPT_BB
    sysl = systems(rank, args.batch)
    blob_bytes = {seed: len(dsdp.dsdp_ligand_pack(lig)) for seed, rec, lig in sysl}  # counted, not timed
    # steps in flight: the next steps are submitted before this one is read back
    window = args.e2e_window if args.pipeline else 1
    batch_chains = args.batch * N_CHAINS if args.e2e_batch_chains < 0 else args.e2e_batch_chains
    ctx = dsdp.dsdp_create(dev, n_streams=8, max_inflight_jobs=max(16, window * args.batch),
                           max_batch_chains=batch_chains)
    h2d = d2h = 0
    latencies = []
    try:
        def submit_step(count):
            # the step's grids are queued first (asynchronous builds), then its
            # jobs in one dsdp_dock_submit_many call (ligands packed on several
            # host threads, queued together: the runtime takes them in few batches)
            nonlocal h2d
            t_sub, grids, jids, bufs, params = {}, [], [], [], []
            for seed, rec, lig in sysl:
                box = dsdp.make_box(rec.pocket_center, BOX, SPACING)
                t_sub[seed] = time.perf_counter()
                grids.append(dsdp.dsdp_grid_build(ctx, rec.xyz, rec.xs_type, box, dtype, dsdp.DSDP_GRID_EQ4))
                p = dsdp.make_params(n_chains=N_CHAINS, n_mc_steps=N_STEPS, n_opt_iters=N_ITERS, optimizer=opt,
                                     seed=seed, top_k=TOP_K)
                params.append(p)
                bufs.append(dsdp.result_buffers(lig.n_atoms, lig.n_torsions, p))
                if count:
                    h2d += rec.xyz.nbytes + rec.xs_type.nbytes + blob_bytes[seed]
            jids = dsdp.dsdp_dock_submit_many(ctx, grids, [lig for _, _, lig in sysl], params)
            return t_sub, grids, jids, bufs

        def finish_step(st, count):
            nonlocal d2h
            t_sub, grids, jids, bufs = st
            for (seed, *_), j, b in zip(sysl, jids, bufs):
                r = dsdp.dsdp_dock_poll(ctx, j, b, wait_ms=-1)
                if count:
                    latencies.append(time.perf_counter() - t_sub[seed])
                    d2h += sum(v.nbytes for k, v in b.items()) + 8
                assert r["n_out"] >= 1
            for g in grids:
                dsdp.dsdp_grid_free(ctx, g)

        finish_step(submit_step(False), False)
        torch.cuda.synchronize()
        batches0 = dsdp.dsdp_get_stats(ctx)["batches"]
        t = time.perf_counter()
        inflight = []
        for _ in range(args.e2e_steps):
            inflight.append(submit_step(True))
            if len(inflight) == window:
                finish_step(inflight.pop(0), True)
        while inflight:
            finish_step(inflight.pop(0), True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        batches = dsdp.dsdp_get_stats(ctx)["batches"] - batches0
    finally:
        dsdp.dsdp_destroy(ctx)
    return dict(value=args.e2e_steps * args.batch / dt, h2d=h2d // args.e2e_steps, d2h=d2h // args.e2e_steps,
                p50_ms=1e3 * float(np.percentile(latencies, 50)), p99_ms=1e3 * float(np.percentile(latencies, 99)),
                batches_per_step=batches / args.e2e_steps)


# ---------------------------------------------------------------- CPU oracle
def oracle_system(seed, rec, lig, n_threads, optimizer):
    """One whole system on the FP64 oracle: full grid maps, all chains, rescoring."""
    import oracle

    ol = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    size = np.array([BOX] * 3)
    t = time.perf_counter()
    g = oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, size, SPACING,
                          n_threads=n_threads)
    t_grid = time.perf_counter() - t
    dp = oracle.dock_params_array(N_STEPS, 0 if optimizer == "bfgs" else 1, 1.2, rec.pocket_center - BOX / 2, size)
    t = time.perf_counter()
    best, e_best, evals = oracle.dock(ol, g, 0, dp, seed, N_CHAINS, n_threads=n_threads,
                                      opt=dict(max_iters=N_ITERS))
    oracle.rescore_topk(ol, rec.xyz.astype(np.float64), rec.xs_type, best, TOP_K)
    t_dock = time.perf_counter() - t
    oracle_system.last_grid = g
    return t_grid, t_dock, float(evals.sum())


def oracle_single_thread(seed, rec, lig, optimizer, g, n_chains=16, box=9.0):
    """The oracle on one host thread, on a bounded sample of the same work: the
    grid maps of a 9 A box of the receptor (24^3 x 8) and 16 chains of the
    typical-4k search on its maps g; evaluations/s and grid vertices/s."""
    import oracle

    ol = oracle.Ligand(lig.xyz.astype(np.float64), lig.xs_type, lig.bonds, lig.rotatable)
    t = time.perf_counter()
    oracle.grid_build(rec.xyz.astype(np.float64), rec.xs_type, rec.pocket_center, np.array([box] * 3), SPACING,
                      n_threads=1)
    t_grid = time.perf_counter() - t
    n_vert = int(np.ceil(box / SPACING)) ** 3
    dp = oracle.dock_params_array(N_STEPS, 0 if optimizer == "bfgs" else 1, 1.2, rec.pocket_center - BOX / 2,
                                  np.array([BOX] * 3))
    t = time.perf_counter()
    _, _, evals = oracle.dock(ol, g, 0, dp, seed, n_chains, n_threads=1, opt=dict(max_iters=N_ITERS))
    t_dock = time.perf_counter() - t
    return {"evals_per_s": float(evals.sum()) / t_dock, "grid_vertices_per_s": n_vert / t_grid,
            "sample": f"{n_chains} chains of the typical-4k search; grid maps of a {box:.0f} A box ({n_vert} vertices)"}


def cpu_baseline(args):
    cores = os.cpu_count() or 1
    (seed, rec, lig), = systems(0, 1)
    t_grid, t_dock, evals = oracle_system(seed, rec, lig, cores, args.optimizer)
    return {"value": 1.0 / (t_grid + t_dock), "unit": "systems/s", "cores": cores, "kind": "oracle",
            "sample": f"one whole typical-4k system (80^3 x 8 FP64 maps, {N_CHAINS} chains x {N_STEPS} steps, "
                      f"rescoring), threads over vertices and chains",
            "grid_s": t_grid, "dock_s": t_dock, "evals_per_s": evals / t_dock,
            "single_thread": oracle_single_thread(seed, rec, lig, args.optimizer, oracle_system.last_grid)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sysl = systems(0, 1)
    seed, rec, lig = sysl[0]
    for _ in range(args.warmup):
        oracle_system(seed, rec, lig, cores, args.optimizer)
    times, evals_s = [], []
    for _ in range(args.steps):
        tg, td, ev = oracle_system(seed, rec, lig, cores, args.optimizer)
        times.append(tg + td)
        evals_s.append(ev / td)
    v = len(times) / sum(times)
    line = {"metric": "docked systems/s (typical-4k: 4k-atom receptor, 80^3 maps, 30-atom ligand, 384x40 MC+BFGS)",
            "value": v, "unit": "systems/s", "impl": "reference", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "typical-4k", "systems_per_step": 1, "runs_on": "host cores"},
            "cpu_baseline": {"value": v, "unit": "systems/s", "cores": cores, "kind": "oracle",
                             "sample": "one whole typical-4k system per step"},
            "evals_per_s": float(np.mean(evals_s)),
            "e2e": {"value": v, "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.gather_bench:
        import __graft_entry__

        __graft_entry__.build()
        print(json.dumps(run_gather_bench(args)), flush=True)
        return
    if args.sweep:
        import __graft_entry__

        __graft_entry__.build()
        rows = run_sweep(args)
        print(json.dumps({"metric": "typical-4k docking time vs copies x MC steps (paper Table 1 grid)", "n_gpus": 1,
                          "unit": "ms per system (one per launch) / systems/s (batched)",
                          "systems_per_batch": args.batch, "dtype": "f32", "data": "synthetic", "sweep": rows}),
              flush=True)
        return
    if args.serve:
        import __graft_entry__

        __graft_entry__.build()
        res = run_serving(args)
        print(json.dumps({"metric": "serving: docked systems/s and p50/p99 latency (8 receptors, Poisson arrivals)",
                          "unit": "systems/s", "value": res["saturated"]["systems_per_s"], "n_gpus": 1,
                          "requests": args.serve_requests, "streams": args.serve_streams,
                          "dtype": "f32 accumulation, bf16 maps",
                          "data": "synthetic", "serving": res}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    import torch

    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    r = run_device(args, rank, world, local, dist)
    e2e = run_e2e(args, rank, local) if args.e2e_steps > 0 else None
    single = run_one_job_per_launch(args, rank, local, 2) if args.forms else None
    uneven = run_uneven_graph(args, local) if args.forms and rank == 0 else None
    variants = run_variants(args, rank, local) if args.forms and rank == 0 else None
    configs = run_configs(args, rank, local) if args.forms and rank == 0 else None
    serving = run_serving(args, n_requests=400, loads=(0.8,)) if args.forms and rank == 0 else None
    e2e_total = sum_over_ranks(dist, e2e["value"] if e2e else 0.0, local)
    if e2e:
        e2e["value"] = e2e_total
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peaks, peaks_src = measured_peaks()
    value = job_throughput(world, args.batch, args.steps, r["elapsed_ms"])
    per_launch_s = r["chain_ms"] * 1e-3
    achieved_tflops = r["flops"] / per_launch_s / 1e12
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_tflops = fp32_peak_tflops(sm_mhz)
    capture = chain_kernel_capture(args.batch, args.map_dtype, describe_tile_config(r["tile_config"]))
    line = {
        "metric": "docked systems/s (typical-4k: 4k-atom receptor, 80^3 maps, 30-atom ligand, 384x40 MC+BFGS)",
        "value": value, "unit": "systems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["elapsed_ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "typical-4k", "systems_per_step": args.batch, "receptor_atoms": N_REC,
                   "grid": "80^3 x 8", "map_dtype": args.map_dtype, "ligand": f"{N_LIG} atoms / {T_LIG} torsions",
                   "chains": N_CHAINS, "mc_steps": N_STEPS, "opt_iters": N_ITERS, "optimizer": args.optimizer,
                   "top_k": TOP_K, "l2": "flushed before each step (256 MB write on the step's stream); each step builds 2.1 GB of maps", "parallelism": f"replicas x{world}",
                   "chain_kernel": describe_tile_config(r["tile_config"]),
                   "autotune_ms_per_launch": ({describe_tile_config(k): round(v, 3) for k, v in
                                               sorted(r["autotune_ms"].items())} if r["autotune_ms"] else None),
                   "pipeline": (f"{args.pipeline_depth} streams: consecutive steps overlap (own maps and outputs "
                                "per stream)"
                                if args.pipeline else "none: steps back to back on one stream")},
        "serial": {"value": job_throughput(world, args.batch, args.steps, r["serial_ms"]),
                   "ms_per_step": r["serial_ms"] / args.steps,
                   "note": "the same steps on one stream (stage_ms and the rooflines are from this pass)"},
        "evals_per_s": world * r["total_evals"] * args.steps / (r["elapsed_ms"] * 1e-3),
        "evals_per_step": r["total_evals"],
        "stage_ms": {"grid_build": r["grid_ms"], "chains": r["chain_ms"], "rescore_topk": r["rescore_ms"]},
        "roofline": chain_roofline(r["gather_bytes"], r["flops"], r["mufu"], per_launch_s, r["gather_gbs"], peaks,
                                   peaks_src, sm_mhz, capture),
        "fp32": {"achieved_tflops": achieved_tflops, "peak_tflops": peak_tflops,
                 "frac": achieved_tflops / peak_tflops},
        "issue": None if not capture else {
            "warp_instructions_per_eval": capture["warp_instructions_per_eval"],
            "achieved_per_s": capture["warp_instructions_per_eval"] * r["total_evals"] / per_launch_s,
            "peak_per_s": issue_peak_per_s(sm_mhz),
            "frac": capture["warp_instructions_per_eval"] * r["total_evals"] / per_launch_s / issue_peak_per_s(sm_mhz),
            "note": "instructions per evaluation from the committed ncu capture; evaluations and time measured here"},
        "gpu_launches": r["launches_per_step"] * args.steps,
        "clocks": r["clocks"],
        "results_ok": r["results_ok"],
    }
    if e2e:
        line["e2e"] = {"value": e2e["value"], "unit": "systems/s", "h2d_bytes_per_step": e2e["h2d"],
                       "d2h_bytes_per_step": e2e["d2h"], "latency_p50_ms": e2e["p50_ms"],
                       "latency_p99_ms": e2e["p99_ms"], "batches_per_step": e2e["batches_per_step"]}
    if single:
        line["forms"] = {"batched_plan": {"systems_per_s": value, "note": f"{args.batch} systems per launch"},
                         "one_job_per_launch": single,
                         "served_host_api": {"systems_per_s": e2e["value"] if e2e else None,
                                             "latency_p50_ms": e2e["p50_ms"] if e2e else None,
                                             "latency_p99_ms": e2e["p99_ms"] if e2e else None}}
    if uneven:
        line["uneven_5k_batch"] = uneven
    if variants:
        line.update(variants)
    if configs:
        line["configs"] = configs
    if serving:
        line["serving"] = dict(serving, workload="400 requests over 8 resident receptors (2,000-8,000 atoms, "
                                                 "20-40 A boxes, BF16 maps), ligands of 10-60 atoms / 0-15 "
                                                 "torsions, 64-384 chains x 40 steps; all queued at once "
                                                 "(saturated), then Poisson arrivals at 0.8 of it",
                               one_job_per_launch=single)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
