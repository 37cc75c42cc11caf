// Device-resident entry points of the C ABI: scoring a batch of
// conformations, and docking plans (chain kernels, FP64 rescoring, top-k)
// that can be enqueued repeatedly or captured into CUDA graphs.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "launch.h"

struct dsdp_plan {
  dsdp_ctx* ctx = nullptr;
  int n_jobs = 0;
  uint32_t flags = 0;
  int warps_per_cta = 1;
  int variant = 0;        // chain kernel register budget (0: 128, 1: 96)
  uint64_t tune_key = 0;  // shape key for the autotuner's choice
  int max_chains = 0;
  // one device arena holding job table, tiles, counters and scratch
  void* arena = nullptr;
  size_t arena_bytes = 0;
  struct Group {
    int fmt, apl, first_tile, n_tiles, blob_smem, max_atoms, max_torsions, max_pairs, apl_mask;
  };
  std::vector<Group> groups;
  void* d_jobs = nullptr;
  void* d_tiles = nullptr;
  void* d_rtiles = nullptr;
  int* d_counters = nullptr;
  int n_rtiles = 0;
  std::vector<int> job_fmt, job_chains;  // to lay chain tiles out again for another warps_per_cta
  int sms = 148;
};

namespace dsdp {

dsdp_status normalize_params(const dsdp_dock_params* in, dsdp_dock_params* out) {
  if (!in) return set_error(DSDP_ERR_INVALID_ARG, "dock params NULL");
  *out = *in;
  if (out->n_chains == 0) out->n_chains = 384;
  if (out->n_mc_steps == 0) out->n_mc_steps = 40;
  if (out->n_opt_iters == 0) out->n_opt_iters = 100;
  if (out->temperature == 0.0) out->temperature = 1.2;
  if (out->top_k == 0) out->top_k = 9;
  if (out->rmsd_dedup == 0.0) out->rmsd_dedup = 1.0;
  if (out->site_radius == 0.f) out->site_radius = 7.0f;
  if (out->n_chains < 1 || out->n_chains > DSDP_MAX_CHAINS)
    return set_error(DSDP_ERR_INVALID_ARG, "n_chains %d outside 1..%d", out->n_chains, DSDP_MAX_CHAINS);
  if (out->n_mc_steps < 0 || out->n_mc_steps > 100000) return set_error(DSDP_ERR_INVALID_ARG, "n_mc_steps out of range");
  if (out->trace < 0 || out->trace > 2) return set_error(DSDP_ERR_INVALID_ARG, "trace must be 0, 1 or 2");
  if (out->n_opt_iters < 0 || out->n_opt_iters > 100000)
    return set_error(DSDP_ERR_INVALID_ARG, "n_opt_iters out of range");
  if (out->optimizer != DSDP_OPT_BFGS && out->optimizer != DSDP_OPT_BB)
    return set_error(DSDP_ERR_INVALID_ARG, "unknown optimizer %d", out->optimizer);
  if (!(out->temperature > 0.0)) return set_error(DSDP_ERR_INVALID_ARG, "temperature must be positive");
  if (out->top_k < 1 || out->top_k > DSDP_MAX_TOP_K)
    return set_error(DSDP_ERR_INVALID_ARG, "top_k %d outside 1..%d", out->top_k, DSDP_MAX_TOP_K);
  if (!(out->rmsd_dedup >= 0.0)) return set_error(DSDP_ERR_INVALID_ARG, "rmsd_dedup must be >= 0");
  if (out->n_site_points < 0 || out->n_site_points > DSDP_MAX_SITE_POINTS)
    return set_error(DSDP_ERR_INVALID_ARG, "n_site_points %d outside 0..%d", out->n_site_points,
                     DSDP_MAX_SITE_POINTS);
  if (!(out->site_radius > 0.f) || !isfinite(out->site_radius))
    return set_error(DSDP_ERR_INVALID_ARG, "site_radius must be positive");
  return DSDP_OK;
}

static cudaError_t launch_chains_dispatch(int fmt, const ChainLaunch& a, cudaStream_t st) {
  switch (fmt) {
    case 0: return launch_chains_fmt0(a, st);
    case 1: return launch_chains_fmt1(a, st);
    case 2: return launch_chains_fmt2(a, st);
    case 3: return launch_chains_fmt3(a, st);
    case 4: return launch_chains_fmt4(a, st);
    default: return launch_chains_fmt5(a, st);
  }
}

static cudaError_t launch_score_dispatch(int fmt, const ScoreLaunch& a, cudaStream_t st) {
  switch (fmt) {
    case 0: return launch_score_fmt0(a, st);
    case 1: return launch_score_fmt1(a, st);
    case 2: return launch_score_fmt2(a, st);
    case 3: return launch_score_fmt3(a, st);
    case 4: return launch_score_fmt4(a, st);
    default: return launch_score_fmt5(a, st);
  }
}

static dsdp_status check_view(const dsdp_grid_view* g) {
  if (!g || !g->d_maps) return set_error(DSDP_ERR_INVALID_ARG, "grid view or maps NULL");
  if (g->dtype < 0 || g->dtype > 2 || g->mode < 0 || g->mode > 1)
    return set_error(DSDP_ERR_INVALID_ARG, "grid view dtype/mode invalid");
  for (int a = 0; a < 3; ++a)
    if (g->n[a] < 2) return set_error(DSDP_ERR_INVALID_ARG, "grid needs >= 2 vertices per axis");
  if (!(g->spacing > 0.0)) return set_error(DSDP_ERR_INVALID_ARG, "grid spacing must be positive");
  if ((double)DSDP_NUM_MAP_TYPES * g->n[0] * g->n[1] * g->n[2] >= 2147483648.0)
    return set_error(DSDP_ERR_INVALID_ARG, "grid exceeds 2^31 nodes (32-bit map indices)");
  return DSDP_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Autotuner choices by plan shape: (format mask, atoms-per-lane, log2 of the
// chain count) -> (variant, persistent).  Written by dsdp_plan_autotune, read
// by plans created with tile_config 0.
struct TuneEntry {
  uint64_t key;
  int variant, persistent, warps;
};
static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;

static uint64_t tune_key(uint32_t fmt_mask, int apl, size_t chains) {
  int lg = 0;
  while ((size_t(1) << lg) < chains) ++lg;
  return ((uint64_t)fmt_mask << 16) | ((uint64_t)apl << 8) | (uint64_t)lg;
}

static bool tune_lookup(uint64_t key, int* variant, int* persistent, int* warps) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const TuneEntry& t : g_tune)
    if (t.key == key) {
      *variant = t.variant;
      *persistent = t.persistent;
      *warps = t.warps;
      return true;
    }
  return false;
}

static void tune_store(uint64_t key, int variant, int persistent, int warps) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (TuneEntry& t : g_tune)
    if (t.key == key) {
      t.variant = variant;
      t.persistent = persistent;
      t.warps = warps;
      return;
    }
  g_tune.push_back(TuneEntry{key, variant, persistent, warps});
}

// Chain tiles of W chains of one job, grouped by map format (one launch per
// format present); fills each group's tile range.
static void plan_tiles(dsdp_plan* P, int W, std::vector<Tile>& tiles) {
  tiles.clear();
  for (dsdp_plan::Group& g : P->groups) {
    g.first_tile = (int)tiles.size();
    for (int j = 0; j < P->n_jobs; ++j) {
      if (P->job_fmt[j] != g.fmt) continue;
      for (int c = 0; c < P->job_chains[j]; c += W)
        tiles.push_back(Tile{j, c, std::min(W, P->job_chains[j] - c), 0});
    }
    g.n_tiles = (int)tiles.size() - g.first_tile;
  }
}

static cudaError_t plan_use_warps(dsdp_plan* P, int W) {
  std::vector<Tile> tiles;
  plan_tiles(P, W, tiles);
  P->warps_per_cta = W;
  return tiles.empty() ? cudaSuccess
                       : cudaMemcpy(P->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
}

}  // namespace dsdp

using namespace dsdp;

extern "C" dsdp_status dsdp_score_eval_device(const dsdp_grid_view* grid, const void* h_blob, const void* d_blob,
                                              const float* d_conf, int32_t n_conf, float* d_energy, float* d_grad,
                                              uint32_t flags, void* stream) {
  dsdp_status s = check_view(grid);
  if (s != DSDP_OK) return s;
  int32_t n_atoms = 0, T = 0, P = 0, B = 0;
  s = dsdp_ligand_blob_info(h_blob, &n_atoms, &T, &P, &B);
  if (s != DSDP_OK) return s;
  if (!d_blob || !d_conf || n_conf < 0) return set_error(DSDP_ERR_INVALID_ARG, "score_eval_device arguments");
  if (n_conf == 0) return DSDP_OK;
  if ((flags & DSDP_TERM_ALL) == 0 || (flags & ~(uint32_t)DSDP_TERM_ALL))
    return set_error(DSDP_ERR_INVALID_ARG, "flags must select DSDP_TERM_INTER and/or DSDP_TERM_INTRA");
  ScoreLaunch a;
  a.map = map_view_of(grid);
  a.blob = (const uint8_t*)d_blob;
  a.conf = d_conf;
  a.n_conf = n_conf;
  a.energy = d_energy;
  a.grad = d_grad;
  a.flags = flags;
  a.apl = n_atoms <= 32 ? 1 : 2;
  a.blob_smem = (int)((const BlobHeader*)h_blob)->stage_bytes;
  a.scratch = scratch_layout(n_atoms, T, P, a.apl);
  return check_cuda(launch_score_dispatch(map_fmt(grid->dtype, grid->mode), a, (cudaStream_t)stream),
                    "score_eval_kernel launch");
}

extern "C" dsdp_status dsdp_plan_create(dsdp_ctx* ctx, int32_t n_jobs, const dsdp_job_device* jobs, uint32_t flags,
                                        int32_t tile_config, dsdp_plan** out) {
  if (!out) return set_error(DSDP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_jobs < 1 || !jobs) return set_error(DSDP_ERR_INVALID_ARG, "plan needs >= 1 job");
  if (tile_config < 0 || tile_config > 12) return set_error(DSDP_ERR_INVALID_ARG, "tile_config outside 0..12");
  std::vector<DevJob> dj(n_jobs);
  std::vector<int> fmt(n_jobs), apl(n_jobs), blob_bytes(n_jobs), pairs(n_jobs), atoms(n_jobs), tors(n_jobs);
  size_t scratch = 0;
  int max_chains = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const dsdp_job_device& J = jobs[j];
    dsdp_status s = check_view(&J.grid);
    if (s != DSDP_OK) return s;
    s = dsdp_ligand_blob_info(J.h_blob, &atoms[j], &tors[j], &pairs[j], nullptr);
    if (s != DSDP_OK) return s;
    if (!J.d_blob) return set_error(DSDP_ERR_INVALID_ARG, "job %d: d_blob NULL", j);
    dsdp_dock_params p;
    s = normalize_params(&J.params, &p);
    if (s != DSDP_OK) return s;
    if (!(flags & DSDP_PLAN_NO_RESCORE) && (J.receptor.n < 1 || !J.receptor.xyz || !J.receptor.xs_type))
      return set_error(DSDP_ERR_INVALID_ARG, "job %d: rescoring needs the receptor's device arrays", j);
    for (int a = 0; a < 3; ++a)
      if (!(J.box_size[a] >= 0.0) || !isfinite(J.box_lo[a]))
        return set_error(DSDP_ERR_INVALID_ARG, "job %d: search box invalid", j);
    if (p.trace && !J.d_trace) return set_error(DSDP_ERR_INVALID_ARG, "job %d: trace requested without d_trace", j);
    if (p.n_site_points > 0 && !J.d_site_points)
      return set_error(DSDP_ERR_INVALID_ARG, "job %d: n_site_points > 0 without d_site_points", j);
    fmt[j] = map_fmt(J.grid.dtype, J.grid.mode);
    apl[j] = atoms[j] <= 32 ? 1 : 2;
    blob_bytes[j] = (int)((const BlobHeader*)J.h_blob)->stage_bytes;
    max_chains = std::max(max_chains, p.n_chains);
    const int nx = 7 + tors[j];
    if (!J.d_chain_best_conf) scratch += up256(sizeof(float) * (size_t)p.n_chains * nx);
    if (!J.d_chain_best_e) scratch += up256(sizeof(float) * (size_t)p.n_chains);
    if (!J.d_chain_evals) scratch += up256(sizeof(uint32_t) * (size_t)p.n_chains);
    scratch += 3 * up256(sizeof(double) * (size_t)p.n_chains);
    scratch += up256(sizeof(double) * (size_t)p.n_chains * atoms[j] * 3);
    DevJob& d = dj[j];
    memset(&d, 0, sizeof(d));
    d.blob = (const uint8_t*)J.d_blob;
    d.maps = J.grid.d_maps;
    for (int a = 0; a < 3; ++a) {
      d.n[a] = J.grid.n[a];
      d.origin[a] = (float)J.grid.origin[a];
      d.box_lo[a] = (float)J.box_lo[a];
      d.box_size[a] = (float)J.box_size[a];
    }
    d.spacing = (float)J.grid.spacing;
    d.inv_spacing = (float)(1.0 / J.grid.spacing);
    d.dtype = J.grid.dtype;
    d.mode = J.grid.mode;
    d.n_chains = p.n_chains;
    d.n_steps = p.n_mc_steps;
    d.n_opt_iters = p.n_opt_iters;
    d.optimizer = p.optimizer;
    d.temperature = (float)p.temperature;
    d.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
    d.seed_hi = (uint32_t)(p.seed >> 32);
    d.chain_best_conf = J.d_chain_best_conf;
    d.chain_best_e = J.d_chain_best_e;
    d.chain_evals = J.d_chain_evals;
    d.trace = p.trace ? J.d_trace : nullptr;
    d.trace_starts = p.trace == 2;
    d.sites = p.n_site_points > 0 ? J.d_site_points : nullptr;
    d.n_sites = p.n_site_points;
    d.site_r2 = p.site_radius * p.site_radius;
    d.n_rec = J.receptor.n;
    d.rec_xyz = J.receptor.xyz;
    d.rec_type = J.receptor.xs_type;
    d.top_k = p.top_k;
    d.rmsd_dedup = (float)p.rmsd_dedup;
    d.out_n = J.d_out_n;
    d.out_chain = J.d_out_chain;
    d.out_score = J.d_out_score;
    d.out_inter = J.d_out_inter;
    d.out_intra = J.d_out_intra;
    d.out_conf = J.d_out_conf;
    d.out_coords = J.d_out_coords;
  }
  dsdp_plan* P = new dsdp_plan();
  P->ctx = ctx;
  P->n_jobs = n_jobs;
  P->flags = flags;
  P->max_chains = max_chains;
  P->sms = ctx_sm_count(ctx);
  // Groups by map format (one launch per format present); a CTA runs a tile of
  // W chains of one job (W = warps per CTA: 1, 2 or 4), staging the ligand once.
  P->job_fmt = fmt;
  P->job_chains.resize(n_jobs);
  size_t total_chains = 0;
  for (int j = 0; j < n_jobs; ++j) total_chains += (size_t)(P->job_chains[j] = dj[j].n_chains);
  for (int f = 0; f < 6; ++f) {
    dsdp_plan::Group g{f, 1, 0, 0, 0, 0, 0, 0, 0};
    bool any = false;
    for (int j = 0; j < n_jobs; ++j) {
      if (fmt[j] != f) continue;
      any = true;
      g.apl = std::max(g.apl, apl[j]);  // largest tile present: part of the autotuner key
      g.apl_mask |= apl[j];             // each job runs at its own tile (see dock_chains_kernel)
      g.blob_smem = std::max(g.blob_smem, blob_bytes[j]);
      g.max_atoms = std::max(g.max_atoms, atoms[j]);
      g.max_torsions = std::max(g.max_torsions, tors[j]);
      g.max_pairs = std::max(g.max_pairs, pairs[j]);
    }
    if (any) P->groups.push_back(g);
  }
  int W = 1;
  {
    uint32_t fmt_mask = 0;
    int apl_max = 1;
    for (const dsdp_plan::Group& g : P->groups) {
      fmt_mask |= 1u << g.fmt;
      apl_max = std::max(apl_max, g.apl);
    }
    P->tune_key = tune_key(fmt_mask, apl_max, total_chains);
    int var = 0, pers = (flags & DSDP_PLAN_PERSISTENT) ? 1 : 0;
    if (tile_config == 0) {
      // without a recorded choice: the 96-register kernel for plans of at least
      // two waves of 16 chains per SM, whose 20 resident warps per SM then issue
      // more per cycle (32 typical-4k systems 69.0 against 72.4 ms per launch at
      // 1 chain per CTA; the uneven 10-60-atom batch 307 - 309 against 317 - 319
      // ms at 4), else the 128-register kernel, whose fewer instructions per
      // evaluation win when the chains run latency-bound on a part-filled GPU
      // (one typical-4k system 17.3 against 19.1 ms; 32 plain-2k systems of 64
      // chains 1,011 against 938 systems/s).  Ligands above 32 atoms stage large
      // blobs, which tiles of 4 chains share (measured faster on mixed
      // batches); else 1 chain.
      var = total_chains >= (size_t)(2 * 16 * P->sms) ? 1 : 0;
      W = apl_max == 2 ? 4 : 1;
      if (tune_lookup(P->tune_key, &var, &pers, &W) && pers) P->flags |= DSDP_PLAN_PERSISTENT;
    } else {
      var = (tile_config - 1) % 4;
      W = 1 << ((tile_config - 1) / 4);
    }
    P->variant = var;
  }
  std::vector<Tile> tiles;
  plan_tiles(P, W, tiles);
  P->warps_per_cta = W;
  std::vector<Tile> rtiles;
  const int rw = rescore_tile_chains();
  for (int j = 0; j < n_jobs; ++j)
    for (int c = 0; c < dj[j].n_chains; c += rw) rtiles.push_back(Tile{j, c, std::min(rw, dj[j].n_chains - c), 0});
  P->n_rtiles = (int)rtiles.size();
  const size_t b_jobs = up256(sizeof(DevJob) * n_jobs), b_tiles = up256(sizeof(Tile) * total_chains),
               b_rtiles = up256(sizeof(Tile) * rtiles.size()), b_cnt = up256(sizeof(int) * 8);
  P->arena_bytes = b_jobs + b_tiles + b_rtiles + b_cnt + scratch;
  P->arena = ctx_alloc(ctx, P->arena_bytes, nullptr);
  if (!P->arena) {
    delete P;
    return set_error(DSDP_ERR_OUT_OF_MEMORY, "plan arena of %zu bytes", (size_t)(b_jobs + b_tiles + b_rtiles + scratch));
  }
  uint8_t* a = (uint8_t*)P->arena;
  P->d_jobs = a;
  P->d_tiles = a + b_jobs;
  P->d_rtiles = a + b_jobs + b_tiles;
  P->d_counters = (int*)(a + b_jobs + b_tiles + b_rtiles);
  uint8_t* sc = a + b_jobs + b_tiles + b_rtiles + b_cnt;
  for (int j = 0; j < n_jobs; ++j) {
    DevJob& d = dj[j];
    const int nx = 7 + tors[j];
    auto take = [&](size_t bytes) {
      uint8_t* p = sc;
      sc += up256(bytes);
      return p;
    };
    if (!d.chain_best_conf) d.chain_best_conf = (float*)take(sizeof(float) * (size_t)d.n_chains * nx);
    if (!d.chain_best_e) d.chain_best_e = (float*)take(sizeof(float) * (size_t)d.n_chains);
    if (!d.chain_evals) d.chain_evals = (uint32_t*)take(sizeof(uint32_t) * (size_t)d.n_chains);
    d.chain_score = (double*)take(sizeof(double) * (size_t)d.n_chains);
    d.chain_inter = (double*)take(sizeof(double) * (size_t)d.n_chains);
    d.chain_intra = (double*)take(sizeof(double) * (size_t)d.n_chains);
    d.chain_coords = (double*)take(sizeof(double) * (size_t)d.n_chains * atoms[j] * 3);
  }
  cudaError_t e = cudaMemcpy(P->d_jobs, dj.data(), sizeof(DevJob) * n_jobs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(P->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !rtiles.empty())
    e = cudaMemcpy(P->d_rtiles, rtiles.data(), sizeof(Tile) * rtiles.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ctx_free(ctx, P->arena, P->arena_bytes, nullptr);
    delete P;
    return check_cuda(e, "plan upload");
  }
  *out = P;
  return DSDP_OK;
}

extern "C" int32_t dsdp_plan_kernel_count(const dsdp_plan* P) {
  if (!P) return 0;
  int n = (int)P->groups.size();
  if (!(P->flags & DSDP_PLAN_NO_RESCORE)) n += 2;
  return n;
}

extern "C" dsdp_status dsdp_plan_launch_stage(dsdp_plan* P, uint32_t stages, void* stream) {
  if (!P) return set_error(DSDP_ERR_INVALID_ARG, "plan is NULL");
  if (stages == 0 || (stages & ~(uint32_t)DSDP_STAGE_ALL)) return set_error(DSDP_ERR_INVALID_ARG, "bad stages");
  const cudaStream_t st = (cudaStream_t)stream;
  const bool persistent = (P->flags & DSDP_PLAN_PERSISTENT) != 0;
  if ((stages & DSDP_STAGE_CHAINS) && persistent) {
    cudaError_t e = cudaMemsetAsync(P->d_counters, 0, sizeof(int) * 8, st);
    if (e != cudaSuccess) return check_cuda(e, "plan counter reset");
  }
  for (size_t gi = 0; (stages & DSDP_STAGE_CHAINS) && gi < P->groups.size(); ++gi) {
    const dsdp_plan::Group& g = P->groups[gi];
    ChainLaunch a;
    a.jobs = P->d_jobs;
    a.tiles = (const Tile*)P->d_tiles + g.first_tile;
    a.n_tiles = g.n_tiles;
    a.tile_counter = P->d_counters + gi;
    a.persistent = persistent ? 1 : 0;
    a.warps_per_cta = P->warps_per_cta;
    a.apl = g.apl;
    a.apl_mask = g.apl_mask;
    a.blob_smem = (g.blob_smem + 15) & ~15;
    a.scratch = scratch_layout(g.max_atoms, g.max_torsions, g.max_pairs, g.apl);
    a.variant = P->variant;
    a.grid = g.n_tiles;  // a persistent launch sizes its grid from the occupancy
    cudaError_t e = launch_chains_dispatch(g.fmt, a, st);
    if (e != cudaSuccess) return check_cuda(e, "dock_chains_kernel launch");
  }
  if ((stages & DSDP_STAGE_RESCORE) && !(P->flags & DSDP_PLAN_NO_RESCORE)) {
    cudaError_t e = launch_rescore(P->d_jobs, P->d_rtiles, P->n_rtiles, st);
    if (e != cudaSuccess) return check_cuda(e, "rescore_kernel launch");
    e = launch_topk(P->d_jobs, P->n_jobs, P->max_chains, st);
    if (e != cudaSuccess) return check_cuda(e, "topk_kernel launch");
  }
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_plan_launch(dsdp_plan* P, void* stream) {
  return dsdp_plan_launch_stage(P, DSDP_STAGE_ALL, stream);
}

extern "C" dsdp_status dsdp_plan_autotune(dsdp_plan* P, void* stream, int32_t repeats, int32_t* chosen,
                                          float* ms_by_config) {
  if (!P) return set_error(DSDP_ERR_INVALID_ARG, "plan is NULL");
  if (ms_by_config)
    for (int i = 0; i < 24; ++i) ms_by_config[i] = -1.f;
  if (repeats < 1) repeats = 1;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return check_cuda(e, "autotune events");
  const uint32_t base_flags = P->flags & ~(uint32_t)DSDP_PLAN_PERSISTENT;
  float best = 1e30f;
  int best_var = P->variant, best_pers = (P->flags & DSDP_PLAN_PERSISTENT) ? 1 : 0, best_w = P->warps_per_cta;
  dsdp_status s = DSDP_OK;
  // register budgets compiled: 128, 96, 80, 72 for one atom per lane, 128 and
  // 96 for two and for mixed tiles (launch_chains_impl)
  int n_var = 2;
  for (const dsdp_plan::Group& g : P->groups) n_var = std::max(n_var, g.apl_mask == 1 ? 4 : 2);
  for (int w = 1; w <= 4 && s == DSDP_OK; w *= 2) {
    e = plan_use_warps(P, w);
    if (e != cudaSuccess) {
      s = check_cuda(e, "autotune tiles");
      break;
    }
  for (int var = 0; var < n_var && s == DSDP_OK; ++var)
    for (int pers = 0; pers < 2 && s == DSDP_OK; ++pers) {
      P->variant = var;
      P->flags = base_flags | (pers ? DSDP_PLAN_PERSISTENT : 0u);
      s = dsdp_plan_launch_stage(P, DSDP_STAGE_CHAINS, stream);  // warm-up
      if (s != DSDP_OK) break;
      cudaEventRecord(a, st);
      for (int r = 0; r < repeats && s == DSDP_OK; ++r) s = dsdp_plan_launch_stage(P, DSDP_STAGE_CHAINS, stream);
      cudaEventRecord(b, st);
      e = cudaEventSynchronize(b);
      if (e != cudaSuccess) {
        s = check_cuda(e, "autotune run");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms_by_config) ms_by_config[var + 4 * (w == 4 ? 2 : w - 1) + 12 * pers] = ms / repeats;
      if (ms < best) {
        best = ms;
        best_var = var;
        best_pers = pers;
        best_w = w;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  P->variant = best_var;
  P->flags = base_flags | (best_pers ? DSDP_PLAN_PERSISTENT : 0u);
  if (s == DSDP_OK) s = check_cuda(plan_use_warps(P, best_w), "plan tiles");
  if (s != DSDP_OK) return s;
  tune_store(P->tune_key, best_var, best_pers, best_w);
  if (chosen) *chosen = 1 + best_var + 4 * (best_w == 4 ? 2 : best_w - 1) + 12 * best_pers;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_plan_destroy(dsdp_ctx* ctx, dsdp_plan* P) {
  if (!P) return DSDP_OK;
  if (P->arena) ctx_free(ctx ? ctx : P->ctx, P->arena, P->arena_bytes, nullptr);
  delete P;
  return DSDP_OK;
}
