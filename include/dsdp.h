/*
 * dsdp.h -- C ABI of the GB300 docking hot path of DSDP
 * ("DSDP: A Blind Docking Strategy Accelerated by GPUs", arXiv 2303.09916).
 *
 * The library docks flexible ligands into rigid receptors the way Sec. 2
 * ("Binding pose search by traditional sampling methods") describes: receptor
 * grid maps that hold the Vina score and its gradient at every vertex (first
 * modification; Appendix Eq. 1 and 4), trilinear interpolation of both
 * (Eq. 2 and 4), many short independent Monte Carlo copies (Sec. 2, "a large
 * number of copies (128-2048) and short search steps (20-200)") each locally
 * optimised by BFGS (Vina's optimiser) or Barzilai-Borwein (second
 * modification), and a postprocess that ranks the resulting poses (Fig. 4).
 *
 * Conventions used by every call
 * ------------------------------
 * - Status: every call returns a dsdp_status; 0 is success, 1 "pending",
 *   negative values are errors.  The library never aborts or exits.  After a
 *   failure dsdp_last_error() returns a message for the calling thread.
 * - Atom types are Vina XS types (DSDP_XS_*).  Ligand atoms use the eight map
 *   types 0..7; N_DA (8) may only appear on receptor atoms.
 * - Conformation ("conf") of a ligand with T torsions: 7 + T numbers
 *   [p (3): world position of the root origin atom,
 *    q (4): unit quaternion (w, x, y, z) rotating the reference geometry about
 *           that atom,
 *    theta (T): torsion angles, radians, relative to the input geometry].
 *   The root rigid body is the one with the most atoms (ties: the one holding
 *   the lowest atom index); its origin atom is its lowest-index atom.  The
 *   identity conformation (p = that atom's input position, q = 1, theta = 0)
 *   reproduces the input coordinates.  Torsion k is the k-th bond flagged
 *   rotatable in input order; positive theta rotates the far side of the bond
 *   (seen from the root) right-handedly about the axis from the near atom to
 *   the far atom.
 * - Gradient of an energy: 6 + T numbers [dE/dp (3), dE/domega (3) where omega
 *   is a world-frame rotation vector applied about p (q <- quat(omega) q),
 *   dE/dtheta (T)].
 * - Grid: n[a] = ceil(size[a] / spacing) vertices per axis, origin =
 *   center - (n - 1) * spacing / 2.  Map layout [type][z][y][x][channel],
 *   x fastest; EQ4 maps have 4 channels (score, dscore/dx, dy, dz; Eq. 4), EQ3
 *   maps 1 channel (score; the gradient is the derivative of the interpolant,
 *   Eq. 3).  An atom outside the grid is scored at its clamped position plus
 *   10 per Angstrom of excess along each axis.
 * - Host pointers passed to a call are borrowed for the duration of the call
 *   only; the library copies what it keeps.  Functions whose names end in
 *   _device take device pointers owned by the caller, enqueue work on the
 *   given CUDA stream (NULL = legacy default stream) and return without
 *   synchronising.
 * - Device: calls run on the device given to dsdp_create (handle API) or on
 *   the device current on the calling thread (_device calls).  Only sm_103a
 *   (GB300) code is built.
 */
#ifndef DSDP_H
#define DSDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int32_t dsdp_status;
#define DSDP_OK 0
#define DSDP_PENDING 1
#define DSDP_ERR_INVALID_ARG (-1)
#define DSDP_ERR_OUT_OF_MEMORY (-2) /* the request can never fit the budget, or an allocation failed */
#define DSDP_ERR_NOT_FOUND (-3)
#define DSDP_ERR_TIMEOUT (-4)
#define DSDP_ERR_CANCELLED (-5)
#define DSDP_ERR_DEVICE (-6) /* a CUDA call failed; the message names it */
#define DSDP_ERR_INTERNAL (-7)

/* Name of a status code (static string). */
const char* dsdp_status_string(dsdp_status s);
/* Message of the last failing call made by this thread (thread-local, static
 * until the next failing call on the same thread). */
const char* dsdp_last_error(void);
/* Library version, "major.minor.patch". */
const char* dsdp_version(void);

/* ------------------------------------------------------------------ types */
enum {
  DSDP_XS_C_H = 0, /* hydrophobic carbon */
  DSDP_XS_C_P = 1, /* polar carbon */
  DSDP_XS_N_P = 2,
  DSDP_XS_N_D = 3, /* donor */
  DSDP_XS_N_A = 4, /* acceptor */
  DSDP_XS_O_A = 5,
  DSDP_XS_O_DA = 6,
  DSDP_XS_S_P = 7,
  DSDP_XS_N_DA = 8 /* receptor only */
};
#define DSDP_NUM_MAP_TYPES 8
#define DSDP_MAX_LIGAND_ATOMS 64
#define DSDP_MAX_TORSIONS 15
#define DSDP_MAX_CHAINS 8192
#define DSDP_MAX_TOP_K 64
#define DSDP_MAX_SITE_POINTS 256

typedef enum { DSDP_MAP_F32 = 0, DSDP_MAP_BF16 = 1, DSDP_MAP_F16 = 2 } dsdp_map_dtype;
typedef enum { DSDP_GRID_EQ4 = 0, DSDP_GRID_EQ3 = 1 } dsdp_grid_mode;
typedef enum { DSDP_OPT_BFGS = 0, DSDP_OPT_BB = 1 } dsdp_optimizer;
/* DSDP_TERM_NORMALISED (dsdp_score_eval only): the selected terms and their
 * gradient divided by 1 + 0.0585 T (T torsions), the torsion normalisation of
 * the reported docking scores; on the device in FP32. */
enum { DSDP_TERM_INTER = 1, DSDP_TERM_INTRA = 2, DSDP_TERM_ALL = 3, DSDP_TERM_NORMALISED = 4 };

/* Receptor atoms (host or device memory, see each call). */
typedef struct {
  int32_t n;              /* number of heavy atoms, >= 1 */
  const float* xyz;       /* [n][3] Angstrom */
  const uint8_t* xs_type; /* [n] DSDP_XS_* */
} dsdp_receptor;

/* Grid box: the region the maps cover and the search region of the chains. */
typedef struct {
  double center[3];
  double size[3];  /* edge lengths, Angstrom, > spacing */
  double spacing;  /* vertex spacing, Angstrom */
} dsdp_box;

/* Ligand topology and reference pose (host memory). */
typedef struct {
  int32_t n_atoms;          /* 1 .. DSDP_MAX_LIGAND_ATOMS heavy atoms */
  const float* xyz;         /* [n_atoms][3] reference coordinates */
  const uint8_t* xs_type;   /* [n_atoms] map types 0..7 */
  int32_t n_bonds;
  const int32_t* bonds;     /* [n_bonds][2] atom indices */
  const uint8_t* rotatable; /* [n_bonds] 1 = rotatable; at most DSDP_MAX_TORSIONS;
                               each must split the molecule (no rotatable ring bond) */
} dsdp_ligand;

/* Docking job parameters.  Zero-initialise, then set what you need; zero
 * fields take the defaults in brackets. */
typedef struct {
  int32_t n_chains;     /* independent MC copies [384], <= DSDP_MAX_CHAINS */
  int32_t n_mc_steps;   /* MC steps per copy [40] */
  int32_t n_opt_iters;  /* local optimiser iterations per optimisation [100] */
  int32_t optimizer;    /* dsdp_optimizer [BFGS] */
  double temperature;   /* Metropolis temperature [1.2] */
  uint64_t seed;        /* Philox key; results depend on (seed, chain index) only */
  int32_t top_k;        /* poses returned after FP64 rescoring [9], <= DSDP_MAX_TOP_K */
  double rmsd_dedup;    /* poses closer than this heavy-atom RMSD to a better kept pose are dropped [1.0] */
  int32_t trace;        /* 1: keep per-step chain traces (tests; costs memory); 2: the same, but row 0
                           holds each chain's initial conformation, drawn before its first local
                           optimisation, instead of the state after it */
  /* Adaptive search space (Sec. 2, third modification; Fig. 3): with
   * n_site_points > 0 each chain's initial position is drawn uniformly from the
   * box intersected with the union of balls of radius site_radius around the
   * predicted binding-site points, instead of from the whole box.  The points
   * come from the caller (the paper's binding-site network is not part of this
   * library).  Rejection sampling: attempt a draws a uniform point of the box
   * from the chain's Philox stream (step 0, block 0 for a = 0, block 64 + a
   * after), accepted when it lies within site_radius of some point; the test
   * runs in FP32 with a fixed operation order (the same on every device); after
   * 64 rejected attempts the first site point is the start.  The MC steps are
   * not restrained beyond the box's wall. */
  float site_radius;    /* Angstrom [7.0] */
  int32_t n_site_points; /* 0 = the whole box, else 1 .. DSDP_MAX_SITE_POINTS */
  int32_t reserved0;
  const float* site_points; /* [n_site_points][3] Angstrom: host memory in dsdp_dock_submit (copied);
                               unused by the device-resident API (see dsdp_job_device) */
  int32_t reserved[2];
} dsdp_dock_params;

/* Result buffers of a finished job (caller-allocated host memory).  Set
 * capacity; any pointer may be NULL to skip that output. */
typedef struct {
  int32_t capacity;   /* in: poses the arrays can hold (>= top_k to get all) */
  int32_t n_out;      /* out: poses written */
  int32_t n_atoms;    /* out */
  int32_t n_torsions; /* out */
  double* score;      /* [capacity] FP64 gridless inter / (1 + 0.0585 T), ascending */
  double* inter;      /* [capacity] FP64 gridless receptor-ligand energy */
  double* intra;      /* [capacity] FP64 intra-ligand energy */
  double* conf;       /* [capacity][7 + T] */
  float* coords;      /* [capacity][n_atoms][3] input atom order */
  int32_t* chain;     /* [capacity] chain that produced the pose */
  float* chain_best_e;    /* [n_chains] best search energy per chain (grid score, FP32) */
  float* chain_best_conf; /* [n_chains][7 + T] */
  float* trace;           /* [n_chains][n_mc_steps + 1][7 + T + 4] when params.trace:
                             current conf after each step, then
                             (candidate E, current E, mode, accepted) */
  uint64_t n_evals;   /* out: score+gradient evaluations of the whole job */
  double device_ms;   /* out: device time of the job's batch, from launch to completion */
  double latency_ms;  /* out: host time from dsdp_dock_submit to the job's retirement (queueing included) */
} dsdp_dock_result;

/* ------------------------------------------------------------------ context */
typedef struct dsdp_ctx dsdp_ctx;
typedef struct dsdp_grid dsdp_grid;

/* Optional device allocator (e.g. a framework's caching allocator).  Must
 * return memory usable on `stream` or NULL on failure. */
typedef void* (*dsdp_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*dsdp_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

typedef struct {
  int32_t device;             /* CUDA device ordinal */
  uint64_t mem_budget_bytes;  /* device bytes jobs and grids may hold; 0 = 80 % of free memory */
  int32_t n_streams;          /* job streams, one batch in flight on each [4] */
  int32_t max_inflight_jobs;  /* jobs on the device at once, all batches [16] */
  dsdp_alloc_fn alloc;        /* NULL = cudaMallocAsync */
  dsdp_free_fn free;
  void* alloc_user;
  int32_t max_batch_chains;   /* chains of one batch at most; 0 = 64 x the SM count */
  void* stream;               /* cudaStream_t for the synchronous work (grid builds, scoring):
                                 ordered after the caller's earlier work on it; NULL = the
                                 context's own high-priority stream.  Not destroyed by
                                 dsdp_destroy. */
} dsdp_create_params;

/* Create a context: owns streams, the job table and a progress thread that
 * admits queued jobs as device memory and slots free up (continuous
 * batching): whenever a stream is free, every queued job that fits (in
 * order; at most max_batch_chains chains) is launched as one batch, a
 * multi-job plan whose chains share one work queue, while earlier batches
 * drain on the other streams.  Thread-safe: any thread may call any function
 * on a ctx. */
dsdp_status dsdp_create(const dsdp_create_params* params, dsdp_ctx** out);
/* Cancel queued jobs, wait for running ones, free everything. */
dsdp_status dsdp_destroy(dsdp_ctx* ctx);

/* ------------------------------------------------------------------ grids */
/* Build the 8 ligand-type maps of a receptor inside a box (Sec. 2 first
 * modification; Appendix Eq. 1 and 4): every vertex m and type t stores
 * E_t(m) = sum_j f(t, t_j, |m - r_j|) over receptor atoms within 8 A and its
 * gradient with respect to m.  Receptor arrays are host memory.  The grid
 * (and a device copy of the receptor, used for FP64 rescoring) stays resident
 * until dsdp_grid_free.  Returns once the receptor has been copied and the
 * build is queued on the device: jobs, scoring and downloads that use the grid
 * are ordered after the build there, so a host thread can submit the next
 * request while the GPU is busy.  An error of the build kernel itself is
 * reported by the first call that waits for it. */
dsdp_status dsdp_grid_build(dsdp_ctx* ctx, const dsdp_receptor* receptor, const dsdp_box* box,
                            dsdp_map_dtype dtype, dsdp_grid_mode mode, dsdp_grid** out);
/* Make a grid from maps computed elsewhere (host, FP32, layout above, C = 4
 * for EQ4, 1 for EQ3), stored in `dtype`.  `receptor` (host) may be NULL;
 * such a grid can score but not dock (docking rescoring needs atoms). */
dsdp_status dsdp_grid_from_maps(dsdp_ctx* ctx, const dsdp_receptor* receptor, const dsdp_box* box,
                                dsdp_map_dtype dtype, dsdp_grid_mode mode, const float* maps, dsdp_grid** out);
/* Copy a grid's maps to host memory as FP32 in the layout above. */
dsdp_status dsdp_grid_download(dsdp_ctx* ctx, const dsdp_grid* grid, float* maps, size_t capacity_floats);
/* Geometry of a grid: vertices per axis, origin, spacing, device bytes of the maps. */
dsdp_status dsdp_grid_info(const dsdp_grid* grid, int32_t n[3], double origin[3], double* spacing,
                           uint64_t* map_bytes);
dsdp_status dsdp_grid_free(dsdp_ctx* ctx, dsdp_grid* grid);

/* ------------------------------------------------------------------ scoring */
/* Score and gradient of n_conf conformations of one ligand on a grid: inter
 * (Eq. 2 and Eq. 4 or Eq. 3 on the maps, plus the out-of-grid wall) and/or
 * intra (pairs in different rigid bodies more than three bonds apart), chosen
 * by flags (DSDP_TERM_*).  Computed in FP32 on the device; host arrays:
 * conf [n_conf][7 + T], energy [n_conf], grad [n_conf][6 + T] (NULL to skip). */
dsdp_status dsdp_score_eval(dsdp_ctx* ctx, const dsdp_grid* grid, const dsdp_ligand* ligand, const double* conf,
                            int32_t n_conf, double* energy, double* grad, uint32_t flags);

/* ------------------------------------------------------------------ docking */
/* Queue a docking job (Sec. 2 / Fig. 4: independent MC copies on the device,
 * then FP64 gridless rescoring, RMSD de-duplication and top-k).  Returns at
 * once with a job id.  The job is admitted when the context's memory budget
 * and job slots allow; jobs on different grids and ligands overlap on the
 * device.  DSDP_ERR_OUT_OF_MEMORY only if the job alone exceeds the budget.
 * The grid must outlive the job. */
dsdp_status dsdp_dock_submit(dsdp_ctx* ctx, const dsdp_grid* grid, const dsdp_ligand* ligand,
                             const dsdp_dock_params* params, uint64_t* job_id);
/* Submit n jobs at once (virtual screening: many ligands, one or a few
 * grids): grids[i], ligands[i] and params[i] as for dsdp_dock_submit; job_ids
 * receives n ids.  The ligands are packed on up to 8 host threads, then all n
 * jobs are queued together, so the progress thread can take them in one batch
 * (as many as max_batch_chains admits).  All or none: on any error no job is
 * queued and the message names the first failing index.  Arrays are borrowed
 * for the call. */
dsdp_status dsdp_dock_submit_many(dsdp_ctx* ctx, int32_t n, const dsdp_grid* const* grids,
                                  const dsdp_ligand* ligands, const dsdp_dock_params* params, uint64_t* job_ids);
/* Wait up to wait_ms (0: do not block, < 0: forever) for a job.  With
 * wait_ms = 0 an unfinished job returns DSDP_PENDING; a positive wait that
 * expires returns DSDP_ERR_TIMEOUT (the job keeps its place: poll again).  On
 * DSDP_OK the results are copied into `out` and the job is released (a second
 * poll returns DSDP_ERR_NOT_FOUND).  A job that failed or was cancelled returns
 * its error (DSDP_ERR_CANCELLED) once and is released. */
dsdp_status dsdp_dock_poll(dsdp_ctx* ctx, uint64_t job_id, dsdp_dock_result* out, int32_t wait_ms);
/* Cancel a job (DSDP_OK).  A queued job is dropped at once; a running job's
 * kernels run to the end of its batch (a batch is one launch shared with other
 * jobs), then its results are dropped and its memory freed.  Either way the
 * next poll that finds it finished returns DSDP_ERR_CANCELLED and releases it.
 * A job that already finished is not affected. */
dsdp_status dsdp_dock_cancel(dsdp_ctx* ctx, uint64_t job_id);

typedef struct {
  uint64_t submitted, completed, failed, cancelled;
  int32_t queued, running;
  uint64_t bytes_in_use, bytes_budget;
  uint64_t batches; /* batches launched (multi-job plans), since dsdp_create */
} dsdp_stats;
dsdp_status dsdp_get_stats(dsdp_ctx* ctx, dsdp_stats* out);

/* ------------------------------------------------------------------ device-resident path
 * For callers that own device memory (e.g. PyTorch tensors) and want the
 * inputs to stay resident: no host copies, no allocation inside the calls
 * except dsdp_plan_create. */

/* Bytes of the maps of a box (all 8 types). */
uint64_t dsdp_grid_map_bytes(const dsdp_box* box, dsdp_map_dtype dtype, dsdp_grid_mode mode);
/* Build maps from device receptor arrays into caller memory d_maps
 * (>= dsdp_grid_map_bytes).  Enqueued on `stream`. */
dsdp_status dsdp_grid_build_device(const dsdp_receptor* d_receptor, const dsdp_box* box, dsdp_map_dtype dtype,
                                   dsdp_grid_mode mode, void* d_maps, uint64_t maps_bytes, void* stream);

/* Pack a ligand's torsion tree, atom order, intra pair list and per-atom pair
 * index into a self-contained blob (host memory, position independent; copy
 * it to the device as is).  With blob == NULL only *blob_bytes is set. */
dsdp_status dsdp_ligand_pack(const dsdp_ligand* ligand, void* blob, uint64_t capacity, uint64_t* blob_bytes);
/* Read a packed blob's sizes. */
dsdp_status dsdp_ligand_blob_info(const void* blob, int32_t* n_atoms, int32_t* n_torsions, int32_t* n_pairs,
                                  int32_t* n_bodies);

/* A grid seen by the device path. */
typedef struct {
  const void* d_maps;
  int32_t n[3];
  double origin[3];
  double spacing;
  int32_t dtype; /* dsdp_map_dtype */
  int32_t mode;  /* dsdp_grid_mode */
} dsdp_grid_view;

/* Score n_conf FP32 conformations (device [n_conf][7 + T]) into d_energy
 * [n_conf] and d_grad [n_conf][6 + T] (may be NULL).  h_blob and d_blob are the
 * host and device copies of the same packed ligand. */
dsdp_status dsdp_score_eval_device(const dsdp_grid_view* grid, const void* h_blob, const void* d_blob,
                                   const float* d_conf, int32_t n_conf, float* d_energy, float* d_grad,
                                   uint32_t flags, void* stream);

/* One job of a device-side docking batch.  Inputs and outputs are device
 * memory owned by the caller. */
typedef struct {
  dsdp_grid_view grid;
  dsdp_receptor receptor;   /* device arrays of the grid's receptor (rescoring) */
  const void* h_blob;       /* packed ligand, host copy (sizes) */
  const void* d_blob;       /* packed ligand, device copy */
  dsdp_dock_params params;
  double box_lo[3];         /* search region of the initial positions */
  double box_size[3];
  /* outputs */
  float* d_chain_best_conf; /* [n_chains][7 + T] */
  float* d_chain_best_e;    /* [n_chains] */
  uint32_t* d_chain_evals;  /* [n_chains] */
  float* d_trace;           /* NULL or [n_chains][n_mc_steps + 1][7 + T + 4] */
  int32_t* d_out_n;         /* [1] poses kept */
  int32_t* d_out_chain;     /* [top_k] */
  double* d_out_score;      /* [top_k] */
  double* d_out_inter;      /* [top_k] */
  double* d_out_intra;      /* [top_k] */
  double* d_out_conf;       /* [top_k][7 + T] */
  float* d_out_coords;      /* [top_k][n_atoms][3] input atom order */
  const float* d_site_points; /* device [params.n_site_points][3] when params.n_site_points > 0 */
} dsdp_job_device;

typedef struct dsdp_plan dsdp_plan;
enum {
  DSDP_PLAN_PERSISTENT = 1, /* one CTA set sized to the GPU pulls chain tiles from a queue */
  DSDP_PLAN_NO_RESCORE = 2  /* stop after the chains (no FP64 rescoring / top-k) */
};
/* Prepare a launch of n_jobs jobs (uneven ligands allowed): uploads job and
 * tile tables, sizes scratch (allocated with the ctx allocator; ctx may be NULL
 * for plain cudaMalloc).  One warp runs one chain; a CTA runs a tile of W
 * chains of one job (W = 1, 2 or 4) and stages that job's ligand once.
 * tile_config: 0 = automatic (the choice dsdp_plan_autotune recorded for a plan
 * of the same shape -- map formats, atoms per lane, chain count rounded up to
 * a power of two -- else the 96-register kernel for plans of at least
 * 32 x (SM count) chains and the 128-register kernel for smaller ones, with
 * W = 1, or W = 4 when a ligand has more than 32 atoms); 1 .. 12 = a fixed
 * choice 1 + variant +
 * 4 log2(W): register budget (variant 0: 128 registers, 16 warps per SM; 1: 96,
 * 20 warps; 2: 80, 24 warps; 3: 72, 28 warps) and W = 1, 2 or 4.  Budgets 80
 * and 72 are compiled for ligands of up to 32 atoms only (one atom per lane);
 * ligands above 32 atoms run at 128 or 96 (variants 2 and 3 take 96), and so
 * does a map-format group that mixes ligands of up to 32 and of more than 32
 * atoms (one kernel holding both tile sizes).  Results do not depend on the
 * configuration. */
dsdp_status dsdp_plan_create(dsdp_ctx* ctx, int32_t n_jobs, const dsdp_job_device* jobs, uint32_t flags,
                             int32_t tile_config, dsdp_plan** out);
/* Autotuner: runs the plan's chain stage `repeats` times for each register
 * budget the plan's kernels are compiled for (128 and 96; also 80 and 72 when
 * a group holds only ligands of at most 32 atoms), each tile of W = 1, 2, 4
 * chains per CTA, with and without the
 * persistent work queue, keeps the fastest for this plan and records it for
 * later plans of the same shape (process-wide).  *chosen = 1 + variant
 * + 4 * log2(W) + 12 * persistent (1 .. 24; the first part is the plan's
 * tile_config).  ms_by_config: NULL, or 24 floats receiving the measured chain
 * stage time (ms per launch) of configuration chosen - 1, -1 where a
 * configuration was not run.  Synchronises the stream. */
dsdp_status dsdp_plan_autotune(dsdp_plan* plan, void* stream, int32_t repeats, int32_t* chosen, float* ms_by_config);
/* Enqueue the plan's kernels on `stream` (chains, then FP64 rescoring and
 * top-k).  No allocation and no host synchronisation: a launch can be
 * captured into a CUDA graph and replayed.  Different plans may run at once
 * on different streams when no two of them write the same output buffers (or
 * have their maps rebuilt while the other reads them); a plan's own launches
 * must be ordered (they share its scratch and work-queue counters). */
dsdp_status dsdp_plan_launch(dsdp_plan* plan, void* stream);
/* Stages of a plan for dsdp_plan_launch_stage. */
enum { DSDP_STAGE_CHAINS = 1, DSDP_STAGE_RESCORE = 2, DSDP_STAGE_ALL = 3 };
/* Enqueue only some stages (e.g. to time the chain kernels alone); stages
 * must run in order: chains before rescoring. */
dsdp_status dsdp_plan_launch_stage(dsdp_plan* plan, uint32_t stages, void* stream);
/* Kernel launches one dsdp_plan_launch performs. */
int32_t dsdp_plan_kernel_count(const dsdp_plan* plan);
dsdp_status dsdp_plan_destroy(dsdp_ctx* ctx, dsdp_plan* plan);

/* Gather microbenchmark behind the roofline: n_points threads each sample
 * `repeats` positions in the grid -- the first from d_points / d_types, the
 * others independent pseudo-random positions and map types -- reading the 8
 * cell corners of one map at each (the bytes of the score path's inter term,
 * Eq. 2-4, with no arithmetic beyond the sum that keeps the loads live).
 * Writes one float per point into d_out.  d_points [n_points][3] device. */
dsdp_status dsdp_gather_bench_device(const dsdp_grid_view* grid, const float* d_points, const uint8_t* d_types,
                                     int32_t n_points, int32_t repeats, float* d_out, void* stream);

/* ------------------------------------------------------------------ receptor voxel features
 * The binding-site network's input (Sec. 2, "Protein-ligand binding site
 * prediction"): the protein as 36 x 36 x 36 voxels with 18 channels over a 70 A
 * cube centred on it; S and Se share one element channel and the freed channel
 * marks the protein surface.  The network itself is not part of this library.
 *   - Voxel k of an axis covers [c - 35 + k 70/36, c - 35 + (k + 1) 70/36): an
 *     atom's voxel is floor((x - (c - 35)) * (36/70)), computed in FP32
 *     (c - 35 rounded to FP32 first); atoms outside the cube are dropped.
 *   - Channels 0..16: sums of the caller's 17 per-atom features over the
 *     voxel's atoms.  Channel 17: the voxel's number of surface atoms, atom i
 *     being on the surface when a test point x_i + (r_i + 1.4) u of its
 *     solvent-accessible sphere (98 directions u: the primitive integer
 *     vectors of {-2..2}^3, normalised) lies outside the sphere of radius
 *     r_j + 1.4 of every other atom (Shrake and Rupley).
 *   - Sums are exact and independent of the atom order: each feature is
 *     rounded to a multiple of 2^-24 and accumulated as a 64-bit integer; a
 *     channel is the sum times 2^-24 rounded to FP32.
 * Arguments: d_xyz [n_atoms][3], d_radius [n_atoms] (van der Waals radii, A),
 * d_features [n_atoms][17], all FP32 device arrays; center (host, A); d_out
 * [36][36][36][18] FP32 (z, y, x, channel) device; d_work: device scratch of
 * at least dsdp_voxel_work_bytes() bytes, 8-byte aligned, owned by the caller.
 * Enqueued on `stream`; DSDP_ERR_INVALID_ARG for a negative count, NULL
 * arrays, a short or misaligned work buffer or a non-finite centre. */
#define DSDP_VOXEL_N 36
#define DSDP_VOXEL_FEATURES 17
#define DSDP_VOXEL_CHANNELS 18
uint64_t dsdp_voxel_work_bytes(void);
dsdp_status dsdp_voxelize_device(int32_t n_atoms, const float* d_xyz, const float* d_radius,
                                 const float* d_features, const double center[3], float* d_out, void* d_work,
                                 uint64_t work_bytes, void* stream);

/* ------------------------------------------------------------------ no-allocation postprocess
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory when they need the postprocess: code holding an
 * allocator's lock, a framework's memory-planning phase, a real-time thread
 * that must stay off the driver's allocation path, or a host that owns a fixed
 * device budget.
 *
 * dsdp_rescore_topk_noalloc runs the FP64 rescoring, RMSD de-duplication and
 * top-k of one job (the work dsdp_plan_launch does after the chains) and
 * allocates nothing: no cudaMalloc / cudaFree, no allocator callback, no
 * library routine that allocates.  Its scratch is one file-scope device array
 * of DSDP_NOALLOC_SCRATCH_BYTES (about 1.6 MB) that every GPU loading the
 * library holds until the process exits.
 *   - job: as for dsdp_plan_create; inputs read: h_blob, d_blob, receptor,
 *     params (n_chains <= DSDP_NOALLOC_MAX_CHAINS, top_k, rmsd_dedup) and
 *     d_chain_best_conf (the chains' best poses, FP32); outputs written: d_out_n,
 *     d_out_chain, d_out_score, d_out_inter, d_out_intra, d_out_conf,
 *     d_out_coords (NULL skips one).  Grid, box and trace fields are ignored.
 *   - Errors: DSDP_ERR_INVALID_ARG for n_chains above the limit or missing
 *     arrays, DSDP_ERR_DEVICE when a launch fails.
 *   - The first call on a device is a set-up call: it resolves the array's
 *     device address (with that device current) and, under CUDA's lazy module
 *     loading (the default), may load this library's rescoring kernels and
 *     commit the array -- device memory the driver allocates.  Make that first
 *     call outside any phase that must not allocate (a warm-up at start-up) and
 *     before capturing a stream; later calls on that device allocate nothing.
 *   - The resolved address is kept for the life of the process: do not use the
 *     library across a cudaDeviceReset or after the primary context is
 *     destroyed and re-created.
 *   - Every call shares the array and it keeps the last call's contents; no
 *     field has to start at zero, since each value read is written earlier in
 *     the same call.  Calls that overlap on the GPU (other streams, or other
 *     host threads, on the same device) race on the array: serialise them. */
#define DSDP_NOALLOC_MAX_CHAINS 1024
#define DSDP_NOALLOC_SCRATCH_BYTES 1600000
dsdp_status dsdp_rescore_topk_noalloc(const dsdp_job_device* job, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DSDP_H */
