// Host side of the C ABI: contexts, grid handles, scoring and the docking job
// queue.  The queue realises the paper's asynchronous pipeline (Sec. 2 /
// Fig. 4: copies prepared on the host, uploaded, run independently on the
// GPU, results postprocessed) as a continuously batched service: a progress
// thread takes every queued job that device memory and the job slots admit
// into one batch -- one multi-job plan, whose chains share one work queue --
// launches it on the next free stream while earlier batches drain, and
// retires each batch through a CUDA event.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dsdp_internal.h"

using namespace dsdp;

struct dsdp_grid {
  dsdp_ctx* ctx = nullptr;
  dsdp_box box{};
  int n[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0};
  int dtype = 0, mode = 0;
  void* d_maps = nullptr;
  uint64_t map_bytes = 0;
  int n_rec = 0;
  float* d_rec_xyz = nullptr;
  uint8_t* d_rec_type = nullptr;
  uint64_t rec_bytes = 0;
  std::atomic<int> users{0};  // jobs referencing the grid
  cudaEvent_t ready = nullptr;  // recorded after the maps are written; jobs wait on it on the device
};

namespace {

enum class JobState { Queued, Running, Done, Failed, Cancelled };

struct Job {
  uint64_t id = 0;
  JobState state = JobState::Queued;
  dsdp_status err = DSDP_OK;
  std::string msg;
  const dsdp_grid* grid = nullptr;
  std::vector<uint8_t> blob;  // packed ligand, then (16-byte aligned) the site points, uploaded together
  size_t sites_off = 0;       // offset of the site points in blob (n_site_points > 0)
  dsdp_dock_params params{};
  int n_atoms = 0, T = 0;
  // device memory: [blob | results]; results copied back with one D2H
  void* d_mem = nullptr;
  uint64_t d_bytes = 0;
  uint64_t plan_bytes = 0;
  size_t res_off = 0, res_bytes = 0;
  // offsets inside the results region
  size_t o_n, o_chain, o_score, o_inter, o_intra, o_conf, o_coords, o_cbe, o_cbc, o_evals, o_trace;
  void* h_res = nullptr;  // pinned, from the context's pool
  size_t h_cap = 0;
  int stream = 0;
  dsdp_job_device jd{};  // the job as the plan sees it
  bool cancel_requested = false;  // cancelled while running: its results are dropped when its batch retires
  float device_ms = 0.f;  // device time of the batch the job ran in
  std::chrono::steady_clock::time_point t_submit, t_done;
};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Jobs launched together: one plan, one stream, one completion event.
struct Batch {
  std::vector<Job*> jobs;
  dsdp_plan* plan = nullptr;
  int stream = 0;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

}  // namespace

struct dsdp_ctx {
  int device = 0;
  int sms = 148;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  int max_inflight = 16;
  int max_batch_chains = 0;            // chains per batch (default 64 per SM)
  std::vector<cudaStream_t> streams;   // one batch in flight per stream
  cudaStream_t sync_stream = nullptr;   // synchronous calls and grid builds
  bool own_sync_stream = true;          // false: the caller's stream (dsdp_create_params.stream)
  cudaStream_t upload_stream = nullptr; // receptor uploads of grid builds (copy engines only)
  cudaStream_t alloc_stream = nullptr;  // allocations done outside a job stream
  cudaMemPool_t pool = nullptr;         // the context's own stream-ordered pool (no caller allocator)
  int next_stream = 0;
  dsdp_alloc_fn alloc = nullptr;
  dsdp_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<uint64_t, Job*> jobs;
  std::deque<uint64_t> queue;
  std::vector<Batch*> batches;                 // in flight
  std::multimap<size_t, void*> pinned_pool;    // capacity -> pinned host buffer
  size_t pinned_pooled = 0;
  uint64_t next_id = 1;
  int running = 0;
  bool stop = false;
  std::thread progress;
  dsdp_stats stats{};
};

namespace dsdp {

int ctx_sm_count(dsdp_ctx* ctx) {
  if (ctx) return ctx->sms;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

void* ctx_alloc(dsdp_ctx* ctx, size_t bytes, void* stream) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (!ctx) return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, stream ? stream : (void*)ctx->alloc_stream, ctx->alloc_user);
    if (p && !stream) cudaStreamSynchronize(ctx->alloc_stream);
    return p;
  }
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->alloc_stream;
  const cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(&p, bytes, ctx->pool, st) : cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (!stream) cudaStreamSynchronize(ctx->alloc_stream);
  return p;
}

void ctx_free(dsdp_ctx* ctx, void* p, size_t bytes, void* stream) {
  if (!p) return;
  if (!ctx) {
    cudaFree(p);
    return;
  }
  if (ctx->free_fn) {
    ctx->free_fn(p, bytes, stream ? stream : (void*)ctx->alloc_stream, ctx->alloc_user);
    return;
  }
  cudaFreeAsync(p, stream ? (cudaStream_t)stream : ctx->alloc_stream);
}

}  // namespace dsdp

// ------------------------------------------------------------------ status
extern "C" const char* dsdp_status_string(dsdp_status s) {
  switch (s) {
    case DSDP_OK: return "DSDP_OK";
    case DSDP_PENDING: return "DSDP_PENDING";
    case DSDP_ERR_INVALID_ARG: return "DSDP_ERR_INVALID_ARG";
    case DSDP_ERR_OUT_OF_MEMORY: return "DSDP_ERR_OUT_OF_MEMORY";
    case DSDP_ERR_NOT_FOUND: return "DSDP_ERR_NOT_FOUND";
    case DSDP_ERR_TIMEOUT: return "DSDP_ERR_TIMEOUT";
    case DSDP_ERR_CANCELLED: return "DSDP_ERR_CANCELLED";
    case DSDP_ERR_DEVICE: return "DSDP_ERR_DEVICE";
    case DSDP_ERR_INTERNAL: return "DSDP_ERR_INTERNAL";
    default: return "DSDP_UNKNOWN_STATUS";
  }
}
extern "C" const char* dsdp_last_error(void) { return dsdp::last_error(); }
extern "C" const char* dsdp_version(void) { return "0.1.0"; }

// ------------------------------------------------------------------ jobs
namespace {

// Pinned host buffers are pooled by power-of-two capacity: pinning pages is
// slow and would otherwise sit on every job's path (ctx->mu held).
constexpr size_t kPinnedPoolLimit = 256u << 20;
void pinned_get(dsdp_ctx* ctx, Job* j, size_t bytes) {
  size_t cap = 4096;
  while (cap < bytes) cap <<= 1;
  auto it = ctx->pinned_pool.find(cap);
  if (it != ctx->pinned_pool.end()) {
    j->h_res = it->second;
    ctx->pinned_pooled -= cap;
    ctx->pinned_pool.erase(it);
  } else if (cudaMallocHost(&j->h_res, cap) != cudaSuccess) {
    cudaGetLastError();
    j->h_res = nullptr;
    return;
  }
  j->h_cap = cap;
}
void pinned_put(dsdp_ctx* ctx, Job* j) {
  if (!j->h_res) return;
  if (ctx->pinned_pooled + j->h_cap <= kPinnedPoolLimit) {
    ctx->pinned_pool.emplace(j->h_cap, j->h_res);
    ctx->pinned_pooled += j->h_cap;
  } else {
    cudaFreeHost(j->h_res);
  }
  j->h_res = nullptr;
}

// Frees a job's device memory (the caller adjusts ctx->in_use).
void job_release_device(dsdp_ctx* ctx, Job* j) {
  if (j->d_mem) {
    ctx_free(ctx, j->d_mem, j->d_bytes, (void*)ctx->streams[j->stream]);
    j->d_mem = nullptr;
  }
}

// Results region layout.
void layout_results(Job* j) {
  const dsdp_dock_params& p = j->params;
  const int nx = 7 + j->T, k = p.top_k, C = p.n_chains;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += up256(bytes);
    return at;
  };
  j->o_n = take(sizeof(int32_t));
  j->o_chain = take(sizeof(int32_t) * k);
  j->o_score = take(sizeof(double) * k);
  j->o_inter = take(sizeof(double) * k);
  j->o_intra = take(sizeof(double) * k);
  j->o_conf = take(sizeof(double) * k * nx);
  j->o_coords = take(sizeof(float) * k * j->n_atoms * 3);
  j->o_cbe = take(sizeof(float) * C);
  j->o_cbc = take(sizeof(float) * (size_t)C * nx);
  j->o_evals = take(sizeof(uint32_t) * C);
  j->o_trace = take(p.trace ? sizeof(float) * (size_t)C * (p.n_mc_steps + 1) * (nx + 4) : 0);
  j->res_bytes = o;
}

// Estimated plan scratch of a job (rescoring arrays and tables).
uint64_t plan_scratch_estimate(const Job* j) {
  const uint64_t C = (uint64_t)j->params.n_chains;
  return 4096 + 3 * 8 * C + 8 * C * j->n_atoms * 3 + 64 * C + 16 * C;
}

// Device memory, pinned buffer and blob upload of one job on stream st, and
// its dsdp_job_device (ctx->mu held).  Returns false (err / msg set, nothing
// held) if a resource could not be had.
bool job_prepare(dsdp_ctx* ctx, Job* j, int stream) {
  const dsdp_grid* g = j->grid;
  j->stream = stream;
  const cudaStream_t st = ctx->streams[stream];
  layout_results(j);
  j->res_off = up256(j->blob.size());
  j->d_bytes = j->res_off + j->res_bytes;
  auto fail = [&](dsdp_status s, const char* what) {
    j->err = s;
    j->msg = what;
    return false;
  };
  j->d_mem = ctx_alloc(ctx, j->d_bytes, (void*)st);
  if (!j->d_mem) return fail(DSDP_ERR_OUT_OF_MEMORY, "job device allocation failed");
  pinned_get(ctx, j, std::max(j->res_bytes, j->blob.size()));
  if (!j->h_res) {
    ctx_free(ctx, j->d_mem, j->d_bytes, (void*)st);
    j->d_mem = nullptr;
    return fail(DSDP_ERR_OUT_OF_MEMORY, "pinned result buffer allocation failed");
  }
  // the blob goes up through the pinned result buffer; the results come back
  // into it later on the same stream, after the upload has completed
  uint8_t* dm = (uint8_t*)j->d_mem;
  uint8_t* res = dm + j->res_off;
  memcpy(j->h_res, j->blob.data(), j->blob.size());
  cudaError_t e = cudaMemcpyAsync(dm, j->h_res, j->blob.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    job_release_device(ctx, j);
    return fail(check_cuda(e, "blob upload"), dsdp_last_error());
  }
  dsdp_job_device& jd = j->jd;
  memset(&jd, 0, sizeof(jd));
  jd.grid.d_maps = g->d_maps;
  for (int a = 0; a < 3; ++a) {
    jd.grid.n[a] = g->n[a];
    jd.grid.origin[a] = g->origin[a];
    jd.box_lo[a] = g->box.center[a] - g->box.size[a] / 2.0;
    jd.box_size[a] = g->box.size[a];
  }
  jd.grid.spacing = g->box.spacing;
  jd.grid.dtype = g->dtype;
  jd.grid.mode = g->mode;
  jd.receptor.n = g->n_rec;
  jd.receptor.xyz = g->d_rec_xyz;
  jd.receptor.xs_type = g->d_rec_type;
  jd.h_blob = j->blob.data();
  jd.d_blob = dm;
  jd.params = j->params;
  if (j->params.n_site_points > 0) jd.d_site_points = (const float*)(dm + j->sites_off);
  jd.d_chain_best_conf = (float*)(res + j->o_cbc);
  jd.d_chain_best_e = (float*)(res + j->o_cbe);
  jd.d_chain_evals = (uint32_t*)(res + j->o_evals);
  jd.d_trace = j->params.trace ? (float*)(res + j->o_trace) : nullptr;
  jd.d_out_n = (int32_t*)(res + j->o_n);
  jd.d_out_chain = (int32_t*)(res + j->o_chain);
  jd.d_out_score = (double*)(res + j->o_score);
  jd.d_out_inter = (double*)(res + j->o_inter);
  jd.d_out_intra = (double*)(res + j->o_intra);
  jd.d_out_conf = (double*)(res + j->o_conf);
  jd.d_out_coords = (float*)(res + j->o_coords);
  return true;
}

void job_fail(dsdp_ctx* ctx, Job* j, dsdp_status s, std::string msg) {
  j->state = JobState::Failed;
  j->err = s;
  j->msg = std::move(msg);
  j->t_done = std::chrono::steady_clock::now();
  ctx->stats.failed++;
}

// Plan, launch and result downloads of prepared jobs as one batch on stream
// `stream` (ctx->mu held).  Returns the batch, or nullptr when its plan or
// launch failed (the jobs stay prepared; the caller decides what to do).
Batch* batch_launch(dsdp_ctx* ctx, const std::vector<Job*>& jobs, int stream) {
  const cudaStream_t st = ctx->streams[stream];
  std::vector<dsdp_job_device> jd(jobs.size());
  for (size_t i = 0; i < jobs.size(); ++i) jd[i] = jobs[i]->jd;
  Batch* b = new Batch();
  b->jobs = jobs;
  b->stream = stream;
  dsdp_status s = dsdp_plan_create(ctx, (int32_t)jd.size(), jd.data(), 0, 0, &b->plan);
  for (size_t i = 0; s == DSDP_OK && i < jobs.size(); ++i)  // the maps may still be in the making
    if (jobs[i]->grid->ready) s = check_cuda(cudaStreamWaitEvent(st, jobs[i]->grid->ready, 0), "grid wait");
  if (s == DSDP_OK) {
    cudaEventCreateWithFlags(&b->ev_start, cudaEventDefault);
    cudaEventCreateWithFlags(&b->ev_done, cudaEventDefault);
    cudaEventRecord(b->ev_start, st);
    s = dsdp_plan_launch(b->plan, (void*)st);
  }
  if (s == DSDP_OK) {
    for (Job* j : jobs) {
      const cudaError_t e = cudaMemcpyAsync(j->h_res, (uint8_t*)j->d_mem + j->res_off, j->res_bytes,
                                            cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) {
        s = check_cuda(e, "result download");
        break;
      }
    }
    if (s == DSDP_OK) s = check_cuda(cudaEventRecord(b->ev_done, st), "batch event");
  }
  if (s != DSDP_OK) {
    cudaStreamSynchronize(st);
    if (b->plan) dsdp_plan_destroy(ctx, b->plan);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_done) cudaEventDestroy(b->ev_done);
    delete b;
    return nullptr;
  }
  for (Job* j : jobs) j->state = JobState::Running;
  return b;
}

// Retire a finished batch: results are in the jobs' pinned buffers.
void batch_retire(dsdp_ctx* ctx, Batch* b, cudaError_t q) {
  float ms = 0.f;
  if (q == cudaSuccess) cudaEventElapsedTime(&ms, b->ev_start, b->ev_done);
  const auto now = std::chrono::steady_clock::now();
  for (Job* j : b->jobs) {
    if (q != cudaSuccess) {
      job_fail(ctx, j, check_cuda(q, "job execution"), dsdp_last_error());
    } else if (j->cancel_requested) {
      j->state = JobState::Cancelled;
      j->t_done = now;
      ctx->stats.cancelled++;
    } else {
      j->state = JobState::Done;
      j->device_ms = ms;
      j->t_done = now;
      ctx->stats.completed++;
    }
    job_release_device(ctx, j);
    ctx->in_use -= j->d_bytes + j->plan_bytes;
    const_cast<dsdp_grid*>(j->grid)->users--;
    ctx->running--;
  }
  dsdp_plan_destroy(ctx, b->plan);
  cudaEventDestroy(b->ev_start);
  cudaEventDestroy(b->ev_done);
  delete b;
}

void progress_loop(dsdp_ctx* ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  std::vector<char> busy;
  while (!ctx->stop) {
    bool changed = false;
    // retire finished batches
    for (size_t i = 0; i < ctx->batches.size();) {
      Batch* b = ctx->batches[i];
      const cudaError_t q = cudaEventQuery(b->ev_done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      batch_retire(ctx, b, q);
      ctx->batches.erase(ctx->batches.begin() + i);
      changed = true;
    }
    // one new batch per free stream: the queued jobs, in order, that memory,
    // the job slots and the batch size admit
    busy.assign(ctx->streams.size(), 0);
    for (Batch* b : ctx->batches) busy[b->stream] = 1;
    while (!ctx->queue.empty() && ctx->running < ctx->max_inflight) {
      int stream = -1;
      for (size_t k = 0; k < busy.size(); ++k) {
        const int c = (ctx->next_stream + (int)k) % (int)busy.size();
        if (!busy[c]) {
          stream = c;
          break;
        }
      }
      if (stream < 0) break;
      std::vector<Job*> take;
      int64_t chains = 0;
      while (!ctx->queue.empty() && ctx->running + (int)take.size() < ctx->max_inflight) {
        Job* j = ctx->jobs[ctx->queue.front()];
        const uint64_t need = up256(j->blob.size()) + j->res_bytes + plan_scratch_estimate(j);
        const bool alone = ctx->running == 0 && take.empty();
        if (ctx->in_use + need > ctx->budget && !alone) break;  // wait for memory
        if (!take.empty() && chains + j->params.n_chains > ctx->max_batch_chains) break;
        ctx->queue.pop_front();
        if (!job_prepare(ctx, j, stream)) {
          job_fail(ctx, j, j->err, j->msg);
          const_cast<dsdp_grid*>(j->grid)->users--;
          changed = true;
          continue;
        }
        j->plan_bytes = plan_scratch_estimate(j);
        ctx->in_use += j->d_bytes + j->plan_bytes;
        chains += j->params.n_chains;
        take.push_back(j);
      }
      if (take.empty()) break;
      ctx->running += (int)take.size();
      Batch* b = batch_launch(ctx, take, stream);
      if (b) {
        ctx->batches.push_back(b);
        ctx->stats.batches++;
      } else {
        // a batch-wide failure: isolate it by running the jobs one by one
        const std::string why = dsdp_last_error();
        for (Job* j : take) {
          Batch* one = batch_launch(ctx, {j}, stream);
          if (one) {
            ctx->batches.push_back(one);
            ctx->stats.batches++;
            continue;
          }
          job_fail(ctx, j, DSDP_ERR_DEVICE, why + "; alone: " + dsdp_last_error());
          job_release_device(ctx, j);
          ctx->in_use -= j->d_bytes + j->plan_bytes;
          const_cast<dsdp_grid*>(j->grid)->users--;
          ctx->running--;
        }
      }
      busy[stream] = 1;
      ctx->next_stream = (stream + 1) % (int)ctx->streams.size();
      changed = true;
    }
    if (changed) ctx->cv_done.notify_all();
    if (!ctx->batches.empty()) ctx->cv_work.wait_for(lk, std::chrono::microseconds(100));
    else ctx->cv_work.wait(lk, [&] { return ctx->stop || !ctx->queue.empty(); });
  }
}

}  // namespace

// ------------------------------------------------------------------ context
extern "C" dsdp_status dsdp_create(const dsdp_create_params* params, dsdp_ctx** out) {
  if (!out) return set_error(DSDP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  dsdp_create_params p{};
  if (params) p = *params;
  int n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDeviceCount");
  if (p.device < 0 || p.device >= n_dev) return set_error(DSDP_ERR_INVALID_ARG, "device %d of %d", p.device, n_dev);
  if ((p.alloc == nullptr) != (p.free == nullptr))
    return set_error(DSDP_ERR_INVALID_ARG, "alloc and free callbacks go together");
  if (p.max_batch_chains < 0) return set_error(DSDP_ERR_INVALID_ARG, "max_batch_chains < 0");
  e = cudaSetDevice(p.device);
  if (e != cudaSuccess) return check_cuda(e, "cudaSetDevice");
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p.device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p.device);
  if (major * 10 + minor != 103)
    return set_error(DSDP_ERR_DEVICE, "libdsdp is built for sm_103a (GB300); device %d is sm_%d%d", p.device, major,
                     minor);
  dsdp_ctx* ctx = new dsdp_ctx();
  ctx->device = p.device;
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, p.device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  ctx->budget = p.mem_budget_bytes ? p.mem_budget_bytes : (uint64_t)(0.8 * (double)free_b);
  ctx->max_inflight = p.max_inflight_jobs > 0 ? p.max_inflight_jobs : 16;
  ctx->max_batch_chains = p.max_batch_chains > 0 ? p.max_batch_chains : 4 * 16 * ctx->sms;
  const int ns = p.n_streams > 0 ? p.n_streams : 4;
  for (int i = 0; i < ns; ++i) {
    cudaStream_t s;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    ctx->streams.push_back(s);
  }
  // Synchronous calls (grid builds, scoring) run at the highest stream priority:
  // their CTAs are scheduled ahead of the job streams' pending chain CTAs, so a
  // grid build does not wait for the docking kernels already on the GPU.
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (p.stream) {
    ctx->sync_stream = (cudaStream_t)p.stream;
    ctx->own_sync_stream = false;
  } else {
    cudaStreamCreateWithPriority(&ctx->sync_stream, cudaStreamNonBlocking, prio_greatest);
  }
  cudaStreamCreateWithPriority(&ctx->alloc_stream, cudaStreamNonBlocking, prio_greatest);
  cudaStreamCreateWithPriority(&ctx->upload_stream, cudaStreamNonBlocking, prio_greatest);
  ctx->alloc = p.alloc;
  ctx->free_fn = p.free;
  if (!ctx->alloc) {
    // A pool of the context's own that keeps freed memory (up to the budget)
    // instead of returning it to the driver at each synchronisation: grids and
    // jobs come and go at serving rates, and re-mapping tens of MB per grid
    // costs milliseconds.
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&ctx->pool, &props) == cudaSuccess) {
      uint64_t keep = ctx->budget;
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      ctx->pool = nullptr;
    }
  }
  ctx->alloc_user = p.alloc_user;
  if (!ctx->alloc) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, p.device) == cudaSuccess) {
      uint64_t thr = ctx->budget;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  ctx->stats.bytes_budget = ctx->budget;
  ctx->progress = std::thread(progress_loop, ctx);
  *out = ctx;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_destroy(dsdp_ctx* ctx) {
  if (!ctx) return DSDP_OK;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (uint64_t id : ctx->queue) ctx->jobs[id]->state = JobState::Cancelled;
    ctx->queue.clear();
    ctx->stop = true;
  }
  ctx->cv_work.notify_all();
  if (ctx->progress.joinable()) ctx->progress.join();
  cudaSetDevice(ctx->device);
  for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s);
  for (Batch* b : ctx->batches) {
    for (Job* j : b->jobs) job_release_device(ctx, j);
    dsdp_plan_destroy(ctx, b->plan);
    cudaEventDestroy(b->ev_start);
    cudaEventDestroy(b->ev_done);
    delete b;
  }
  ctx->batches.clear();
  for (auto& kv : ctx->jobs) {
    Job* j = kv.second;
    if (j->h_res) cudaFreeHost(j->h_res);
    delete j;
  }
  ctx->jobs.clear();
  for (auto& kv : ctx->pinned_pool) cudaFreeHost(kv.second);
  ctx->pinned_pool.clear();
  for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s), cudaStreamDestroy(s);
  cudaStreamSynchronize(ctx->alloc_stream);
  cudaStreamDestroy(ctx->alloc_stream);
  cudaStreamSynchronize(ctx->upload_stream);
  cudaStreamDestroy(ctx->upload_stream);
  cudaStreamSynchronize(ctx->sync_stream);
  if (ctx->own_sync_stream) cudaStreamDestroy(ctx->sync_stream);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_get_stats(dsdp_ctx* ctx, dsdp_stats* out) {
  if (!ctx || !out) return set_error(DSDP_ERR_INVALID_ARG, "ctx/out NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  *out = ctx->stats;
  out->queued = (int32_t)ctx->queue.size();
  out->running = ctx->running;
  out->bytes_in_use = ctx->in_use;
  out->bytes_budget = ctx->budget;
  return DSDP_OK;
}

// ------------------------------------------------------------------ grids
static dsdp_status check_receptor_host(const dsdp_receptor* r) {
  if (!r || r->n < 1 || !r->xyz || !r->xs_type) return set_error(DSDP_ERR_INVALID_ARG, "receptor arrays invalid");
  for (int i = 0; i < r->n; ++i) {
    if (r->xs_type[i] > DSDP_XS_N_DA) return set_error(DSDP_ERR_INVALID_ARG, "receptor atom %d type %d", i, r->xs_type[i]);
    for (int a = 0; a < 3; ++a)
      if (!isfinite(r->xyz[3 * i + a])) return set_error(DSDP_ERR_INVALID_ARG, "receptor atom %d not finite", i);
  }
  return DSDP_OK;
}

static dsdp_status grid_alloc(dsdp_ctx* ctx, const dsdp_receptor* receptor, const dsdp_box* box,
                              dsdp_map_dtype dtype, dsdp_grid_mode mode, dsdp_grid** out) {
  dsdp_status s = validate_box(box);
  if (s != DSDP_OK) return s;
  if ((int)dtype < 0 || (int)dtype > 2 || (int)mode < 0 || (int)mode > 1)
    return set_error(DSDP_ERR_INVALID_ARG, "bad map dtype/mode");
  dsdp_grid* g = new dsdp_grid();
  g->ctx = ctx;
  g->box = *box;
  grid_geometry(box, g->n, g->origin);
  g->dtype = (int)dtype;
  g->mode = (int)mode;
  g->map_bytes = dsdp_grid_map_bytes(box, dtype, mode);
  if (receptor) {
    g->n_rec = receptor->n;
    g->rec_bytes = up256((size_t)receptor->n * 12) + up256((size_t)receptor->n);
  }
  const uint64_t need = g->map_bytes + g->rec_bytes;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (need > ctx->budget) {
      delete g;
      return set_error(DSDP_ERR_OUT_OF_MEMORY, "grid of %llu bytes exceeds the budget", (unsigned long long)need);
    }
    ctx->in_use += need;
  }
  g->d_maps = ctx_alloc(ctx, g->map_bytes, nullptr);
  if (receptor) {
    uint8_t* r = (uint8_t*)ctx_alloc(ctx, g->rec_bytes, nullptr);
    if (r) {
      g->d_rec_xyz = (float*)r;
      g->d_rec_type = r + up256((size_t)receptor->n * 12);
    }
  }
  if (!g->d_maps || (receptor && !g->d_rec_xyz)) {
    dsdp_grid_free(ctx, g);
    return set_error(DSDP_ERR_OUT_OF_MEMORY, "grid device allocation failed");
  }
  cudaError_t e = cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming);
  if (e == cudaSuccess && receptor) {
    // pageable sources: each copy returns once the caller's array has been read;
    // the upload stream holds only such copies, so it never waits for kernels
    e = cudaMemcpyAsync(g->d_rec_xyz, receptor->xyz, (size_t)receptor->n * 12, cudaMemcpyHostToDevice,
                        ctx->upload_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g->d_rec_type, receptor->xs_type, receptor->n, cudaMemcpyHostToDevice, ctx->upload_stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->ready, ctx->upload_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->sync_stream, g->ready, 0);
  }
  if (e != cudaSuccess) {
    dsdp_grid_free(ctx, g);
    return check_cuda(e, "receptor upload");
  }
  *out = g;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_grid_build(dsdp_ctx* ctx, const dsdp_receptor* receptor, const dsdp_box* box,
                                       dsdp_map_dtype dtype, dsdp_grid_mode mode, dsdp_grid** out) {
  if (!ctx || !out) return set_error(DSDP_ERR_INVALID_ARG, "ctx/out NULL");
  *out = nullptr;
  dsdp_status s = check_receptor_host(receptor);
  if (s != DSDP_OK) return s;
  cudaSetDevice(ctx->device);
  dsdp_grid* g = nullptr;
  s = grid_alloc(ctx, receptor, box, dtype, mode, &g);
  if (s != DSDP_OK) return s;
  dsdp_receptor dr{g->n_rec, g->d_rec_xyz, g->d_rec_type};
  s = dsdp_grid_build_device(&dr, box, dtype, mode, g->d_maps, g->map_bytes, (void*)ctx->sync_stream);
  // no host wait: jobs on this grid wait for `ready` on the device
  if (s == DSDP_OK) s = check_cuda(cudaEventRecord(g->ready, ctx->sync_stream), "grid build event");
  if (s != DSDP_OK) {
    dsdp_grid_free(ctx, g);
    return s;
  }
  *out = g;
  return DSDP_OK;
}

// FP32 host maps -> stored dtype (round to nearest even).
static uint16_t f32_to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffff) ? 0x40 : 0));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static float bf16_to_f32(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
static uint16_t f32_to_f16(float f) {
  uint32_t x;
  memcpy(&x, &f, 4);
  const uint32_t sign = (x >> 16) & 0x8000u;
  int32_t exp = (int32_t)((x >> 23) & 0xff) - 127 + 15;
  uint32_t mant = x & 0x7fffffu;
  if (((x >> 23) & 0xff) == 0xff) return (uint16_t)(sign | 0x7c00u | (mant ? 0x200u : 0u));
  if (exp >= 31) return (uint16_t)(sign | 0x7c00u);
  if (exp <= 0) {
    if (exp < -10) return (uint16_t)sign;
    mant |= 0x800000u;
    const int shift = 14 - exp;
    uint32_t half = mant >> shift;
    const uint32_t rem = mant & ((1u << shift) - 1u), mid = 1u << (shift - 1);
    if (rem > mid || (rem == mid && (half & 1u))) ++half;
    return (uint16_t)(sign | half);
  }
  uint32_t h = sign | ((uint32_t)exp << 10) | (mant >> 13);
  const uint32_t rem = mant & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
  return (uint16_t)h;
}
static float f16_to_f32(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const int exp = (h >> 10) & 0x1f;
  const uint32_t mant = h & 0x3ffu;
  float f;
  if (exp == 0) {
    f = ldexpf((float)mant, -24);
    uint32_t u;
    memcpy(&u, &f, 4);
    u |= sign;
    memcpy(&f, &u, 4);
    return f;
  }
  uint32_t u = exp == 31 ? (sign | 0x7f800000u | (mant << 13)) : (sign | ((uint32_t)(exp - 15 + 127) << 23) | (mant << 13));
  memcpy(&f, &u, 4);
  return f;
}

extern "C" dsdp_status dsdp_grid_from_maps(dsdp_ctx* ctx, const dsdp_receptor* receptor, const dsdp_box* box,
                                           dsdp_map_dtype dtype, dsdp_grid_mode mode, const float* maps,
                                           dsdp_grid** out) {
  if (!ctx || !out || !maps) return set_error(DSDP_ERR_INVALID_ARG, "ctx/out/maps NULL");
  *out = nullptr;
  if (receptor) {
    dsdp_status s = check_receptor_host(receptor);
    if (s != DSDP_OK) return s;
  }
  cudaSetDevice(ctx->device);
  dsdp_grid* g = nullptr;
  dsdp_status s = grid_alloc(ctx, receptor, box, dtype, mode, &g);
  if (s != DSDP_OK) return s;
  const size_t count = (size_t)DSDP_NUM_MAP_TYPES * g->n[0] * g->n[1] * g->n[2] * (mode == DSDP_GRID_EQ4 ? 4 : 1);
  cudaError_t e;
  if (dtype == DSDP_MAP_F32) {
    e = cudaMemcpy(g->d_maps, maps, count * 4, cudaMemcpyHostToDevice);
  } else {
    std::vector<uint16_t> h(count);
    for (size_t i = 0; i < count; ++i) h[i] = dtype == DSDP_MAP_BF16 ? f32_to_bf16(maps[i]) : f32_to_f16(maps[i]);
    e = cudaMemcpy(g->d_maps, h.data(), count * 2, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    dsdp_grid_free(ctx, g);
    return check_cuda(e, "maps upload");
  }
  *out = g;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_grid_download(dsdp_ctx* ctx, const dsdp_grid* g, float* maps, size_t capacity_floats) {
  if (!ctx || !g || !maps) return set_error(DSDP_ERR_INVALID_ARG, "ctx/grid/maps NULL");
  const size_t count = (size_t)DSDP_NUM_MAP_TYPES * g->n[0] * g->n[1] * g->n[2] * (g->mode == DSDP_GRID_EQ4 ? 4 : 1);
  if (capacity_floats < count) return set_error(DSDP_ERR_INVALID_ARG, "capacity %zu < %zu floats", capacity_floats, count);
  cudaSetDevice(ctx->device);
  cudaError_t e = g->ready ? cudaEventSynchronize(g->ready) : cudaSuccess;  // the build may still run
  if (e != cudaSuccess) return check_cuda(e, "grid build");
  if (g->dtype == DSDP_MAP_F32) {
    e = cudaMemcpy(maps, g->d_maps, count * 4, cudaMemcpyDeviceToHost);
  } else {
    std::vector<uint16_t> h(count);
    e = cudaMemcpy(h.data(), g->d_maps, count * 2, cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < count; ++i) maps[i] = g->dtype == DSDP_MAP_BF16 ? bf16_to_f32(h[i]) : f16_to_f32(h[i]);
  }
  return check_cuda(e, "maps download");
}

extern "C" dsdp_status dsdp_grid_info(const dsdp_grid* g, int32_t n[3], double origin[3], double* spacing,
                                      uint64_t* map_bytes) {
  if (!g) return set_error(DSDP_ERR_INVALID_ARG, "grid NULL");
  for (int a = 0; a < 3; ++a) {
    if (n) n[a] = g->n[a];
    if (origin) origin[a] = g->origin[a];
  }
  if (spacing) *spacing = g->box.spacing;
  if (map_bytes) *map_bytes = g->map_bytes;
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_grid_free(dsdp_ctx* ctx, dsdp_grid* g) {
  if (!g) return DSDP_OK;
  if (!ctx) ctx = g->ctx;
  if (g->users.load() > 0) return set_error(DSDP_ERR_INVALID_ARG, "grid still used by %d job(s)", g->users.load());
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->upload_stream);
  cudaStreamSynchronize(ctx->sync_stream);
  ctx_free(ctx, g->d_maps, g->map_bytes, nullptr);
  ctx_free(ctx, g->d_rec_xyz, g->rec_bytes, nullptr);
  if (g->ready) cudaEventDestroy(g->ready);
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->in_use -= g->map_bytes + g->rec_bytes;
  }
  delete g;
  return DSDP_OK;
}

static void grid_view_of(const dsdp_grid* g, dsdp_grid_view* v) {
  memset(v, 0, sizeof(*v));
  v->d_maps = g->d_maps;
  for (int a = 0; a < 3; ++a) {
    v->n[a] = g->n[a];
    v->origin[a] = g->origin[a];
  }
  v->spacing = g->box.spacing;
  v->dtype = g->dtype;
  v->mode = g->mode;
}

// ------------------------------------------------------------------ scoring
namespace dsdp {
cudaError_t launch_scale_scores(float* energy, float* grad, int n_conf, int nd, int n_torsions, cudaStream_t st);
}

extern "C" dsdp_status dsdp_score_eval(dsdp_ctx* ctx, const dsdp_grid* grid, const dsdp_ligand* ligand,
                                       const double* conf, int32_t n_conf, double* energy, double* grad,
                                       uint32_t flags) {
  if (!ctx || !grid || !conf || n_conf < 0) return set_error(DSDP_ERR_INVALID_ARG, "score_eval arguments");
  if ((flags & DSDP_TERM_ALL) == 0 || (flags & ~(uint32_t)(DSDP_TERM_ALL | DSDP_TERM_NORMALISED)))
    return set_error(DSDP_ERR_INVALID_ARG, "flags must select DSDP_TERM_INTER and/or DSDP_TERM_INTRA "
                                           "(optionally with DSDP_TERM_NORMALISED)");
  if (n_conf == 0) return DSDP_OK;
  uint64_t bytes = 0;
  dsdp_status s = dsdp_ligand_pack(ligand, nullptr, 0, &bytes);
  if (s != DSDP_OK) return s;
  std::vector<uint8_t> blob(bytes);
  s = dsdp_ligand_pack(ligand, blob.data(), bytes, &bytes);
  if (s != DSDP_OK) return s;
  int32_t N, T, P, B;
  dsdp_ligand_blob_info(blob.data(), &N, &T, &P, &B);
  const size_t nx = 7 + T, nd = 6 + T;
  std::vector<float> cf((size_t)n_conf * nx);
  for (size_t i = 0; i < cf.size(); ++i) cf[i] = (float)conf[i];
  cudaSetDevice(ctx->device);
  const size_t o_conf = up256(bytes), o_e = o_conf + up256(cf.size() * 4), o_g = o_e + up256((size_t)n_conf * 4);
  const size_t total = o_g + up256((size_t)n_conf * nd * 4);
  uint8_t* d = (uint8_t*)ctx_alloc(ctx, total, nullptr);
  if (!d) return set_error(DSDP_ERR_OUT_OF_MEMORY, "score_eval buffers");
  cudaError_t e = cudaMemcpyAsync(d, blob.data(), bytes, cudaMemcpyHostToDevice, ctx->sync_stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + o_conf, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice, ctx->sync_stream);
  dsdp_grid_view v;
  grid_view_of(grid, &v);
  if (e == cudaSuccess) {
    s = dsdp_score_eval_device(&v, blob.data(), d, (const float*)(d + o_conf), n_conf, (float*)(d + o_e),
                               grad ? (float*)(d + o_g) : nullptr, flags & DSDP_TERM_ALL, (void*)ctx->sync_stream);
    if (s == DSDP_OK && (flags & DSDP_TERM_NORMALISED))
      s = check_cuda(launch_scale_scores((float*)(d + o_e), grad ? (float*)(d + o_g) : nullptr, n_conf, (int)nd, T,
                                         ctx->sync_stream),
                     "score normalisation");
  } else {
    s = check_cuda(e, "score_eval upload");
  }
  std::vector<float> he((size_t)n_conf), hg(grad ? (size_t)n_conf * nd : 0);
  if (s == DSDP_OK) {
    e = cudaMemcpyAsync(he.data(), d + o_e, he.size() * 4, cudaMemcpyDeviceToHost, ctx->sync_stream);
    if (e == cudaSuccess && grad)
      e = cudaMemcpyAsync(hg.data(), d + o_g, hg.size() * 4, cudaMemcpyDeviceToHost, ctx->sync_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->sync_stream);
    if (e != cudaSuccess) s = check_cuda(e, "score_eval");
  } else {
    cudaStreamSynchronize(ctx->sync_stream);
  }
  ctx_free(ctx, d, total, nullptr);
  if (s != DSDP_OK) return s;
  if (energy)
    for (int i = 0; i < n_conf; ++i) energy[i] = he[i];
  if (grad)
    for (size_t i = 0; i < hg.size(); ++i) grad[i] = hg[i];
  return DSDP_OK;
}

// ------------------------------------------------------------------ docking
// A job from its arguments: parameters normalised, ligand packed, binding-site
// points copied behind the blob, result layout computed.  Touches no ctx
// state, so several threads may build jobs at once; on failure the message is
// in this thread's dsdp_last_error().
static dsdp_status job_build(const dsdp_grid* grid, const dsdp_ligand* ligand, const dsdp_dock_params* params,
                             Job** out) {
  *out = nullptr;
  if (!grid) return set_error(DSDP_ERR_INVALID_ARG, "grid is NULL");
  if (!grid->d_rec_xyz) return set_error(DSDP_ERR_INVALID_ARG, "grid has no receptor atoms (needed to rescore)");
  Job* j = new Job();
  dsdp_status s = normalize_params(params, &j->params);
  if (s != DSDP_OK) {
    delete j;
    return s;
  }
  uint64_t bytes = 0;
  s = dsdp_ligand_pack(ligand, nullptr, 0, &bytes);
  if (s == DSDP_OK) {
    j->blob.resize(bytes);
    s = dsdp_ligand_pack(ligand, j->blob.data(), bytes, &bytes);
  }
  if (s != DSDP_OK) {
    delete j;
    return s;
  }
  int32_t P, B;
  dsdp_ligand_blob_info(j->blob.data(), &j->n_atoms, &j->T, &P, &B);
  if (j->params.n_site_points > 0) {
    // the caller's points are borrowed for this call: keep a copy behind the blob
    if (!params->site_points) {
      delete j;
      return set_error(DSDP_ERR_INVALID_ARG, "n_site_points > 0 but site_points is NULL");
    }
    for (int i = 0; i < 3 * j->params.n_site_points; ++i)
      if (!isfinite(params->site_points[i])) {
        delete j;
        return set_error(DSDP_ERR_INVALID_ARG, "site point coordinate %d not finite", i);
      }
    j->sites_off = (j->blob.size() + 15) & ~(size_t)15;
    j->blob.resize(j->sites_off + sizeof(float) * 3 * j->params.n_site_points);
    memcpy(j->blob.data() + j->sites_off, params->site_points, sizeof(float) * 3 * j->params.n_site_points);
  }
  j->params.site_points = nullptr;
  j->grid = grid;
  layout_results(j);
  *out = j;
  return DSDP_OK;
}

// Queue built jobs, all or none (a job larger than the whole budget refuses
// the set), and wake the progress thread once: jobs queued together can be
// taken in one batch.
static dsdp_status job_enqueue(dsdp_ctx* ctx, const std::vector<Job*>& jobs, uint64_t* job_ids) {
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (size_t i = 0; i < jobs.size(); ++i) {
      const Job* j = jobs[i];
      const uint64_t need = up256(j->blob.size()) + j->res_bytes + plan_scratch_estimate(j);
      if (need > ctx->budget) {
        for (Job* d : jobs) delete d;
        return set_error(DSDP_ERR_OUT_OF_MEMORY, "job %zu needs %llu bytes, budget %llu", i,
                         (unsigned long long)need, (unsigned long long)ctx->budget);
      }
    }
    const auto now = std::chrono::steady_clock::now();
    for (size_t i = 0; i < jobs.size(); ++i) {
      Job* j = jobs[i];
      j->id = ctx->next_id++;
      j->t_submit = now;
      const_cast<dsdp_grid*>(j->grid)->users++;
      ctx->jobs[j->id] = j;
      ctx->queue.push_back(j->id);
      ctx->stats.submitted++;
      job_ids[i] = j->id;
    }
  }
  ctx->cv_work.notify_all();
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_dock_submit(dsdp_ctx* ctx, const dsdp_grid* grid, const dsdp_ligand* ligand,
                                        const dsdp_dock_params* params, uint64_t* job_id) {
  if (!ctx || !grid || !job_id) return set_error(DSDP_ERR_INVALID_ARG, "ctx/grid/job_id NULL");
  Job* j = nullptr;
  const dsdp_status s = job_build(grid, ligand, params, &j);
  if (s != DSDP_OK) return s;
  return job_enqueue(ctx, {j}, job_id);
}

extern "C" dsdp_status dsdp_dock_submit_many(dsdp_ctx* ctx, int32_t n, const dsdp_grid* const* grids,
                                             const dsdp_ligand* ligands, const dsdp_dock_params* params,
                                             uint64_t* job_ids) {
  if (!ctx || n < 0 || (n > 0 && (!grids || !ligands || !params || !job_ids)))
    return set_error(DSDP_ERR_INVALID_ARG, "ctx/grids/ligands/params/job_ids NULL or n < 0");
  if (n == 0) return DSDP_OK;
  std::vector<Job*> jobs((size_t)n, nullptr);
  std::vector<dsdp_status> st((size_t)n, DSDP_OK);
  std::vector<std::string> msg((size_t)n);
  // ligand packing (torsion tree, pair list, step schedule) is the host's
  // work per job: spread it over a few threads
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int n_thr = (int)std::min<unsigned>(std::min<unsigned>(hw, 8u), (unsigned)n);
  auto work = [&](int t) {
    for (int i = t; i < n; i += n_thr) {
      st[i] = job_build(grids[i], &ligands[i], &params[i], &jobs[i]);
      if (st[i] != DSDP_OK) msg[i] = dsdp_last_error();
    }
  };
  if (n_thr == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    pool.reserve(n_thr - 1);
    for (int t = 1; t < n_thr; ++t) pool.emplace_back(work, t);
    work(0);
    for (std::thread& th : pool) th.join();
  }
  for (int i = 0; i < n; ++i)
    if (st[i] != DSDP_OK) {
      for (Job* j : jobs) delete j;
      return set_error(st[i], "job %d: %s", i, msg[i].c_str());
    }
  return job_enqueue(ctx, jobs, job_ids);
}

static void copy_results(const Job* j, dsdp_dock_result* out) {
  const uint8_t* r = (const uint8_t*)j->h_res;
  const int nx = 7 + j->T, k = j->params.top_k, C = j->params.n_chains;
  int n_out = *(const int32_t*)(r + j->o_n);
  if (n_out < 0 || n_out > k) n_out = 0;
  const int m = std::min(n_out, std::max(out->capacity, 0));
  out->n_out = m;
  out->n_atoms = j->n_atoms;
  out->n_torsions = j->T;
  if (out->score) memcpy(out->score, r + j->o_score, sizeof(double) * m);
  if (out->inter) memcpy(out->inter, r + j->o_inter, sizeof(double) * m);
  if (out->intra) memcpy(out->intra, r + j->o_intra, sizeof(double) * m);
  if (out->conf) memcpy(out->conf, r + j->o_conf, sizeof(double) * m * nx);
  if (out->coords) memcpy(out->coords, r + j->o_coords, sizeof(float) * m * j->n_atoms * 3);
  if (out->chain) memcpy(out->chain, r + j->o_chain, sizeof(int32_t) * m);
  if (out->chain_best_e) memcpy(out->chain_best_e, r + j->o_cbe, sizeof(float) * C);
  if (out->chain_best_conf) memcpy(out->chain_best_conf, r + j->o_cbc, sizeof(float) * (size_t)C * nx);
  if (out->trace && j->params.trace)
    memcpy(out->trace, r + j->o_trace, sizeof(float) * (size_t)C * (j->params.n_mc_steps + 1) * (nx + 4));
  const uint32_t* ev = (const uint32_t*)(r + j->o_evals);
  uint64_t total = 0;
  for (int c = 0; c < C; ++c) total += ev[c];
  out->n_evals = total;
}

extern "C" dsdp_status dsdp_dock_poll(dsdp_ctx* ctx, uint64_t job_id, dsdp_dock_result* out, int32_t wait_ms) {
  if (!ctx) return set_error(DSDP_ERR_INVALID_ARG, "ctx NULL");
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto it = ctx->jobs.find(job_id);
  if (it == ctx->jobs.end()) return set_error(DSDP_ERR_NOT_FOUND, "job %llu not found", (unsigned long long)job_id);
  Job* j = it->second;
  auto finished = [&] { return j->state != JobState::Queued && j->state != JobState::Running; };
  if (!finished() && wait_ms != 0) {
    if (wait_ms < 0) ctx->cv_done.wait(lk, finished);
    else ctx->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), finished);
  }
  if (!finished()) {
    if (wait_ms > 0)
      return set_error(DSDP_ERR_TIMEOUT, "job %llu not finished after %d ms (still %s; poll again)",
                       (unsigned long long)job_id, wait_ms, j->state == JobState::Queued ? "queued" : "running");
    return DSDP_PENDING;
  }
  dsdp_status s = DSDP_OK;
  if (j->state == JobState::Done) {
    if (out) {
      copy_results(j, out);
      out->device_ms = j->device_ms;
      out->latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    }
  } else if (j->state == JobState::Cancelled) {
    s = set_error(DSDP_ERR_CANCELLED, "job %llu was cancelled", (unsigned long long)job_id);
  } else {
    s = set_error(j->err, "job %llu failed: %s", (unsigned long long)job_id, j->msg.c_str());
  }
  pinned_put(ctx, j);
  ctx->jobs.erase(it);
  lk.unlock();
  delete j;
  return s;
}

extern "C" dsdp_status dsdp_dock_cancel(dsdp_ctx* ctx, uint64_t job_id) {
  if (!ctx) return set_error(DSDP_ERR_INVALID_ARG, "ctx NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->jobs.find(job_id);
  if (it == ctx->jobs.end()) return set_error(DSDP_ERR_NOT_FOUND, "job %llu not found", (unsigned long long)job_id);
  Job* j = it->second;
  if (j->state == JobState::Queued) {
    ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), job_id), ctx->queue.end());
    j->state = JobState::Cancelled;
    const_cast<dsdp_grid*>(j->grid)->users--;
    ctx->stats.cancelled++;
    ctx->cv_done.notify_all();
    return DSDP_OK;
  }
  if (j->state == JobState::Running) {
    // its kernels are in flight with other jobs' (a batch is one launch): they
    // finish, and the job's results are dropped when the batch retires
    j->cancel_requested = true;
    return DSDP_OK;
  }
  return DSDP_OK;
}
