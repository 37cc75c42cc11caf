// Postprocess of a docking job (Fig. 4: the sampled poses are ranked after the
// copies finish), on the device and in FP64: every chain's best pose is
// rebuilt with FP64 kinematics and scored gridless (exact pair sums against
// the receptor atoms, plus intra); poses are sorted by the torsion-normalised
// inter score, near-duplicates (heavy-atom RMSD below a cut) are dropped and
// the best top_k are written out.
#include <string.h>

#include <mutex>

#include "launch.h"
#include "chain_device.cuh"

namespace dsdp {
namespace {

constexpr int kRescoreWarps = 8;
constexpr int kRecTile = 1024;

struct DQuat {
  double w, x, y, z;
};
__device__ __forceinline__ DQuat dqmul(const DQuat& a, const DQuat& b) {
  return DQuat{a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
               a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ double3 dqrot(const DQuat& q, double3 v) {
  const double tx = 2.0 * (q.y * v.z - q.z * v.y), ty = 2.0 * (q.z * v.x - q.x * v.z),
               tz = 2.0 * (q.x * v.y - q.y * v.x);
  return make_double3(v.x + q.w * tx + (q.y * tz - q.z * ty), v.y + q.w * ty + (q.z * tx - q.x * tz),
                      v.z + q.w * tz + (q.x * ty - q.y * tx));
}
__device__ __forceinline__ double shd(double v, int src) { return __shfl_sync(kFull, v, src); }

// One warp per chain: FP64 pose, exact inter (receptor staged through shared
// memory in tiles, FP32 pre-filter then FP64 distance) and intra.
__global__ void __launch_bounds__(32 * kRescoreWarps) rescore_kernel(const DevJob* __restrict__ jobs,
                                                                     const Tile* __restrict__ tiles) {
  __shared__ float4 s_rec[kRecTile];
  __shared__ double s_xyz[kRescoreWarps][kMaxAtoms * 3];
  __shared__ int s_type[kRescoreWarps][kMaxAtoms];
  __shared__ uint32_t s_list[kRescoreWarps][64];
  const Tile tile = tiles[blockIdx.x];
  const DevJob& J = jobs[tile.job];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool has_chain = warp < tile.count;
  const int chain = tile.chain0 + warp;
  const LigView L = view_blob(J.blob);  // read through the cache; small
  const double* atom64 = reinterpret_cast<const double*>(J.blob + L.h->off_atom64);
  const double* body64 = reinterpret_cast<const double*>(J.blob + L.h->off_body64);
  const int T = L.T, N = L.n_atoms, nb = L.n_bodies;
  double3 pos[2];
  int type[2];
  bool valid[2];
  if (has_chain) {
    const float* cf = J.chain_best_conf + (size_t)chain * (7 + T);
    DQuat q{(double)cf[3], (double)cf[4], (double)cf[5], (double)cf[6]};
    const double qn = sqrt(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
    q = DQuat{q.w / qn, q.x / qn, q.y / qn, q.z / qn};
    const double3 p = make_double3(cf[0], cf[1], cf[2]);
    DQuat Q{1.0, 0.0, 0.0, 0.0};
    double3 O = make_double3(0.0, 0.0, 0.0);
    int ptr = -1;
    if (lane == 0) {
      Q = q;
      O = p;
    } else if (lane < nb) {
      const BodyRec& b = L.body[lane];
      const double* g = body64 + 6 * lane;
      const double th = (double)cf[7 + b.torsion];
      const double s = sin(0.5 * th), c = cos(0.5 * th);
      Q = DQuat{c, s * g[3], s * g[4], s * g[5]};
      O = make_double3(g[0], g[1], g[2]);
      ptr = b.parent;
    }
    for (int r = 0; r < L.rounds; ++r) {
      const int src = ptr >= 0 ? ptr : lane;
      const DQuat Qp{shd(Q.w, src), shd(Q.x, src), shd(Q.y, src), shd(Q.z, src)};
      const double3 Op = make_double3(shd(O.x, src), shd(O.y, src), shd(O.z, src));
      const int pp = __shfl_sync(kFull, ptr, src);
      if (ptr >= 0) {
        const double3 ro = dqrot(Qp, O);
        O = make_double3(Op.x + ro.x, Op.y + ro.y, Op.z + ro.z);
        Q = dqmul(Qp, Q);
        ptr = pp;
      }
    }
    for (int s = 0; s < 2; ++s) {
      const int i = lane + 32 * s;
      valid[s] = i < N;
      const float4 a = valid[s] ? L.atom[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      const int packed = __float_as_int(a.w);
      type[s] = packed & 0xff;
      const int b = valid[s] ? (packed >> 8) & 0xff : 0;
      const DQuat Qb{shd(Q.w, b), shd(Q.x, b), shd(Q.y, b), shd(Q.z, b)};
      const double3 Ob = make_double3(shd(O.x, b), shd(O.y, b), shd(O.z, b));
      const double3 r = valid[s] ? dqrot(Qb, make_double3(atom64[3 * i], atom64[3 * i + 1], atom64[3 * i + 2]))
                                 : make_double3(0.0, 0.0, 0.0);
      pos[s] = make_double3(Ob.x + r.x, Ob.y + r.y, Ob.z + r.z);
      if (valid[s]) {
        s_type[warp][i] = type[s];
        s_xyz[warp][3 * i + 0] = pos[s].x;
        s_xyz[warp][3 * i + 1] = pos[s].y;
        s_xyz[warp][3 * i + 2] = pos[s].z;
        double* out = J.chain_coords + ((size_t)chain * N + i) * 3;
        out[0] = pos[s].x;
        out[1] = pos[s].y;
        out[2] = pos[s].z;
      }
    }
  } else {
    valid[0] = valid[1] = false;
    type[0] = type[1] = 0;
    pos[0] = pos[1] = make_double3(0.0, 0.0, 0.0);
  }
  // Inter, exact: for each receptor tile staged in shared memory, the warp scans
  // (ligand atom, receptor atom) pairs with an FP32 pre-filter (cutoff + 0.05 A),
  // compacts the survivors into a per-warp list by ballot, and evaluates them in
  // FP64 32 at a time with every lane busy.
  const float pre2 = (kCutoff + 0.05f) * (kCutoff + 0.05f);
  uint32_t* list = s_list[warp];
  int n_list = 0;
  double e_inter = 0.0;
  auto flush = [&](int count) {
    if (lane < count) {
      const uint32_t ent = list[lane];
      const int i = ent >> 16, k = ent & 0xffff;
      const float4 a = s_rec[k];
      const double dx = s_xyz[warp][3 * i] - (double)a.x, dy = s_xyz[warp][3 * i + 1] - (double)a.y,
                   dz = s_xyz[warp][3 * i + 2] - (double)a.z;
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r < kCutoffD) {
        const int ti = s_type[warp][i], tj = min(__float_as_int(a.w), 8);
        e_inter += vina_pair_f64(r - (c_xs_radius_d[ti] + c_xs_radius_d[tj]), pair_bits(ti, tj));
      }
    }
  };
  for (int r0 = 0; r0 < J.n_rec; r0 += kRecTile) {
    const int cnt = min(kRecTile, J.n_rec - r0);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const int j = r0 + k;
      s_rec[k] = make_float4(J.rec_xyz[3 * j], J.rec_xyz[3 * j + 1], J.rec_xyz[3 * j + 2],
                             __int_as_float((int)J.rec_type[j]));
    }
    __syncthreads();
    if (!has_chain) continue;
    for (int i = 0; i < N; ++i) {
      const float px = (float)s_xyz[warp][3 * i], py = (float)s_xyz[warp][3 * i + 1],
                  pz = (float)s_xyz[warp][3 * i + 2];
      for (int k0 = 0; k0 < cnt; k0 += 32) {
        const int k = k0 + lane;
        bool pass = false;
        if (k < cnt) {
          const float4 a = s_rec[k];
          const float fx = px - a.x, fy = py - a.y, fz = pz - a.z;
          pass = fx * fx + fy * fy + fz * fz < pre2;
        }
        const unsigned bal = __ballot_sync(kFull, pass);
        if (pass) list[n_list + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)i << 16) | (uint32_t)k;
        n_list += __popc(bal);
        __syncwarp();
        if (n_list >= 32) {
          flush(32);
          __syncwarp();
          const uint32_t rest = lane < n_list - 32 ? list[32 + lane] : 0u;
          __syncwarp();
          if (lane < n_list - 32) list[lane] = rest;
          n_list -= 32;
          __syncwarp();
        }
      }
    }
    flush(n_list);  // the list refers to this tile: empty it before the next one is staged
    n_list = 0;
    __syncwarp();
  }
  if (!has_chain) return;
  __syncwarp();
  double e_intra = 0.0;
  for (int p = lane; p < L.n_pairs; p += 32) {
    const uint32_t pr = L.pair_rec[p].x;
    const int i = (pr & 0xffff) >> 4, j = pr >> 20;
    const double dx = s_xyz[warp][3 * i] - s_xyz[warp][3 * j], dy = s_xyz[warp][3 * i + 1] - s_xyz[warp][3 * j + 1],
                 dz = s_xyz[warp][3 * i + 2] - s_xyz[warp][3 * j + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r < kCutoffD)) continue;
    const int ti = __float_as_int(L.atom[i].w) & 0xff, tj = __float_as_int(L.atom[j].w) & 0xff;
    e_intra += vina_pair_f64(r - (c_xs_radius_d[ti] + c_xs_radius_d[tj]), pair_bits(ti, tj));
  }
  e_inter = warp_sum_d(e_inter);
  e_intra = warp_sum_d(e_intra);
  if (lane == 0) {
    J.chain_inter[chain] = e_inter;
    J.chain_intra[chain] = e_intra;
    J.chain_score[chain] = e_inter / (1.0 + kWRot * (double)T);
  }
}

// One CTA per job: bitonic sort of (score, chain), greedy RMSD de-duplication,
// top-k output in the caller's atom order.
__global__ void __launch_bounds__(512) topk_kernel(const DevJob* __restrict__ jobs, int np2) {
  extern __shared__ __align__(16) uint8_t smem[];
  double* key = reinterpret_cast<double*>(smem);
  int* idx = reinterpret_cast<int*>(smem + sizeof(double) * np2);
  __shared__ int s_kept[DSDP_MAX_TOP_K];
  __shared__ int s_nkept;
  __shared__ int s_dup;
  const DevJob& J = jobs[blockIdx.x];
  const int n = J.n_chains;
  const LigView L = view_blob(J.blob);
  const int N = L.n_atoms, T = L.T;
  int size = 1;
  while (size < n) size <<= 1;
  for (int i = threadIdx.x; i < size; i += blockDim.x) {
    double k = 1.0 / 0.0;
    if (i < n) {
      k = J.chain_score[i];
      if (k != k) k = 1.0 / 0.0;  // NaN ranks last
    }
    key[i] = k;
    idx[i] = i < n ? i : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= size; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < size; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const bool gt = key[i] > key[ixj] || (key[i] == key[ixj] && idx[i] > idx[ixj]);
          if (gt == up) {
            const double tk = key[i];
            key[i] = key[ixj];
            key[ixj] = tk;
            const int ti = idx[i];
            idx[i] = idx[ixj];
            idx[ixj] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) s_nkept = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const double cut2n = (double)J.rmsd_dedup * (double)J.rmsd_dedup * (double)N;
  for (int pos = 0; pos < n; ++pos) {
    const int kept = s_nkept;
    if (kept >= J.top_k) break;
    const int c = idx[pos];
    if (threadIdx.x == 0) s_dup = 0;
    __syncthreads();
    for (int q = warp; q < kept; q += nwarps) {
      const double* a = J.chain_coords + (size_t)c * N * 3;
      const double* b = J.chain_coords + (size_t)s_kept[q] * N * 3;
      double sum = 0.0;
      for (int i = lane; i < N; i += 32) {
        const double dx = a[3 * i] - b[3 * i], dy = a[3 * i + 1] - b[3 * i + 1], dz = a[3 * i + 2] - b[3 * i + 2];
        sum += dx * dx + dy * dy + dz * dz;
      }
      sum = warp_sum_d(sum);
      if (lane == 0 && sum < cut2n) s_dup = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0 && !s_dup) {
      s_kept[kept] = c;
      s_nkept = kept + 1;
    }
    __syncthreads();
  }
  const int kept = s_nkept;
  if (threadIdx.x == 0 && J.out_n) J.out_n[0] = kept;
  for (int q = threadIdx.x; q < kept; q += blockDim.x) {
    const int c = s_kept[q];
    if (J.out_chain) J.out_chain[q] = c;
    if (J.out_score) J.out_score[q] = J.chain_score[c];
    if (J.out_inter) J.out_inter[q] = J.chain_inter[c];
    if (J.out_intra) J.out_intra[q] = J.chain_intra[c];
  }
  if (J.out_conf)
    for (int e = threadIdx.x; e < kept * (7 + T); e += blockDim.x) {
      const int q = e / (7 + T), k = e % (7 + T);
      J.out_conf[e] = (double)J.chain_best_conf[(size_t)s_kept[q] * (7 + T) + k];
    }
  if (J.out_coords)
    for (int e = threadIdx.x; e < kept * N; e += blockDim.x) {
      const int q = e / N, i = e % N;
      const int u = L.atom_user[i];
      const double* src = J.chain_coords + ((size_t)s_kept[q] * N + i) * 3;
      float* dst = J.out_coords + ((size_t)q * N + u) * 3;
      dst[0] = (float)src[0];
      dst[1] = (float)src[1];
      dst[2] = (float)src[2];
    }
}

}  // namespace

cudaError_t launch_rescore(const void* jobs, const void* tiles, int n_tiles, cudaStream_t st) {
  if (n_tiles <= 0) return cudaSuccess;
  rescore_kernel<<<n_tiles, 32 * kRescoreWarps, 0, st>>>(reinterpret_cast<const DevJob*>(jobs),
                                                         reinterpret_cast<const Tile*>(tiles));
  return cudaGetLastError();
}

int rescore_tile_chains() { return kRescoreWarps; }

cudaError_t launch_topk(const void* jobs, int n_jobs, int max_chains, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  int np2 = 1;
  while (np2 < max_chains) np2 <<= 1;
  const size_t smem = (size_t)np2 * (sizeof(double) + sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  topk_kernel<<<n_jobs, 512, smem, st>>>(reinterpret_cast<const DevJob*>(jobs), np2);
  return cudaGetLastError();
}

}  // namespace dsdp

// ---------------------------------------------------------------------------
// FP64 rescoring + top-k without any allocation (dsdp_rescore_topk_noalloc).
//
// For callers that cannot allocate device memory at the point of the call --
// code running under an allocator lock or inside a framework's memory-planning
// phase, a real-time thread that must not take the driver's allocation path,
// or a host that owns a fixed device budget -- the scratch this postprocess
// needs (the job record, the rescoring tiles, per-chain scores and FP64
// coordinates) lives in one file-scope device array.  Every GPU that loads the
// library holds it (DSDP_NOALLOC_SCRATCH_BYTES) until the process exits.
// ---------------------------------------------------------------------------
namespace dsdp {
namespace {

constexpr int kNoAllocMaxChains = DSDP_NOALLOC_MAX_CHAINS;
constexpr size_t kNoAllocJobOff = 0;
constexpr size_t kNoAllocTileOff = 512;
constexpr size_t kNoAllocTiles = (kNoAllocMaxChains + kRescoreWarps - 1) / kRescoreWarps;
constexpr size_t kNoAllocScoreOff = kNoAllocTileOff + ((sizeof(Tile) * kNoAllocTiles + 255) & ~(size_t)255);
constexpr size_t kNoAllocInterOff = kNoAllocScoreOff + sizeof(double) * kNoAllocMaxChains;
constexpr size_t kNoAllocIntraOff = kNoAllocInterOff + sizeof(double) * kNoAllocMaxChains;
constexpr size_t kNoAllocCoordOff = kNoAllocIntraOff + sizeof(double) * kNoAllocMaxChains;
constexpr size_t kNoAllocBytes = kNoAllocCoordOff + sizeof(double) * 3 * kMaxAtoms * kNoAllocMaxChains;
static_assert(sizeof(DevJob) <= kNoAllocTileOff, "job record must fit its slot");
static_assert(kNoAllocBytes == DSDP_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Writes the job record and its rescoring tiles into the scratch array; the
// record arrives as a kernel parameter, so no host buffer has to outlive the call.
__global__ void noalloc_tables_kernel(DevJob job, DevJob* job_out, Tile* tiles_out, int n_tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *job_out = job;
  if (t < n_tiles) {
    const int c0 = t * kRescoreWarps;
    tiles_out[t] = Tile{0, c0, min(kRescoreWarps, job.n_chains - c0), 0};
  }
}

// Device address of g_noalloc_scratch, resolved once per device by the first
// call there (the host-side symbol is only a stand-in and must never reach a
// kernel).  Under lazy module loading that first call may also load this
// file's kernels and commit the array; the cached address is valid for the
// life of the device's primary context, so the library is not used across a
// device reset.
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

dsdp_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return check_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(DSDP_ERR_DEVICE, "device ordinal %d beyond 63", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return check_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return DSDP_OK;
}

}  // namespace
}  // namespace dsdp

using namespace dsdp;

extern "C" dsdp_status dsdp_rescore_topk_noalloc(const dsdp_job_device* job, void* stream) {
  if (!job) return set_error(DSDP_ERR_INVALID_ARG, "job is NULL");
  int32_t n_atoms = 0, T = 0, P = 0, B = 0;
  dsdp_status s = dsdp_ligand_blob_info(job->h_blob, &n_atoms, &T, &P, &B);
  if (s != DSDP_OK) return s;
  dsdp_dock_params p;
  s = normalize_params(&job->params, &p);
  if (s != DSDP_OK) return s;
  if (p.n_chains > kNoAllocMaxChains)
    return set_error(DSDP_ERR_INVALID_ARG, "n_chains %d exceeds the no-alloc limit of %d chains (scratch %zu bytes)",
                     p.n_chains, kNoAllocMaxChains, (size_t)kNoAllocBytes);
  if (!job->d_blob || !job->d_chain_best_conf || job->receptor.n < 1 || !job->receptor.xyz ||
      !job->receptor.xs_type)
    return set_error(DSDP_ERR_INVALID_ARG, "no-alloc rescoring needs d_blob, d_chain_best_conf and the receptor");
  void* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != DSDP_OK) return s;
  unsigned char* sc = static_cast<unsigned char*>(base);
  DevJob d;
  memset(&d, 0, sizeof(d));
  d.blob = (const uint8_t*)job->d_blob;
  d.n_chains = p.n_chains;
  d.chain_best_conf = job->d_chain_best_conf;
  d.n_rec = job->receptor.n;
  d.rec_xyz = job->receptor.xyz;
  d.rec_type = job->receptor.xs_type;
  d.chain_score = reinterpret_cast<double*>(sc + kNoAllocScoreOff);
  d.chain_inter = reinterpret_cast<double*>(sc + kNoAllocInterOff);
  d.chain_intra = reinterpret_cast<double*>(sc + kNoAllocIntraOff);
  d.chain_coords = reinterpret_cast<double*>(sc + kNoAllocCoordOff);
  d.top_k = p.top_k;
  d.rmsd_dedup = (float)p.rmsd_dedup;
  d.out_n = job->d_out_n;
  d.out_chain = job->d_out_chain;
  d.out_score = job->d_out_score;
  d.out_inter = job->d_out_inter;
  d.out_intra = job->d_out_intra;
  d.out_conf = job->d_out_conf;
  d.out_coords = job->d_out_coords;
  const cudaStream_t st = (cudaStream_t)stream;
  DevJob* d_job = reinterpret_cast<DevJob*>(sc + kNoAllocJobOff);
  Tile* d_tiles = reinterpret_cast<Tile*>(sc + kNoAllocTileOff);
  const int n_tiles = (p.n_chains + kRescoreWarps - 1) / kRescoreWarps;
  noalloc_tables_kernel<<<(n_tiles + 127) / 128, 128, 0, st>>>(d, d_job, d_tiles, n_tiles);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_rescore(d_job, d_tiles, n_tiles, st);
  if (e == cudaSuccess) e = launch_topk(d_job, 1, p.n_chains, st);
  return check_cuda(e, "no-alloc rescoring launch");
}
