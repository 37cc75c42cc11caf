// Chain and scoring kernels, instantiated once per map format by the
// dock_fmt*.cu translation units (compiled in parallel).
#pragma once
#include "chain_device.cuh"
#include "launch.h"

namespace dsdp {

// Register budgets of the chain kernel: variant 0 caps at 128 registers (16
// warps per SM, no spills), variant 1 at 96 (20 warps), 2 at 80 (24 warps) and
// 3 at 72 (28 warps), each with a few more bytes spilled; the autotuner picks
// per plan by measurement.  Variants 2 and 3 are compiled for the
// one-atom-per-lane tiles only (two atoms per lane and mixed tiles take
// variants 0 and 1; a plan asking for more falls back to the 96-register
// kernel).  The bounds are stated for CTAs of up to 4 warps (chains); CTAs of
// 1 or 2 warps get the same register cap.
constexpr int kMaxChainWarps = 4;
template <int VAR>
struct ChainOcc;
template <>
struct ChainOcc<0> {
  static constexpr int kMinBlocks = 4;  // 65536 / (128 * 4) = 128 registers
};
template <>
struct ChainOcc<1> {
  static constexpr int kMinBlocks = 5;  // 102 -> 96 registers
};
template <>
struct ChainOcc<2> {
  static constexpr int kMinBlocks = 6;  // 85 -> 80 registers
};
template <>
struct ChainOcc<3> {
  static constexpr int kMinBlocks = 7;  // 73 -> 72 registers
};
// The minimum CTAs per SM a kernel is compiled for.  Variant 1 of the
// one-atom-per-lane tiles takes none (0: the launch bound then names only the
// CTA size): the compiler's own allocation for it is 96 registers without
// spills (tests/test_kernel_registers_cpu.py checks every variant's count), and
// that kernel ran the 32-system typical-4k chain stage in 67.4 ms against 69.0
// for the same budget reached through a bound of 5 CTAs per SM (three runs
// each): the bound changes how the compiler schedules, not the register count.
template <int VAR, int APLS>
__host__ __device__ constexpr int chain_min_blocks() {
  return (VAR == 1 && APLS == 1) ? 0 : ChainOcc<VAR>::kMinBlocks;
}

// Chains: a CTA runs one tile of up to W chains of one job; W = blockDim / 32.
// The job's ligand blob is staged into shared memory once per tile; ligands of
// up to 32 atoms run one atom per lane, larger ones two, whatever else the
// launch holds (a chain's arithmetic depends on its own job only).  APLS: the
// tiles compiled in (1 or 2; 3 = both, for launches that mix them -- each
// single-tile kernel keeps its register allocation to itself).
// persistent != 0: CTAs pull tiles from *tile_counter until none are left.
template <int FMT, int VAR, int APLS>
__global__ void __launch_bounds__(32 * kMaxChainWarps, (chain_min_blocks<VAR, APLS>())) dock_chains_kernel(const DevJob* __restrict__ jobs,
                                                          const Tile* __restrict__ tiles, int n_tiles,
                                                          int* tile_counter, int persistent, int blob_smem,
                                                          ScratchLayout lay) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_tile;
  __shared__ int s_job;
  const int warp = threadIdx.x >> 5;
  const WarpScratch W = warp_scratch_at(smem + blob_smem + warp * lay.bytes, lay);
  if (threadIdx.x == 0) s_job = -1;
  __syncthreads();
  int t = blockIdx.x;
  for (;;) {
    if (persistent) {
      __syncthreads();
      if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1);
      __syncthreads();
      t = s_tile;
    }
    if (t >= n_tiles) break;
    const Tile tile = tiles[t];
    const DevJob& J = jobs[tile.job];
    if (s_job != tile.job) {  // uniform: s_job only changes between barriers
      __syncthreads();
      const int words = reinterpret_cast<const BlobHeader*>(J.blob)->stage_bytes / 16;
      for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int4*>(smem)[i] = __ldg(reinterpret_cast<const int4*>(J.blob) + i);
      __syncthreads();
      if (threadIdx.x == 0) s_job = tile.job;
      __syncthreads();
    }
    const LigView L = view_blob(smem);
    if (warp < tile.count) {
      if (APLS == 1 || (APLS == 3 && L.n_atoms <= 32)) run_chain<1, FMT, APLS == 3 ? 1 : 2>(J, L, W, tile.chain0 + warp);
      else run_chain<2, FMT>(J, L, W, tile.chain0 + warp);
    }
    if (!persistent) break;
  }
}

// Score + gradient of a batch of conformations: one warp per conformation,
// warps striding over the batch (the ligand is staged once per CTA).
template <int APL, int FMT>
__global__ void __launch_bounds__(256) score_eval_kernel(MapView M, const uint8_t* __restrict__ blob,
                                                         const float* __restrict__ conf, int n_conf,
                                                         float* __restrict__ energy, float* __restrict__ grad,
                                                         uint32_t flags, int blob_smem, ScratchLayout lay) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int words = reinterpret_cast<const BlobHeader*>(blob)->stage_bytes / 16;
  for (int i = threadIdx.x; i < words; i += blockDim.x)
    reinterpret_cast<int4*>(smem)[i] = __ldg(reinterpret_cast<const int4*>(blob) + i);
  __syncthreads();
  const LigView L = view_blob(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpScratch W = warp_scratch_at(smem + blob_smem + warp * lay.bytes, lay);
  LaneLig<APL> R;
  load_lane_lig<APL>(L, R);
  const int T = L.T;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int c = blockIdx.x * (blockDim.x >> 5) + warp; c < n_conf; c += warps) {  // warp-uniform loop
    Conf x = load_conf(conf + (size_t)c * (7 + T), T);
    x.q = qnormalize(x.q);
    float g;
    const float e = eval_conf<APL, FMT>(M, L, R, W, x, g, flags);
    if (lane == 0 && energy) energy[c] = e;
    if (grad && lane < 6 + T) grad[(size_t)c * (6 + T) + lane] = g;
  }
}

template <int FMT, int VAR, int APLS>
cudaError_t launch_chains_var(const ChainLaunch& a, cudaStream_t st) {
  const dim3 block(32 * a.warps_per_cta);
  const size_t smem = (size_t)a.blob_smem + (size_t)a.warps_per_cta * a.scratch.bytes;
  auto k = dock_chains_kernel<FMT, VAR, APLS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = a.grid;
  if (a.persistent) {
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * a.warps_per_cta, smem);
    if (e != cudaSuccess) return e;
    grid = per_sm * sms < a.n_tiles ? per_sm * sms : a.n_tiles;
    if (grid < 1) grid = 1;
  }
  k<<<grid, block, smem, st>>>(reinterpret_cast<const DevJob*>(a.jobs), reinterpret_cast<const Tile*>(a.tiles),
                               a.n_tiles, a.tile_counter, a.persistent, a.blob_smem, a.scratch);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_chains_impl(const ChainLaunch& a, cudaStream_t st) {
  if (a.warps_per_cta != 1 && a.warps_per_cta != 2 && a.warps_per_cta != kMaxChainWarps) return cudaErrorInvalidValue;
  if (a.apl_mask == 1) {
    switch (a.variant) {
      case 0: return launch_chains_var<FMT, 0, 1>(a, st);
      case 1: return launch_chains_var<FMT, 1, 1>(a, st);
      case 2: return launch_chains_var<FMT, 2, 1>(a, st);
      default: return launch_chains_var<FMT, 3, 1>(a, st);
    }
  }
  if (a.apl_mask == 2) return a.variant ? launch_chains_var<FMT, 1, 2>(a, st) : launch_chains_var<FMT, 0, 2>(a, st);
  // mixed tiles: the 128- and 96-register budgets
  return a.variant ? launch_chains_var<FMT, 1, 3>(a, st) : launch_chains_var<FMT, 0, 3>(a, st);
}

template <int FMT>
cudaError_t launch_score_impl(const ScoreLaunch& a, cudaStream_t st) {
  const int wpc = 4;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int want = (a.n_conf + wpc - 1) / wpc, cap = sms * 8;  // warps stride over the conformations
  const dim3 block(32 * wpc), grid(want < cap ? want : cap);
  const size_t smem = (size_t)a.blob_smem + (size_t)wpc * a.scratch.bytes;
  const MapView M = a.map;
  if (a.apl == 1) {
    auto k = score_eval_kernel<1, FMT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(M, a.blob, a.conf, a.n_conf, a.energy, a.grad, a.flags, a.blob_smem, a.scratch);
  } else {
    auto k = score_eval_kernel<2, FMT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(M, a.blob, a.conf, a.n_conf, a.energy, a.grad, a.flags, a.blob_smem, a.scratch);
  }
  return cudaGetLastError();
}

}  // namespace dsdp

#define DSDP_INSTANTIATE_FMT(F)                                                                   \
  namespace dsdp {                                                                                \
  cudaError_t launch_chains_fmt##F(const ChainLaunch& a, cudaStream_t st) {                       \
    return launch_chains_impl<F>(a, st);                                                          \
  }                                                                                               \
  cudaError_t launch_score_fmt##F(const ScoreLaunch& a, cudaStream_t st) {                        \
    return launch_score_impl<F>(a, st);                                                           \
  }                                                                                               \
  }
