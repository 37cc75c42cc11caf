// Host-side launch descriptions of the kernels (included by the .cu files only).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "chain_device.cuh"

namespace dsdp {

struct ChainLaunch {
  const void* jobs;   // DevJob[] (device)
  const void* tiles;  // Tile[] (device)
  int n_tiles;
  int* tile_counter;  // device int, zeroed before a persistent launch
  int persistent;
  int grid;           // CTAs
  int warps_per_cta;
  int apl;            // largest atoms-per-lane tile present
  int apl_mask;       // tiles present: bit 0 one atom per lane (<= 32 atoms), bit 1 two (<= 64)
  int blob_smem;      // bytes reserved for the largest staged blob prefix
  ScratchLayout scratch;  // per-warp scratch, sized for the group's largest ligand
  int variant;        // register budget of the chain kernel (0: 128, 1: 96)
};

struct ScoreLaunch {
  MapView map;
  const uint8_t* blob;  // device
  const float* conf;
  int n_conf;
  float* energy;
  float* grad;
  uint32_t flags;
  int apl;
  int blob_smem;
  ScratchLayout scratch;
};

#define DSDP_DECLARE_FMT(F)                                               \
  cudaError_t launch_chains_fmt##F(const ChainLaunch& a, cudaStream_t st); \
  cudaError_t launch_score_fmt##F(const ScoreLaunch& a, cudaStream_t st);
DSDP_DECLARE_FMT(0)
DSDP_DECLARE_FMT(1)
DSDP_DECLARE_FMT(2)
DSDP_DECLARE_FMT(3)
DSDP_DECLARE_FMT(4)
DSDP_DECLARE_FMT(5)
#undef DSDP_DECLARE_FMT

MapView map_view_of(const dsdp_grid_view* g);
cudaError_t launch_rescore(const void* jobs, const void* tiles, int n_tiles, cudaStream_t st);
int rescore_tile_chains();
cudaError_t launch_topk(const void* jobs, int n_jobs, int max_chains, cudaStream_t st);

}  // namespace dsdp
