// Torsion normalisation of scores evaluated by the handle API: energies (and
// their gradients) divided by 1 + w_rot T, the convention of the reported
// docking scores (Vina's torsion term, which the paper keeps).
#include <cuda_runtime.h>

#include "dsdp_internal.h"

namespace dsdp {
namespace {

__global__ void scale_scores_kernel(float* __restrict__ energy, float* __restrict__ grad, int n_conf, int nd,
                                    float s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_conf) return;
  if (energy) energy[i] *= s;
  if (grad)
    for (int k = 0; k < nd; ++k) grad[(size_t)i * nd + k] *= s;
}

}  // namespace

cudaError_t launch_scale_scores(float* energy, float* grad, int n_conf, int nd, int n_torsions, cudaStream_t st) {
  if (n_conf <= 0) return cudaSuccess;
  const float s = (float)(1.0 / (1.0 + kWRot * n_torsions));
  const int block = 256, grid = (n_conf + block - 1) / block;
  scale_scores_kernel<<<grid, block, 0, st>>>(energy, grad, n_conf, nd, s);
  return cudaGetLastError();
}

}  // namespace dsdp
