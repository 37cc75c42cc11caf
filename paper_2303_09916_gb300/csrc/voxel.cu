// Receptor voxel features (Sec. 2, "Protein-ligand binding site prediction"):
// the input of the binding-site network, 36 x 36 x 36 voxels with 18
// channels over a 70 A cube centred on the protein; S and Se share one
// element channel and the freed channel marks the protein surface.
//
//   * voxel k of an axis covers [c - 35 + k 70/36, c - 35 + (k + 1) 70/36); an
//     atom's voxel is floor((x - (c - 35)) * (36/70)), FP32, subtraction then
//     multiplication; atoms outside the cube are dropped;
//   * channels 0..16: sums of the caller's 17 per-atom features over the
//     voxel's atoms; channel 17: the number of its surface atoms;
//   * surface atom (Shrake & Rupley, J. Mol. Biol. 79, 351 (1973)): some test
//     point x_i + (r_i + 1.4) u_k of its solvent-accessible sphere lies outside
//     the sphere of radius r_j + 1.4 of every other atom j; u_k are the 98
//     primitive integer vectors of {-2..2}^3, normalised (FP32, correctly
//     rounded square root and division); every point and distance test is FP32
//     with a fixed operation order (no contraction);
//   * sums are exact and order-free: features are rounded to multiples of 2^-24
//     and accumulated as 64-bit integers; a channel is the sum times 2^-24
//     rounded to FP32.
//
// One warp per atom: lanes hold the atom's 98 test points (four per lane); the
// warp scans the receptor 32 atoms at a time, keeps those whose sphere can
// reach the atom's (a conservative FP32 pre-test), and each lane checks its
// points against them, broadcast by shuffle.  No shared memory, no scratch
// beyond the caller's accumulator.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dsdp_internal.h"

namespace dsdp {
namespace {

constexpr int kVoxN = DSDP_VOXEL_N;
constexpr int kVoxF = DSDP_VOXEL_FEATURES;
constexpr int kVoxC = DSDP_VOXEL_CHANNELS;
constexpr int kPointsPerLane = 4;  // 128 slots for the 98 directions
constexpr float kProbe = 1.4f;
constexpr float kFix = 16777216.0f;  // 2^24

// The 98 test directions as integer vectors (a, b, c) in {-2..2}^3 with
// gcd(|a|, |b|, |c|) = 1, built at compile time; a lane normalises its own.
struct SasDirs {
  signed char v[98][3];
};
constexpr int gcd_abs(int x, int y) {
  x = x < 0 ? -x : x;
  y = y < 0 ? -y : y;
  while (y) {
    const int t = x % y;
    x = y;
    y = t;
  }
  return x;
}
constexpr SasDirs make_sas_dirs() {
  SasDirs d{};
  int m = 0;
  for (int a = -2; a <= 2; ++a)
    for (int b = -2; b <= 2; ++b)
      for (int c = -2; c <= 2; ++c) {
        if ((a == 0 && b == 0 && c == 0) || gcd_abs(gcd_abs(a, b), c) != 1) continue;
        d.v[m][0] = (signed char)a;
        d.v[m][1] = (signed char)b;
        d.v[m][2] = (signed char)c;
        ++m;
      }
  return d;
}
static_assert(make_sas_dirs().v[97][0] == 2 && make_sas_dirs().v[97][1] == 2 && make_sas_dirs().v[97][2] == 1,
              "98 primitive directions");
__constant__ SasDirs c_sas_dirs = make_sas_dirs();

// Unit test direction m (0..97): the integer vector over its FP32 length
// (correctly rounded square root and division).
__device__ __forceinline__ float3 sas_direction(int m) {
  const int a = c_sas_dirs.v[m][0], b = c_sas_dirs.v[m][1], c = c_sas_dirs.v[m][2];
  const float len = __fsqrt_rn((float)(a * a + b * b + c * c));
  return make_float3(__fdiv_rn((float)a, len), __fdiv_rn((float)b, len), __fdiv_rn((float)c, len));
}

__global__ void __launch_bounds__(256) voxel_atoms_kernel(int n, const float* __restrict__ xyz,
                                                          const float* __restrict__ radius,
                                                          const float* __restrict__ feat, float lox, float loy,
                                                          float loz, unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  float3 u[kPointsPerLane];
  bool used[kPointsPerLane];
#pragma unroll
  for (int s = 0; s < kPointsPerLane; ++s) {
    const int m = lane + 32 * s;
    used[s] = m < 98;
    u[s] = used[s] ? sas_direction(m) : make_float3(0.f, 0.f, 0.f);
  }
  const float inv = 36.0f / 70.0f;
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {  // warp-uniform
    const float xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    const float ux = __fmul_rn(__fsub_rn(xi, lox), inv), uy = __fmul_rn(__fsub_rn(yi, loy), inv),
                uz = __fmul_rn(__fsub_rn(zi, loz), inv);
    // floor(u) in [0, 36) exactly when u in [0, 36) (false for NaN): tested before any conversion
    if (!(ux >= 0.f && ux < (float)kVoxN && uy >= 0.f && uy < (float)kVoxN && uz >= 0.f && uz < (float)kVoxN))
      continue;
    const int kx = (int)ux, ky = (int)uy, kz = (int)uz;
    unsigned long long* v = acc + (((size_t)kz * kVoxN + ky) * kVoxN + kx) * kVoxC;
    if (lane < kVoxF)
      atomicAdd(v + lane, (unsigned long long)__float2ll_rn(__fmul_rn(feat[(size_t)kVoxF * i + lane], kFix)));
    // ---- surface test
    const float Ri = __fadd_rn(radius[i], kProbe);
    float px[kPointsPerLane], py[kPointsPerLane], pz[kPointsPerLane];
    bool buried[kPointsPerLane];
#pragma unroll
    for (int s = 0; s < kPointsPerLane; ++s) {
      px[s] = __fadd_rn(xi, __fmul_rn(Ri, u[s].x));
      py[s] = __fadd_rn(yi, __fmul_rn(Ri, u[s].y));
      pz[s] = __fadd_rn(zi, __fmul_rn(Ri, u[s].z));
      buried[s] = !used[s];
    }
    for (int j0 = 0; j0 < n; j0 += 32) {
      const int j = j0 + lane;
      float xj = 0.f, yj = 0.f, zj = 0.f, Rj = 0.f;
      bool near = false;
      if (j < n && j != i) {
        xj = xyz[3 * j];
        yj = xyz[3 * j + 1];
        zj = xyz[3 * j + 2];
        Rj = __fadd_rn(radius[j], kProbe);
        // a sphere farther than Ri + Rj cannot cover a point of atom i's sphere;
        // 0.01 A of slack keeps the pre-test conservative under FP32 rounding
        const float dx = xj - xi, dy = yj - yi, dz = zj - zi, reach = Ri + Rj + 0.01f;
        near = dx * dx + dy * dy + dz * dz < reach * reach;
      }
      unsigned m = __ballot_sync(0xffffffffu, near);
      while (m) {  // warp-uniform
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float bx = __shfl_sync(0xffffffffu, xj, src), by = __shfl_sync(0xffffffffu, yj, src),
                    bz = __shfl_sync(0xffffffffu, zj, src), bR = __shfl_sync(0xffffffffu, Rj, src);
        const float R2 = __fmul_rn(bR, bR);
#pragma unroll
        for (int s = 0; s < kPointsPerLane; ++s) {
          const float dx = __fsub_rn(px[s], bx), dy = __fsub_rn(py[s], by), dz = __fsub_rn(pz[s], bz);
          const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
          buried[s] = buried[s] || d2 < R2;
        }
      }
    }
    bool exposed = false;
#pragma unroll
    for (int s = 0; s < kPointsPerLane; ++s) exposed = exposed || !buried[s];
    if (__any_sync(0xffffffffu, exposed) && lane == 0) atomicAdd(v + kVoxF, (unsigned long long)(1ll << 24));
  }
}

__global__ void voxel_finish_kernel(const unsigned long long* __restrict__ acc, float* __restrict__ out, int n) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    out[q] = __double2float_rn(__ll2double_rn((long long)acc[q]) * (1.0 / 16777216.0));
}

}  // namespace
}  // namespace dsdp

using namespace dsdp;

extern "C" uint64_t dsdp_voxel_work_bytes(void) {
  return sizeof(unsigned long long) * (uint64_t)kVoxN * kVoxN * kVoxN * kVoxC;
}

extern "C" dsdp_status dsdp_voxelize_device(int32_t n_atoms, const float* d_xyz, const float* d_radius,
                                            const float* d_features, const double center[3], float* d_out,
                                            void* d_work, uint64_t work_bytes, void* stream) {
  if (n_atoms < 0) return set_error(DSDP_ERR_INVALID_ARG, "n_atoms %d < 0", n_atoms);
  if (!center || !d_out || !d_work) return set_error(DSDP_ERR_INVALID_ARG, "voxelize: center, out or work NULL");
  if (n_atoms > 0 && (!d_xyz || !d_radius || !d_features))
    return set_error(DSDP_ERR_INVALID_ARG, "voxelize: atom arrays NULL");
  if (work_bytes < dsdp_voxel_work_bytes())
    return set_error(DSDP_ERR_INVALID_ARG, "voxelize: work of %llu bytes < %llu", (unsigned long long)work_bytes,
                     (unsigned long long)dsdp_voxel_work_bytes());
  if (((uintptr_t)d_work & 7) != 0) return set_error(DSDP_ERR_INVALID_ARG, "voxelize: work not 8-byte aligned");
  for (int a = 0; a < 3; ++a)
    if (!isfinite(center[a])) return set_error(DSDP_ERR_INVALID_ARG, "voxelize: center not finite");
  const cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* acc = (unsigned long long*)d_work;
  cudaError_t e = cudaMemsetAsync(acc, 0, dsdp_voxel_work_bytes(), st);
  if (e == cudaSuccess && n_atoms > 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int want = (n_atoms + 7) / 8, cap = sms * 8;  // 8 warps (atoms) per CTA
    voxel_atoms_kernel<<<want < cap ? want : cap, 256, 0, st>>>(
        n_atoms, d_xyz, d_radius, d_features, (float)(center[0] - 35.0), (float)(center[1] - 35.0),
        (float)(center[2] - 35.0), acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int total = kVoxN * kVoxN * kVoxN * kVoxC;
    voxel_finish_kernel<<<(total + 255) / 256, 256, 0, st>>>(acc, d_out, total);
    e = cudaGetLastError();
  }
  return check_cuda(e, "voxelize launch");
}
