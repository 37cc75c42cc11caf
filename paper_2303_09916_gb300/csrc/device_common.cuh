// Device helpers shared by the kernels of libdsdp (sm_103a).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dsdp_internal.h"

namespace dsdp {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kPiF = 3.14159265358979323846f;
constexpr float kTwoPiF = 6.28318530717958647692f;

// Per-type tables (Vina XS types 0..8): radius and bits (1 hydrophobic,
// 2 donor, 4 acceptor).
static __constant__ float c_xs_radius[9] = {1.9f, 1.9f, 1.8f, 1.8f, 1.8f, 1.7f, 1.7f, 2.0f, 1.8f};
static __constant__ int c_xs_bits[9] = {1, 0, 0, 2, 4, 4, 6, 0, 6};
static __constant__ double c_xs_radius_d[9] = {1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0, 1.8};

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): ten rounds; each round multiplies words 0 and 2 by the two Philox
// constants, swaps in the high halves xor-ed with the key and the other words,
// and bumps the key by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint32_t pick(uint4 v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// Stream of one chain: word w of block b at MC step s is word w of
// Philox(counter (chain, s, b, 0), key (seed_lo, seed_hi)).
struct ChainStream {
  uint32_t k0, k1, chain;
  __device__ __forceinline__ uint4 block(uint32_t step, uint32_t b) const {
    return philox4x32_10(make_uint4(chain, step, b, 0u), k0, k1);
  }
  // top 24 bits * 2^-24: exact in FP32
  __device__ __forceinline__ static float to_uniform(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
};

// Uniform point in the unit ball: attempt a (0..15) uses block 1 + a; the
// coordinates are (word >> 8) - 2^23, accepted when the integer sum of squares
// is <= 2^46; the point is v / 2^23.  All lanes compute the same point.
__device__ __forceinline__ float3 unit_ball(const ChainStream& s, uint32_t step) {
  for (int a = 0; a < 16; ++a) {
    const uint4 v = s.block(step, 1u + a);
    const long long x = (long long)(v.x >> 8) - (1ll << 23);
    const long long y = (long long)(v.y >> 8) - (1ll << 23);
    const long long z = (long long)(v.z >> 8) - (1ll << 23);
    if (x * x + y * y + z * z <= (1ll << 46))
      return make_float3((float)x * (1.0f / 8388608.0f), (float)y * (1.0f / 8388608.0f),
                         (float)z * (1.0f / 8388608.0f));
  }
  return make_float3(0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------ small math
// Hardware approximations (PTX ISA rsqrt.approx, sin.approx, cos.approx) in
// their .ftz forms: subnormal inputs and results flush to zero.  Every caller
// passes normal numbers (or zero), where the .ftz and non-.ftz forms return the
// same value; the .ftz forms skip the subnormal scaling the non-.ftz ones add
// around each instruction (45 warp instructions per ligand evaluation).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sin_ftz(float x) {
  float y;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float cos_ftz(float x) {
  float y;
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
struct Quat {
  float w, x, y, z;
};

__device__ __forceinline__ Quat qmul(const Quat& a, const Quat& b) {
  Quat r;
  r.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  r.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  r.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  r.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  return r;
}

// R(q) v for a unit quaternion: v + w t + u x t with t = 2 u x v.
__device__ __forceinline__ float3 qrot(const Quat& q, const float3& v) {
  const float tx = 2.f * (q.y * v.z - q.z * v.y);
  const float ty = 2.f * (q.z * v.x - q.x * v.z);
  const float tz = 2.f * (q.x * v.y - q.y * v.x);
  return make_float3(v.x + q.w * tx + (q.y * tz - q.z * ty), v.y + q.w * ty + (q.z * tx - q.x * tz),
                     v.z + q.w * tz + (q.x * ty - q.y * tx));
}

__device__ __forceinline__ Quat qnormalize(const Quat& q) {
  const float inv = rsqrt_ftz(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return Quat{q.w * inv, q.x * inv, q.y * inv, q.z * inv};
}

// Unit quaternion of a rotation vector w: (cos(|w|/2), sin(|w|/2) w/|w|).  Below
// |w| = 1/16 the Taylor series of cos(x/2) and sin(x/2)/x is used (truncation
// error < 1e-12).  Above it, h = |w|/2 = a2 rsqrt(a2) / 2 is reduced to
// [-pi, pi] by h - 2 pi n, n = rint(h / 2 pi), with 2 pi split in two FP32
// parts (Cody & Waite) so that the reduction adds no error of its own for the
// angles a line search tries, and the hardware sin / cos approximations (absolute
// error a few 1e-7 on [-pi, pi]) take the reduced angle.  Every caller
// normalises the product it forms with the result.
__device__ __forceinline__ Quat quat_from_rotvec(float wx, float wy, float wz) {
  const float a2 = wx * wx + wy * wy + wz * wz;
  float c, k;
  if (a2 < 1.f / 256.f) {
    c = 1.f + a2 * (-1.f / 8.f + a2 * (1.f / 384.f));
    k = 0.5f + a2 * (-1.f / 48.f + a2 * (1.f / 3840.f));
  } else {
    constexpr float kTwoPiHi = 6.28318548f;     // 2 pi rounded to FP32
    constexpr float kTwoPiLo = -1.74845553e-7f;  // 2 pi - kTwoPiHi
    const float r = rsqrt_ftz(a2);
    const float h = 0.5f * (a2 * r);
    const float n = rintf(h * (1.f / kTwoPiHi));
    const float hr = fmaf(-n, kTwoPiLo, fmaf(-n, kTwoPiHi, h));
    c = cos_ftz(hr);
    k = sin_ftz(hr) * r;
  }
  return Quat{c, wx * k, wy * k, wz * k};
}

// Wrap to (-pi, pi].
__device__ __forceinline__ float wrap_angle(float t) {
  return t - kTwoPiF * ceilf((t - kPiF) * (1.f / kTwoPiF));
}

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float3 shfl3(float3 v, int src) {
  return make_float3(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src), __shfl_sync(kFull, v.z, src));
}
__device__ __forceinline__ Quat shflq(const Quat& q, int src) {
  return Quat{__shfl_sync(kFull, q.w, src), __shfl_sync(kFull, q.x, src), __shfl_sync(kFull, q.y, src),
              __shfl_sync(kFull, q.z, src)};
}

// ------------------------------------------------------------------ pair score
// 2^x by the ex2.approx instruction (PTX ISA: relative error about 2^-22,
// subnormal results flushed to zero).  exp(x) = 2^(x / ln 2): callers fold the
// 1 / ln 2 into their constants.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kLog2E = 1.44269504088896340736f;  // 1 / ln 2
constexpr float kFarD = 100.f;                     // surface distance where every term and slope is 0

__device__ __forceinline__ float2 splat2(float a) { return make_float2(a, a); }

// gauss1 + gauss2 + repulsion of two surface distances in packed FP32x2
// arithmetic (fma / mul / add .f32x2 of sm_100+): returns e and de/dd of each.
__device__ __forceinline__ void steric_x2(float2 d, float2& e, float2& de) {
  const float2 u1 = __fmul2_rn(__fmul2_rn(d, d), splat2(-4.f * kLog2E));  // -(d / 0.5)^2 / ln 2
  const float2 b = __ffma2_rn(d, splat2(0.5f), splat2(-1.5f));             // (d - 3) / 2
  const float2 u2 = __fmul2_rn(__fmul2_rn(b, b), splat2(-kLog2E));        // -b^2 / ln 2
  const float2 g1 = make_float2(ex2_approx(u1.x), ex2_approx(u1.y));
  const float2 g2 = make_float2(ex2_approx(u2.x), ex2_approx(u2.y));
  const float2 m = make_float2(fminf(d.x, 0.f), fminf(d.y, 0.f));
  float2 ee = __fmul2_rn(g1, splat2(kWGauss1));
  ee = __ffma2_rn(g2, splat2(kWGauss2), ee);
  e = __ffma2_rn(__fmul2_rn(m, m), splat2(kWRepulsion), ee);
  float2 dd = __fmul2_rn(g1, __fmul2_rn(d, splat2(-8.f * kWGauss1)));
  dd = __ffma2_rn(g2, __fmul2_rn(b, splat2(-kWGauss2)), dd);
  de = __ffma2_rn(m, splat2(2.f * kWRepulsion), dd);
}

// Two intra-ligand pairs per lane in packed FP32x2 arithmetic: the Vina-form
// pair score (the scoring function DSDP keeps, Sec. 2: weighted gauss1, gauss2,
// repulsion, hydrophobic and H-bond terms of the surface distance d) without
// per-lane branches, with d = r2 / r + nrs, nrs = -(R_i + R_j), returning e and
// (de/dd) / r.  hydrophobic = min(max(1.5 - d, 0), 1) and H-bond =
// min(max(-d / 0.7, 0), 1) equal the piecewise forms (1 below 0.5 / -0.7, 0 from
// 1.5 / 0); their slopes are taken on the half-open intervals [0.5, 1.5) and
// [-0.7, 0), the branch of the strict inequality at a breakpoint.
// Pairs at or beyond the cutoff take d = kFarD, and idle slots get a surface
// distance at least kStepIdleNrs: there every term and slope is exactly zero.
// cls0 / cls1: terms the two pairs carry (1 hydrophobic, 2 H-bond); use_hyd /
// use_hb: warp-uniform, false when no pair of the two steps carries the term.
__device__ __forceinline__ void vina_pair_x2(float2 r2, float2 nrs, uint32_t cls0, uint32_t cls1, bool use_hyd,
                                             bool use_hb, float2& e, float2& s) {
  // 1e-30 keeps an idle slot's r2 = 0 finite (r2 ir = 0 there); real pairs are
  // Angstroms apart, where it changes nothing
  const float2 rp = __fadd2_rn(r2, splat2(1e-30f));
  const float2 ir = make_float2(rsqrt_ftz(rp.x), rsqrt_ftz(rp.y));
  float2 d = __ffma2_rn(r2, ir, nrs);
  d.x = r2.x < kCutoff * kCutoff ? d.x : kFarD;
  d.y = r2.y < kCutoff * kCutoff ? d.y : kFarD;
  float2 ee, de;
  steric_x2(d, ee, de);
  if (use_hyd) {  // min(max(1.5 - d, 0), 1), slope on [0.5, 1.5)
    const float2 wh = make_float2((cls0 & 1u) ? kWHydrophobic : 0.f, (cls1 & 1u) ? kWHydrophobic : 0.f);
    const float2 t = __ffma2_rn(d, splat2(-1.f), splat2(1.5f));
    ee = __ffma2_rn(wh, make_float2(__saturatef(t.x), __saturatef(t.y)), ee);
    if (d.x >= 0.5f && d.x < 1.5f) de.x -= wh.x;
    if (d.y >= 0.5f && d.y < 1.5f) de.y -= wh.y;
  }
  if (use_hb) {  // min(max(-d / 0.7, 0), 1), slope on [-0.7, 0)
    const float2 wb = make_float2((cls0 & 2u) ? kWHBond : 0.f, (cls1 & 2u) ? kWHBond : 0.f);
    const float2 t = __fmul2_rn(d, splat2(-1.f / 0.7f));
    ee = __ffma2_rn(wb, make_float2(__saturatef(t.x), __saturatef(t.y)), ee);
    if (d.x >= -0.7f && d.x < 0.f) de.x -= wb.x * (1.f / 0.7f);
    if (d.y >= -0.7f && d.y < 0.f) de.y -= wb.y * (1.f / 0.7f);
  }
  e = ee;
  s = __fmul2_rn(de, ir);
}

__device__ __forceinline__ int pair_bits(int ti, int tj) {
  const int a = c_xs_bits[ti], b = c_xs_bits[tj];
  int bits = (a & b & 1);
  if (((a & 2) && (b & 4)) || ((a & 4) && (b & 2))) bits |= 2;
  return bits;
}

// FP64 version for the rescoring (same terms; exp in double).
__device__ __forceinline__ double vina_pair_f64(double d, int bits) {
  const double a = 2.0 * d;
  const double b = 0.5 * (d - 3.0);
  double e = kWGauss1D * exp(-a * a) + kWGauss2D * exp(-b * b);
  if (d < 0.0) e += kWRepulsionD * d * d;
  if (bits & 1) {
    if (d < 0.5) e += kWHydrophobicD;
    else if (d < 1.5) e += kWHydrophobicD * (1.5 - d);
  }
  if (bits & 2) {
    if (d < -0.7) e += kWHBondD;
    else if (d < 0.0) e += kWHBondD * (-d / 0.7);
  }
  return e;
}

// ------------------------------------------------------------------ map formats
// FMT encodes (dtype, mode): 0 F32 EQ4, 1 BF16 EQ4, 2 F16 EQ4, 3 F32 EQ3,
// 4 BF16 EQ3, 5 F16 EQ3.
__host__ __device__ constexpr int map_fmt(int dtype, int mode) { return mode * 3 + dtype; }
__host__ __device__ constexpr int fmt_channels(int fmt) { return fmt < 3 ? 4 : 1; }
__host__ __device__ constexpr int fmt_elem_bytes(int fmt) { return (fmt % 3 == 0) ? 4 : 2; }

template <int FMT>
__device__ __forceinline__ float4 load_node(const void* maps, unsigned idx) {
  if (FMT == 0) {
    return __ldg(reinterpret_cast<const float4*>(maps) + idx);
  } else if (FMT == 1 || FMT == 2) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(maps) + idx);
    if (FMT == 1) {
      const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
      const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
      const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      return make_float4(fa.x, fa.y, fb.x, fb.y);
    } else {
      const __half2 a = *reinterpret_cast<const __half2*>(&raw.x);
      const __half2 b = *reinterpret_cast<const __half2*>(&raw.y);
      const float2 fa = __half22float2(a), fb = __half22float2(b);
      return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
  } else if (FMT == 3) {
    return make_float4(__ldg(reinterpret_cast<const float*>(maps) + idx), 0.f, 0.f, 0.f);
  } else {
    const unsigned short raw = __ldg(reinterpret_cast<const unsigned short*>(maps) + idx);
    float v;
    if (FMT == 4) v = __bfloat162float(__ushort_as_bfloat16(raw));
    else v = __half2float(__ushort_as_half(raw));
    return make_float4(v, 0.f, 0.f, 0.f);
  }
}

struct MapView {
  const void* maps;
  int nx, ny, nz;
  float ox, oy, oz;
  float h, inv_h;
};

// Cell of a point in the grid: clamped position u = (r - origin) / h in
// [0, n - 1], cell index (lower corner, at most n - 2), fractions within the
// cell, and the signed excess (Angstrom) along each axis outside the grid.
struct MapCell {
  unsigned base;     // node index of corner (ix, iy, iz) of type 0; add type * nxyz
  float fx, fy, fz;
  float ex, ey, ez;
};

__device__ __forceinline__ MapCell map_cell(const MapView& M, float3 r) {
  const float ux = (r.x - M.ox) * M.inv_h, uy = (r.y - M.oy) * M.inv_h, uz = (r.z - M.oz) * M.inv_h;
  const float cx = fminf(fmaxf(ux, 0.f), (float)(M.nx - 1));
  const float cy = fminf(fmaxf(uy, 0.f), (float)(M.ny - 1));
  const float cz = fminf(fmaxf(uz, 0.f), (float)(M.nz - 1));
  const int ix = min((int)cx, M.nx - 2), iy = min((int)cy, M.ny - 2), iz = min((int)cz, M.nz - 2);
  MapCell c;
  // 32-bit node indices: the host rejects grids with 8 nx ny nz >= 2^31 nodes.
  c.base = ((unsigned)iz * (unsigned)M.ny + (unsigned)iy) * (unsigned)M.nx + (unsigned)ix;
  c.fx = cx - (float)ix;
  c.fy = cy - (float)iy;
  c.fz = cz - (float)iz;
  c.ex = (ux - cx) * M.h;
  c.ey = (uy - cy) * M.h;
  c.ez = (uz - cz) * M.h;
  return c;
}

// Trilinear score (Eq. 2) and gradient (Eq. 4 from the gradient maps, or
// Eq. 3 as the derivative of the interpolant) for map type t in cell c, with the
// out-of-grid wall: evaluated at the clamped point plus kWallSlope per
// Angstrom of excess along each axis; along such an axis the gradient is the
// wall slope.
template <int FMT>
__device__ __forceinline__ float map_interp(const MapView& M, int t, const MapCell& c, float3& g) {
  const unsigned sxy = (unsigned)M.nx * (unsigned)M.ny;
  const unsigned base = (unsigned)t * sxy * (unsigned)M.nz + c.base;
  const float4 v000 = load_node<FMT>(M.maps, base);
  const float4 v100 = load_node<FMT>(M.maps, base + 1);
  const float4 v010 = load_node<FMT>(M.maps, base + M.nx);
  const float4 v110 = load_node<FMT>(M.maps, base + M.nx + 1);
  const float4 v001 = load_node<FMT>(M.maps, base + sxy);
  const float4 v101 = load_node<FMT>(M.maps, base + sxy + 1);
  const float4 v011 = load_node<FMT>(M.maps, base + sxy + M.nx);
  const float4 v111 = load_node<FMT>(M.maps, base + sxy + M.nx + 1);
  const float fx = c.fx, fy = c.fy, fz = c.fz;
  const float gx0 = 1.f - fx, gy0 = 1.f - fy, gz0 = 1.f - fz;
  const float w000 = gx0 * gy0 * gz0, w100 = fx * gy0 * gz0, w010 = gx0 * fy * gz0, w110 = fx * fy * gz0;
  const float w001 = gx0 * gy0 * fz, w101 = fx * gy0 * fz, w011 = gx0 * fy * fz, w111 = fx * fy * fz;
  float e = w000 * v000.x + w100 * v100.x + w010 * v010.x + w110 * v110.x + w001 * v001.x + w101 * v101.x +
            w011 * v011.x + w111 * v111.x;
  if (fmt_channels(FMT) == 4) {
    g.x = w000 * v000.y + w100 * v100.y + w010 * v010.y + w110 * v110.y + w001 * v001.y + w101 * v101.y +
          w011 * v011.y + w111 * v111.y;
    g.y = w000 * v000.z + w100 * v100.z + w010 * v010.z + w110 * v110.z + w001 * v001.z + w101 * v101.z +
          w011 * v011.z + w111 * v111.z;
    g.z = w000 * v000.w + w100 * v100.w + w010 * v010.w + w110 * v110.w + w001 * v001.w + w101 * v101.w +
          w011 * v011.w + w111 * v111.w;
  } else {
    // d/dx of the trilinear interpolant: difference of the x = 1 and x = 0 faces / h
    const float f0 = gy0 * gz0 * v000.x + fy * gz0 * v010.x + gy0 * fz * v001.x + fy * fz * v011.x;
    const float f1 = gy0 * gz0 * v100.x + fy * gz0 * v110.x + gy0 * fz * v101.x + fy * fz * v111.x;
    const float e0 = gx0 * gz0 * v000.x + fx * gz0 * v100.x + gx0 * fz * v001.x + fx * fz * v101.x;
    const float e1 = gx0 * gz0 * v010.x + fx * gz0 * v110.x + gx0 * fz * v011.x + fx * fz * v111.x;
    const float d0 = gx0 * gy0 * v000.x + fx * gy0 * v100.x + gx0 * fy * v010.x + fx * fy * v110.x;
    const float d1 = gx0 * gy0 * v001.x + fx * gy0 * v101.x + gx0 * fy * v011.x + fx * fy * v111.x;
    g.x = (f1 - f0) * M.inv_h;
    g.y = (e1 - e0) * M.inv_h;
    g.z = (d1 - d0) * M.inv_h;
  }
  if (c.ex != 0.f) {
    e += kWallSlope * fabsf(c.ex);
    g.x = c.ex > 0.f ? kWallSlope : -kWallSlope;
  }
  if (c.ey != 0.f) {
    e += kWallSlope * fabsf(c.ey);
    g.y = c.ey > 0.f ? kWallSlope : -kWallSlope;
  }
  if (c.ez != 0.f) {
    e += kWallSlope * fabsf(c.ez);
    g.z = c.ez > 0.f ? kWallSlope : -kWallSlope;
  }
  return e;
}

template <int FMT>
__device__ __forceinline__ float sample_map(const MapView& M, int t, float3 r, float3& g) {
  return map_interp<FMT>(M, t, map_cell(M, r), g);
}

__host__ __device__ inline MapView make_map_view(const DevJob& J) {
  MapView M;
  M.maps = J.maps;
  M.nx = J.n[0];
  M.ny = J.n[1];
  M.nz = J.n[2];
  M.ox = J.origin[0];
  M.oy = J.origin[1];
  M.oz = J.origin[2];
  M.h = J.spacing;
  M.inv_h = J.inv_spacing;
  return M;
}

}  // namespace dsdp
