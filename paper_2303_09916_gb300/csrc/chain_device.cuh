// Warp-per-chain score + gradient, local optimisers and Monte Carlo chain.
//
// One warp owns one conformation.  Lanes hold atoms (APL atoms per lane, in
// the blob's depth-first order), rigid bodies (lane b = body b) and the
// components of 6 + T dimensional vectors (lane j = component j: 0..2
// position, 3..5 rotation vector, 6 + k torsion k).  The ligand topology sits
// in shared memory; grid maps are read from L2 through the read-only path.
#pragma once
#include "device_common.cuh"

namespace dsdp {

// Pointers into a staged (shared-memory) blob.
struct LigView {
  const BlobHeader* h;
  const float4* atom;
  const int32_t* atom_user;
  const BodyRec* body;
  const uint2* pair_rec;  // after the staged prefix: read from the global blob only
  const uint2* steps;
  const int32_t* torsion_body;
  const int16_t* lane_map;  // [32][2]: atom in slot s of lane l (-1 empty); lane l holds atom l up to 32 atoms
  int n_atoms, T, n_bodies, n_pairs, n_steps, rounds;
};

__device__ __forceinline__ LigView view_blob(const uint8_t* b) {
  LigView v;
  v.h = reinterpret_cast<const BlobHeader*>(b);
  v.atom = reinterpret_cast<const float4*>(b + v.h->off_atom);
  v.atom_user = reinterpret_cast<const int32_t*>(b + v.h->off_atom_user);
  v.body = reinterpret_cast<const BodyRec*>(b + v.h->off_body);
  v.pair_rec = reinterpret_cast<const uint2*>(b + v.h->off_pairs);
  v.steps = reinterpret_cast<const uint2*>(b + v.h->off_steps);
  v.torsion_body = reinterpret_cast<const int32_t*>(b + v.h->off_torsion_body);
  v.lane_map = reinterpret_cast<const int16_t*>(b + v.h->off_lane_map);
  v.n_atoms = v.h->n_atoms;
  v.T = v.h->n_torsions;
  v.n_bodies = v.h->n_bodies;
  v.n_pairs = v.h->n_pairs;
  v.n_steps = v.h->n_steps;
  v.rounds = v.h->rounds;
  return v;
}

// Per-lane ligand data: the atoms of the lane's slots (atom lane with one atom
// per lane; the blob's lane map with two) and, on lane b < n_bodies, body b's
// record; re-read from the staged blob (shared memory) where used.
template <int APL>
struct LaneLig {
  int n_atoms, nb, T, tbody;
};

template <int APL>
__device__ __forceinline__ void load_lane_lig(const LigView& L, LaneLig<APL>& R) {
  const int lane = threadIdx.x & 31;
  R.n_atoms = L.n_atoms;
  R.nb = L.n_bodies;
  R.T = L.T;
  R.tbody = (lane >= 6 && lane < 6 + L.T) ? L.torsion_body[lane - 6] : 0;
}

// Conformation held by a warp: p and q replicated in every lane, torsion k in lane 6 + k.
struct Conf {
  float3 p;
  Quat q;
  float th;
};

// Per-warp shared scratch (layout in scratch_layout).
struct WarpScratch {
  float4* pre;     // [kMaxAtoms][2] inclusive prefix sums of (g, (r - p) x g): (gx, gy, gz, cx), (cy, cz, -, -)
  float* H;        // [6 + T][kHStride] BFGS inverse Hessian, row j owned by lane j
  float* vec;      // [5][kHStride] + 24: g', s, u broadcast to the H rows (BFGS update);
                   // the chain's g and d; its ChainVars
  float* x;        // [7 + kMaxDim] local optimiser: current iterate (BFGS) / best iterate (BB)
  float* cur;      // [7 + kMaxDim] current conformation of the chain
  float* best;     // [7 + kMaxDim] best conformation of the chain
};

constexpr int kConfFloats = 7 + kMaxDim;
// Row stride of H (floats): >= kMaxDim rounded up to float4, and 7 float4 per row
// so that rows j = 0..7 fall on distinct 16-byte bank groups (float4 row reads
// by the lanes need the minimum number of shared-memory wavefronts).
constexpr int kHStride = 28;
static_assert(kHStride >= ((kMaxDim + 3) & ~3) && (kHStride / 4) % 2 == 1, "H row stride");
__host__ __device__ constexpr int align16i(int x) { return (x + 15) & ~15; }
// Per-warp scratch sized for a group's largest ligand (n_atoms, torsions).
struct ScratchLayout {
  int pre, H, vec, x, cur, best, bytes;
};
__host__ __device__ inline ScratchLayout scratch_layout(int n_atoms, int n_torsions, int n_pairs, int apl) {
  (void)n_pairs;
  (void)apl;
  ScratchLayout l;
  const int D = 6 + n_torsions;
  l.pre = 0;
  l.H = l.pre + align16i(32 * n_atoms);
  l.vec = l.H + align16i(4 * kHStride * D);
  l.x = l.vec + align16i(4 * (5 * kHStride + 24));
  l.cur = l.x + align16i(4 * kConfFloats);
  l.best = l.cur + align16i(4 * kConfFloats);
  l.bytes = l.best + align16i(4 * kConfFloats);
  return l;
}
__device__ __forceinline__ WarpScratch warp_scratch_at(uint8_t* base, const ScratchLayout& l) {
  WarpScratch W;
  W.pre = reinterpret_cast<float4*>(base + l.pre);
  W.H = reinterpret_cast<float*>(base + l.H);
  W.vec = reinterpret_cast<float*>(base + l.vec);
  W.x = reinterpret_cast<float*>(base + l.x);
  W.cur = reinterpret_cast<float*>(base + l.cur);
  W.best = reinterpret_cast<float*>(base + l.best);
  return W;
}

// Body frames for a conformation: lane b < n_bodies returns body b's world
// rotation Q and origin O, composed from the local transforms by pointer
// jumping (ceil(log2(depth + 1)) rounds of shuffles).
__device__ __forceinline__ void body_frames(const LigView& L, const Conf& c, Quat& Q, float3& O) {
  const int lane = threadIdx.x & 31;
  const int nb = L.n_bodies;
  const bool child = lane > 0 && lane < nb;
  float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
  if (child) {
    const float4* rec = reinterpret_cast<const float4*>(L.body + lane);
    b0 = rec[0];  // off xyz, parent
    b1 = rec[1];  // axis xyz, torsion
  }
  const int tors = __float_as_int(b1.w);
  const float tb = __shfl_sync(kFull, c.th, child ? 6 + tors : 0);
  int ptr = -1;
  if (lane == 0) {
    Q = c.q;
    O = c.p;
  } else if (child) {
    const float s = sin_ftz(0.5f * tb), co = cos_ftz(0.5f * tb);  // |theta / 2| <= pi / 2: absolute error < 4e-7
    Q = Quat{co, s * b1.x, s * b1.y, s * b1.z};
    O = make_float3(b0.x, b0.y, b0.z);
    ptr = __float_as_int(b0.w);
  } else {
    Q = Quat{1.f, 0.f, 0.f, 0.f};
    O = make_float3(0.f, 0.f, 0.f);
  }
  for (int r = 0; r < L.rounds; ++r) {
    const int src = ptr >= 0 ? ptr : lane;
    const Quat Qp = shflq(Q, src);
    const float3 Op = shfl3(O, src);
    const int pp = __shfl_sync(kFull, ptr, src);
    if (ptr >= 0) {
      O = Op + qrot(Qp, O);
      Q = qmul(Qp, Q);
      ptr = pp;
    }
  }
}

// Score and gradient of one conformation (all lanes return the same E;
// lane j < 6 + T returns gradient component j, other lanes 0).  IU: how many
// step pairs of the one-atom-per-lane intra loop are unrolled.
template <int APL, int FMT, int IU = 2>
__device__ __forceinline__ float eval_conf(const MapView& M, const LigView& L, const LaneLig<APL>& R,
                                           const WarpScratch& W, const Conf& c, float& grad, uint32_t flags) {
  const int lane = threadIdx.x & 31;
  const int N = L.n_atoms, nb = L.n_bodies;
  Quat Q;
  float3 O;
  body_frames(L, c, Q, O);
  // ---- atom positions
  float3 pos[APL];
  int type[APL];
  int atom[APL];  // the slot's atom, -1 when empty
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    atom[s] = APL == 1 ? (lane < N ? lane : -1) : (int)L.lane_map[2 * lane + s];
    const int i = atom[s];
    const float4 a = L.atom[i >= 0 ? i : 0];
    const int packed = __float_as_int(a.w);
    type[s] = packed & 0xff;
    const int b = i >= 0 ? (packed >> 8) & 0xff : 0;
    const Quat Qb = shflq(Q, b);
    const float3 Ob = shfl3(O, b);
    pos[s] = Ob + qrot(Qb, make_float3(a.x, a.y, a.z));
  }
  float e_lane = 0.f;
  float3 g[APL];
#pragma unroll
  for (int s = 0; s < APL; ++s) g[s] = make_float3(0.f, 0.f, 0.f);
  // ---- intra: the pair steps of the blob, two per pass (packed FP32x2 pair
  //      terms).  In a step each lane computes at most one pair -- its active atom
  //      against the passive atom of a partner lane, fetched by shuffle -- and takes
  //      the reaction force of at most one pair back from the lane that computed it.
  if (flags & DSDP_TERM_INTRA) {
    float2 e_pair = make_float2(0.f, 0.f);
    const uint2* tab = L.steps + lane;
    if (APL == 1) {
      // packed accumulators: component .x collects the even steps, .y the odd ones
      const float2 px = splat2(pos[0].x), py = splat2(pos[0].y), pz = splat2(pos[0].z);
      float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
      // unrolled (IU = 2): the shuffles of one step pair overlap the arithmetic of
      // the next; four measured slower, and the kernel that holds both tiles
      // (more live registers) runs faster without unrolling
#pragma unroll IU
      for (int st = 0; st < L.n_steps; st += 2) {
        const uint2 t0 = tab[st * 32], t1 = tab[st * 32 + 32];
        // shfl.idx reads the source lane from bits 0-4 only: the entry's partner field
        const float3 b0 = shfl3(pos[0], (int)t0.x), b1 = shfl3(pos[0], (int)t1.x);
        const float2 dx = __ffma2_rn(make_float2(b0.x, b1.x), splat2(-1.f), px);
        const float2 dy = __ffma2_rn(make_float2(b0.y, b1.y), splat2(-1.f), py);
        const float2 dz = __ffma2_rn(make_float2(b0.z, b1.z), splat2(-1.f), pz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const uint32_t both = t0.x | t1.x;  // bits 14 / 15: warp-uniform
        float2 e, sp;
        vina_pair_x2(r2, make_float2(__uint_as_float(t0.y), __uint_as_float(t1.y)), t0.x >> 12, t1.x >> 12,
                     (both >> 14) & 1, (both >> 15) & 1, e, sp);
        e_pair = __fadd2_rn(e_pair, e);
        const float2 fx = __fmul2_rn(sp, dx), fy = __fmul2_rn(sp, dy), fz = __fmul2_rn(sp, dz);
        // reaction forces of the pairs this lane is passive in (source lane: bits 5-9)
        const float3 c0 = shfl3(make_float3(fx.x, fy.x, fz.x), (int)(t0.x >> 5));
        const float3 c1 = shfl3(make_float3(fx.y, fy.y, fz.y), (int)(t1.x >> 5));
        ax = __ffma2_rn(make_float2(c0.x, c1.x), splat2(-1.f), __fadd2_rn(ax, fx));
        ay = __ffma2_rn(make_float2(c0.y, c1.y), splat2(-1.f), __fadd2_rn(ay, fy));
        az = __ffma2_rn(make_float2(c0.z, c1.z), splat2(-1.f), __fadd2_rn(az, fz));
      }
      g[0].x += ax.x + ax.y;
      g[0].y += ay.x + ay.y;
      g[0].z += az.x + az.y;
    } else {
#pragma unroll 1
      for (int st = 0; st < L.n_steps; st += 2) {
        const uint2 t0 = tab[st * 32], t1 = tab[st * 32 + 32];
        const bool ac0 = t0.x & (1u << 10), ac1 = t1.x & (1u << 10);
        const bool pc0 = t0.x & (1u << 11), pc1 = t1.x & (1u << 11);
        const float3 a0 = ac0 ? pos[APL - 1] : pos[0], a1 = ac1 ? pos[APL - 1] : pos[0];
        const float3 s0 = pc0 ? pos[APL - 1] : pos[0], s1 = pc1 ? pos[APL - 1] : pos[0];
        const float3 b0 = shfl3(s0, (int)t0.x), b1 = shfl3(s1, (int)t1.x);
        const float2 dx = make_float2(a0.x - b0.x, a1.x - b1.x);
        const float2 dy = make_float2(a0.y - b0.y, a1.y - b1.y);
        const float2 dz = make_float2(a0.z - b0.z, a1.z - b1.z);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const uint32_t both = t0.x | t1.x;
        float2 e, sp;
        vina_pair_x2(r2, make_float2(__uint_as_float(t0.y), __uint_as_float(t1.y)), t0.x >> 12, t1.x >> 12,
                     (both >> 14) & 1, (both >> 15) & 1, e, sp);
        e_pair = __fadd2_rn(e_pair, e);
        const float2 fx = __fmul2_rn(sp, dx), fy = __fmul2_rn(sp, dy), fz = __fmul2_rn(sp, dz);
        const float3 c0 = shfl3(make_float3(fx.x, fy.x, fz.x), (int)(t0.x >> 5));
        const float3 c1 = shfl3(make_float3(fx.y, fy.y, fz.y), (int)(t1.x >> 5));
        // each force goes to the slot its bit names (per-lane predication, no selects)
        if (ac0) g[APL - 1].x += fx.x, g[APL - 1].y += fy.x, g[APL - 1].z += fz.x;
        else g[0].x += fx.x, g[0].y += fy.x, g[0].z += fz.x;
        if (ac1) g[APL - 1].x += fx.y, g[APL - 1].y += fy.y, g[APL - 1].z += fz.y;
        else g[0].x += fx.y, g[0].y += fy.y, g[0].z += fz.y;
        if (pc0) g[APL - 1].x -= c0.x, g[APL - 1].y -= c0.y, g[APL - 1].z -= c0.z;
        else g[0].x -= c0.x, g[0].y -= c0.y, g[0].z -= c0.z;
        if (pc1) g[APL - 1].x -= c1.x, g[APL - 1].y -= c1.y, g[APL - 1].z -= c1.z;
        else g[0].x -= c1.x, g[0].y -= c1.y, g[0].z -= c1.z;
      }
    }
    e_lane += e_pair.x + e_pair.y;
  }
  // ---- inter: trilinear score and gradient (Eq. 2, Eq. 4 / Eq. 3)
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    if ((flags & DSDP_TERM_INTER) && atom[s] >= 0) {
      float3 gi;
      // the cell is located here, where it is used: holding it across the intra
      // block miscompiled the two-atoms-per-lane kernels (gradient x channel lost)
      e_lane += map_interp<FMT>(M, type[s], map_cell(M, pos[s]), gi);
      g[s] = g[s] + gi;
    }
  }
  const float E = warp_sum(e_lane);
  // ---- back-propagation: inclusive prefix sums over atoms (depth-first
  //      order) of (g_i, (r_i - p) x g_i); a subtree is a contiguous range.
  //      With two atoms per lane the lane map is not in atom order: each slot
  //      first parks its raw terms at its atom's place, and lane l then scans
  //      atoms 2l and 2l + 1 of the atom order.
  if (APL == 2) {
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      if (atom[s] < 0) continue;
      const float3 t = cross3(pos[s] - c.p, g[s]);
      W.pre[2 * atom[s]] = make_float4(g[s].x, g[s].y, g[s].z, t.x);
      W.pre[2 * atom[s] + 1] = make_float4(t.y, t.z, 0.f, 0.f);
    }
    __syncwarp();
  }
  float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float raw[APL][6];
#pragma unroll
  for (int s = 0; s < APL; ++s) {
    const int i = lane * APL + s;  // atom order
#pragma unroll
    for (int k = 0; k < 6; ++k) raw[s][k] = 0.f;
    if (i >= N) continue;
    if (APL == 1) {
      const float3 t = cross3(pos[s] - c.p, g[s]);
      raw[s][0] = g[s].x, raw[s][1] = g[s].y, raw[s][2] = g[s].z;
      raw[s][3] = t.x, raw[s][4] = t.y, raw[s][5] = t.z;
    } else {
      const float4 h0 = W.pre[2 * i], h1 = W.pre[2 * i + 1];
      raw[s][0] = h0.x, raw[s][1] = h0.y, raw[s][2] = h0.z;
      raw[s][3] = h0.w, raw[s][4] = h1.x, raw[s][5] = h1.y;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] += raw[s][k];
  }
  float inc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) inc[k] = v[k];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float t = __shfl_up_sync(kFull, inc[k], o);
      if (lane >= o) inc[k] += t;
    }
  }
  if (APL == 2) __syncwarp();  // every raw value read before the prefix overwrites it
  {
    // this lane's atoms (atom order): exclusive prefix of the lane plus its own slots
    float run[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) run[k] = inc[k] - v[k];
#pragma unroll
    for (int s = 0; s < APL; ++s) {
      const int i = lane * APL + s;
      if (i >= N) continue;
#pragma unroll
      for (int k = 0; k < 6; ++k) run[k] += raw[s][k];
      W.pre[2 * i] = make_float4(run[0], run[1], run[2], run[3]);
      W.pre[2 * i + 1] = make_float4(run[4], run[5], 0.f, 0.f);
    }
  }
  __syncwarp();
  float tor = 0.f;
  if (lane > 0 && lane < nb) {
    const float4* rec = reinterpret_cast<const float4*>(L.body + lane);
    const float4 b1 = rec[1];
    const int4 b2 = *reinterpret_cast<const int4*>(rec + 2);  // atom_begin, atom_end, depth, pad
    const float4 h0 = W.pre[2 * (b2.y - 1)], h1 = W.pre[2 * (b2.y - 1) + 1];
    const float4 l0 = W.pre[2 * (b2.x - 1)], l1 = W.pre[2 * (b2.x - 1) + 1];
    const float3 G = make_float3(h0.x - l0.x, h0.y - l0.y, h0.z - l0.z);
    const float3 C = make_float3(h0.w - l0.w, h1.x - l1.x, h1.y - l1.y);
    const float3 axis = qrot(Q, make_float3(b1.x, b1.y, b1.z));
    tor = dot3(axis, C - cross3(O - c.p, G));
  }
  const float tv = __shfl_sync(kFull, tor, R.tbody);
  float gl = 0.f;
  if (lane < 6) {
    const float* tot = reinterpret_cast<const float*>(W.pre + 2 * (N - 1));
    gl = tot[lane];
  } else if (lane < 6 + L.T) {
    gl = tv;
  }
  __syncwarp();  // W.pre is rewritten by the next evaluation
  grad = gl;
  return E;
}

// c (+) s for a step held in lane layout.
__device__ __forceinline__ Conf apply_step(const Conf& c, float s, int T) {
  const int lane = threadIdx.x & 31;
  Conf o;
  o.p = make_float3(c.p.x + __shfl_sync(kFull, s, 0), c.p.y + __shfl_sync(kFull, s, 1),
                    c.p.z + __shfl_sync(kFull, s, 2));
  const Quat dq = quat_from_rotvec(__shfl_sync(kFull, s, 3), __shfl_sync(kFull, s, 4), __shfl_sync(kFull, s, 5));
  o.q = qnormalize(qmul(dq, c.q));
  o.th = (lane >= 6 && lane < 6 + T) ? wrap_angle(c.th + s) : c.th;
  return o;
}

// Four warp sums at once, every lane getting all four.  Transposed butterfly:
// the first two exchanges halve the values each lane carries (lanes with bit 4
// clear keep a, b, the others c, d; then bit 3 picks one of the two), the last
// three sum one value over a group of 8 lanes, and lanes 0, 8, 16, 24 hold a, b,
// c, d: 10 shuffles and 6 adds instead of 20 and 20.
__device__ __forceinline__ void warp_sum4(float& a, float& b, float& c, float& d) {
  const int lane = threadIdx.x & 31;
  const bool hi16 = lane & 16, hi8 = lane & 8;
  float k0 = hi16 ? c : a, k1 = hi16 ? d : b;
  const float s0 = hi16 ? a : c, s1 = hi16 ? b : d;
  k0 += __shfl_xor_sync(kFull, s0, 16);
  k1 += __shfl_xor_sync(kFull, s1, 16);
  float k = hi8 ? k1 : k0;
  k += __shfl_xor_sync(kFull, hi8 ? k0 : k1, 8);
  k += __shfl_xor_sync(kFull, k, 4);
  k += __shfl_xor_sync(kFull, k, 2);
  k += __shfl_xor_sync(kFull, k, 1);
  a = __shfl_sync(kFull, k, 0);
  b = __shfl_sync(kFull, k, 8);
  c = __shfl_sync(kFull, k, 16);
  d = __shfl_sync(kFull, k, 24);
}

// BFGS inverse-Hessian step after an accepted line search (Nocedal & Wright
// Eq. 6.17), lane j holding row j of H and component j of the vectors.  With
// d = -H g and y = g' - g, H y = H g' + d, so one product H g' gives both the
// update and the next direction:
//   H' g' = H g' - rho (s (Hy.g') + Hy (s.g')) + (rho^2 y.Hy + rho) s (s.g').
// H is updated in place as H_jk += s_j u_k - rho Hy_j s_k, u = (rho^2 y.Hy + rho) s
// - rho Hy.  Returns the new direction -H' g' (0 beyond D).
__device__ __forceinline__ float bfgs_update(const WarpScratch& W, int D, float s, float y, float gn, float d) {
  const int lane = threadIdx.x & 31;
  const int D4 = (D + 3) & ~3;
  float* vg = W.vec;
  float* vs = W.vec + kHStride;
  float* vu = W.vec + 2 * kHStride;
  const float4* Hrow = reinterpret_cast<const float4*>(W.H + kHStride * (lane < D ? lane : 0));
  if (lane < D4) vg[lane] = lane < D ? gn : 0.f;
  __syncwarp();
  float hg = 0.f;  // (H g')_lane: four independent partial sums
  if (lane < D) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < D4; k += 4) {
      const float4 h = Hrow[k >> 2], v = *reinterpret_cast<const float4*>(vg + k);
      acc.x = fmaf(h.x, v.x, acc.x);
      acc.y = fmaf(h.y, v.y, acc.y);
      acc.z = fmaf(h.z, v.z, acc.z);
      acc.w = fmaf(h.w, v.w, acc.w);
    }
    hg = (acc.x + acc.y) + (acc.z + acc.w);
  }
  const float hy = lane < D ? hg + d : 0.f;
  float sy = s * y, yhy = y * hy, hyg = hy * gn, sg = s * gn;
  warp_sum4(sy, yhy, hyg, sg);
  float dn;
  if (sy > kMinCurvature) {
    const float rho = 1.f / sy;
    const float coef = rho * rho * yhy + rho;
    if (lane < D4) {
      vs[lane] = lane < D ? s : 0.f;
      vu[lane] = lane < D ? coef * s - rho * hy : 0.f;
    }
    __syncwarp();
    if (lane < D) {
      float4* Hw = reinterpret_cast<float4*>(W.H + kHStride * lane);
      const float a = -rho * hy;
      for (int k = 0; k < D4; k += 4) {
        float4 h = Hw[k >> 2];
        const float4 u = *reinterpret_cast<const float4*>(vu + k), v = *reinterpret_cast<const float4*>(vs + k);
        h.x = fmaf(s, u.x, fmaf(a, v.x, h.x));
        h.y = fmaf(s, u.y, fmaf(a, v.y, h.y));
        h.z = fmaf(s, u.z, fmaf(a, v.z, h.z));
        h.w = fmaf(s, u.w, fmaf(a, v.w, h.w));
        Hw[k >> 2] = h;
      }
    }
    dn = -(hg - rho * (s * hyg + hy * sg) + coef * s * sg);
  } else {
    dn = -hg;
  }
  __syncwarp();  // vec is rewritten by the next update
  return lane < D ? dn : 0.f;
}

// H = I (rows 0..D-1, columns up to D rounded to float4).
__device__ __forceinline__ void bfgs_reset(const WarpScratch& W, int D) {
  const int lane = threadIdx.x & 31;
  const int D4 = (D + 3) & ~3;
  if (lane < D) {
    float4* Hw = reinterpret_cast<float4*>(W.H + kHStride * lane);
    for (int k = 0; k < D4; k += 4)
      Hw[k >> 2] = make_float4(k == lane ? 1.f : 0.f, k + 1 == lane ? 1.f : 0.f, k + 2 == lane ? 1.f : 0.f,
                               k + 3 == lane ? 1.f : 0.f);
  }
}

// Write conf (7 + T floats) from lane layout: lanes 0..2 p, 3..6 q, 7 + k theta_k.
__device__ __forceinline__ void store_conf(float* out, const Conf& c, int T) {
  const int lane = threadIdx.x & 31;
  const float th = __shfl_sync(kFull, c.th, lane >= 7 ? lane - 1 : 0);
  if (lane < 7 + T) {
    float v;
    if (lane == 0) v = c.p.x;
    else if (lane == 1) v = c.p.y;
    else if (lane == 2) v = c.p.z;
    else if (lane == 3) v = c.q.w;
    else if (lane == 4) v = c.q.x;
    else if (lane == 5) v = c.q.y;
    else if (lane == 6) v = c.q.z;
    else v = th;
    out[lane] = v;
  }
}

// Make the conformation written by store_conf visible to the whole warp, then read it.
__device__ __forceinline__ Conf load_conf(const float* in, int T) {
  const int lane = threadIdx.x & 31;
  Conf c;
  c.p = make_float3(in[0], in[1], in[2]);
  c.q = Quat{in[3], in[4], in[5], in[6]};
  c.th = (lane >= 6 && lane < 6 + T) ? in[lane + 1] : 0.f;
  return c;
}

// Adaptive search space (Sec. 2, third modification; Fig. 3): a start position
// uniform in the box intersected with the union of balls of radius R around the
// predicted binding-site points, by rejection.  Attempt 0 is the box draw p0
// (block 0 of step 0), attempt a >= 1 takes words 0-2 of block 64 + a; a
// candidate is accepted when some point lies within R of it.  The candidate
// (one fused multiply-add per axis) and the squared distances ((dx dx + dy dy)
// + dz dz, no contraction) are FP32 with a fixed operation order, so every
// device and the oracle take the same decisions; the lanes share the points.
// After 64 rejected attempts the start is the first point.
__device__ __forceinline__ float3 site_start(const DevJob& J, const ChainStream& rs, float3 p0) {
  const int lane = threadIdx.x & 31;
  for (int a = 0; a < 64; ++a) {
    float3 c = p0;
    if (a > 0) {
      const uint4 b = rs.block(0, 64u + (uint32_t)a);
      c = make_float3(__fmaf_rn(J.box_size[0], ChainStream::to_uniform(b.x), J.box_lo[0]),
                      __fmaf_rn(J.box_size[1], ChainStream::to_uniform(b.y), J.box_lo[1]),
                      __fmaf_rn(J.box_size[2], ChainStream::to_uniform(b.z), J.box_lo[2]));
    }
    bool inside = false;
    for (int k = lane; k < J.n_sites; k += 32) {
      const float dx = __fsub_rn(c.x, __ldg(J.sites + 3 * k)), dy = __fsub_rn(c.y, __ldg(J.sites + 3 * k + 1)),
                  dz = __fsub_rn(c.z, __ldg(J.sites + 3 * k + 2));
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      inside |= d2 <= J.site_r2;
    }
    if (__any_sync(kFull, inside)) return c;
  }
  return make_float3(__ldg(J.sites), __ldg(J.sites + 1), __ldg(J.sites + 2));
}

// Chain and optimiser variables that wait in shared memory while a
// conformation is evaluated (read back through volatile loads, so that none of
// them holds a register during the evaluation).
struct ChainVars {
  int phase, it, trial, step;
  float e, gd, alpha, e_opt_best;
  float e_cur, e_best;
  uint32_t evals;
  int T;
  int bb, max_iters, n_steps;
  float temperature;
  float inv_gyr;
  uint32_t seed_lo, seed_hi, chain;
  float* trace;
};
static_assert(sizeof(ChainVars) <= 4 * 24, "ChainVars must fit its 24 words of the vec area");

// One Monte Carlo chain (Sec. 2: one of many short independent copies; Vina's
// mutation and Metropolis rules) with its local optimisations -- BFGS with
// Armijo backtracking (Vina's optimiser; Nocedal & Wright Alg. 6.1) or
// Barzilai-Borwein (the paper's second modification, Sec. 2 / ref. 37: BB1 step
// s.s / s.y, clamped, no line search, best iterate returned).
//
// The whole chain is one loop around a single score + gradient evaluation: a
// small state machine decides, from each evaluation, the next conformation to
// evaluate.  Only the conformation under evaluation stays in registers across
// an evaluation; the optimiser's vectors g and d, the chain's scalars and the
// iterate / current / best conformations wait in shared memory.
template <int APL, int FMT, int IU = 2>
__device__ void run_chain(const DevJob& J, const LigView& L, const WarpScratch& W, int chain) {
  enum : int { kStart = 0, kTrial = 1, kBB = 2 };
  const int lane = threadIdx.x & 31;
  const MapView M = make_map_view(J);
  LaneLig<APL> R;
  load_lane_lig<APL>(L, R);
  volatile float* const Vg = W.vec + 3 * kHStride;  // g, component `lane` (lane < kHStride)
  volatile float* const Vd = W.vec + 4 * kHStride;  // search direction / step
  volatile ChainVars& V = *reinterpret_cast<volatile ChainVars*>(W.vec + 5 * kHStride);
  Conf xt;
  {
    const int T = L.T;
    const ChainStream rs{J.seed_lo, J.seed_hi, (uint32_t)chain};
    // initial conformation: uniform word n of step 0 is word n % 4 of block n / 4
    const uint4 b0 = rs.block(0, 0), b1 = rs.block(0, 1);
    xt.p = make_float3(__fmaf_rn(J.box_size[0], ChainStream::to_uniform(b0.x), J.box_lo[0]),
                       __fmaf_rn(J.box_size[1], ChainStream::to_uniform(b0.y), J.box_lo[1]),
                       __fmaf_rn(J.box_size[2], ChainStream::to_uniform(b0.z), J.box_lo[2]));
    if (J.n_sites > 0) xt.p = site_start(J, rs, xt.p);
    const float u1 = ChainStream::to_uniform(b0.w), u2 = ChainStream::to_uniform(b1.x),
                u3 = ChainStream::to_uniform(b1.y);
    float s2, c2, s3, c3;
    sincosf(kTwoPiF * u2, &s2, &c2);
    sincosf(kTwoPiF * u3, &s3, &c3);
    const float a = sqrtf(1.f - u1), b = sqrtf(u1);
    xt.q = Quat{b * c3, a * s2, a * c2, b * s3};
    float th = 0.f;
    if (lane >= 6 && lane < 6 + T) {
      const uint4 bk = rs.block(0, (uint32_t)(lane >> 2));
      th = kPiF - kTwoPiF * ChainStream::to_uniform(pick(bk, lane & 3));
    }
    xt.th = th;
    // every lane writes the same values
    V.phase = kStart;
    V.it = V.trial = V.step = 0;
    V.e = V.gd = V.e_opt_best = V.e_cur = V.e_best = 0.f;
    V.alpha = 1.f;
    V.evals = 0;
    V.T = T;
    V.bb = J.optimizer == DSDP_OPT_BB;
    V.max_iters = J.n_opt_iters;
    V.n_steps = J.n_steps;
    V.temperature = J.temperature;
    V.inv_gyr = 1.f / L.h->gyration_radius;
    V.seed_lo = J.seed_lo;
    V.seed_hi = J.seed_hi;
    V.chain = (uint32_t)chain;
    V.trace = J.trace ? J.trace + (size_t)chain * (J.n_steps + 1) * ((size_t)7 + T + 4) : nullptr;
    if (lane < kHStride) Vg[lane] = Vd[lane] = 0.f;
    if (J.trace && J.trace_starts) {  // row 0: the drawn start, before any optimisation
      float* t = J.trace + (size_t)chain * (J.n_steps + 1) * ((size_t)7 + T + 4);
      store_conf(t, xt, T);
      if (lane == 0) {
        t[7 + T + 0] = 0.f;
        t[7 + T + 1] = 0.f;
        t[7 + T + 2] = -2.f;
        t[7 + T + 3] = 0.f;
      }
    }
    __syncwarp();
  }
  for (;;) {
    float gn;
    const float en = eval_conf<APL, FMT, IU>(M, L, R, W, xt, gn, DSDP_TERM_ALL);
    const int T = V.T, nx = 7 + T, D = 6 + T;
    const bool bb = V.bb;
    const int max_iters = V.max_iters;
    int phase = V.phase, it = V.it, trial = V.trial;
    float e = V.e, gd = V.gd, alpha = V.alpha, e_opt_best = V.e_opt_best;
    float g = lane < kHStride ? Vg[lane] : 0.f, dir = lane < kHStride ? Vd[lane] : 0.f;
    const uint32_t evals = V.evals + 1;
    bool done = false;
    if (phase == kStart) {  // first evaluation of a local optimisation
      e = en;
      g = gn;
      store_conf(W.x, xt, T);
      if (max_iters == 0) {
        done = true;
      } else if (!bb) {
        bfgs_reset(W, D);
        dir = -g;  // H0 = I
        gd = -warp_sum(g * g);
        it = trial = 0;
        alpha = 1.f;
        xt = apply_step(xt, dir, T);
        phase = kTrial;
      } else {
        e_opt_best = e;
        alpha = kBBAlpha0;
        it = 0;
        dir = -alpha * g;
        xt = apply_step(xt, dir, T);
        phase = kBB;
      }
    } else if (phase == kTrial) {  // BFGS: Armijo test of the trial point x + alpha d
      if (en <= e + kArmijoC1 * alpha * gd) {
        const float s = alpha * dir, y = gn - g;
        g = gn;
        e = en;
        store_conf(W.x, xt, T);
        if (++it == max_iters) {
          done = true;
        } else {
          dir = bfgs_update(W, D, s, y, gn, dir);
          gd = warp_sum(g * dir);  // computed directly: the sufficient-decrease test must see the true slope
          alpha = 1.f;
          trial = 0;
          xt = apply_step(xt, dir, T);
        }
      } else {
        alpha *= kShrink;
        if (++trial == kMaxTrials) {
          done = true;  // no acceptable step: the optimisation ends at the current iterate
        } else {
          __syncwarp();
          xt = apply_step(load_conf(W.x, T), alpha * dir, T);
        }
      }
    } else {  // BB: x_{k+1} = x_k + s_k evaluated; next step length from s.s / s.y
      const float sy = warp_sum(dir * (gn - g));
      const float ss = warp_sum(dir * dir);
      alpha = sy > 0.f ? fminf(fmaxf(ss / sy, kBBAlphaMin), kBBAlphaMax) : kBBAlphaMax;
      g = gn;
      if (en < e_opt_best) {
        e_opt_best = en;
        store_conf(W.x, xt, T);
      }
      if (++it == max_iters) {
        done = true;
      } else {
        dir = -alpha * g;
        xt = apply_step(xt, dir, T);
      }
    }
    if (done) {
      // ---- local optimisation finished: its result is W.x with energy eo
      const float eo = (bb && max_iters > 0) ? e_opt_best : e;
      const ChainStream rs{V.seed_lo, V.seed_hi, V.chain};
      float* const trace = V.trace;
      const size_t trace_stride = (size_t)nx + 4;
      int step = V.step;
      float e_cur = V.e_cur, e_best = V.e_best;
      __syncwarp();
      if (step == 0) {
        e_cur = e_best = eo;
        if (lane < nx) {
          W.cur[lane] = W.x[lane];
          W.best[lane] = W.x[lane];
        }
        if (trace && !J.trace_starts) {
          if (lane < nx) trace[lane] = W.x[lane];
          if (lane == 0) {
            trace[nx + 0] = e_cur;
            trace[nx + 1] = e_cur;
            trace[nx + 2] = -1.f;
            trace[nx + 3] = 1.f;
          }
        }
      } else {
        const uint4 w0 = rs.block((uint32_t)step, 0);
        const int mode = (int)(((unsigned long long)(w0.x >> 8) * (unsigned long long)(2 + T)) >> 24);
        const float u = ChainStream::to_uniform(w0.y);
        const bool accept = (eo < e_cur) || (u < expf(-(eo - e_cur) / V.temperature));
        if (accept) {
          e_cur = eo;
          if (lane < nx) W.cur[lane] = W.x[lane];
          if (eo < e_best) {
            e_best = eo;
            if (lane < nx) W.best[lane] = W.x[lane];
          }
        }
        if (trace) {
          float* t = trace + (size_t)step * trace_stride;
          if (lane < nx) t[lane] = W.cur[lane];
          if (lane == 0) {
            t[nx + 0] = eo;
            t[nx + 1] = e_cur;
            t[nx + 2] = (float)mode;
            t[nx + 3] = accept ? 1.f : 0.f;
          }
        }
      }
      __syncwarp();
      if (++step > V.n_steps) {
        if (lane < nx) J.chain_best_conf[(size_t)chain * nx + lane] = W.best[lane];
        if (lane == 0) {
          J.chain_best_e[chain] = e_best;
          J.chain_evals[chain] = evals;
        }
        __syncwarp();
        return;
      }
      // ---- mutation of the current conformation (the next local optimisation's start)
      const uint4 w0 = rs.block((uint32_t)step, 0);
      const int mode = (int)(((unsigned long long)(w0.x >> 8) * (unsigned long long)(2 + T)) >> 24);
      xt = load_conf(W.cur, T);
      if (mode == 0) {
        const float3 b = unit_ball(rs, (uint32_t)step);
        xt.p = xt.p + kMutationAmplitude * b;
      } else if (mode == 1) {
        const float3 b = unit_ball(rs, (uint32_t)step);
        const float k = kMutationAmplitude * V.inv_gyr;
        xt.q = qnormalize(qmul(quat_from_rotvec(k * b.x, k * b.y, k * b.z), xt.q));
      } else if (lane == 6 + (mode - 2)) {
        xt.th = kPiF - kTwoPiF * ChainStream::to_uniform(w0.z);
      }
      phase = kStart;
      V.step = step;
      V.e_cur = e_cur;
      V.e_best = e_best;
    }
    V.phase = phase;
    V.it = it;
    V.trial = trial;
    V.e = e;
    V.gd = gd;
    V.alpha = alpha;
    V.e_opt_best = e_opt_best;
    V.evals = evals;
    if (lane < kHStride) {
      Vg[lane] = g;
      Vd[lane] = dir;
    }
    __syncwarp();
  }
}

}  // namespace dsdp
