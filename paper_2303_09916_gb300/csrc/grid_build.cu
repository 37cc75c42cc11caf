// Receptor grid maps (Sec. 2 first modification; Appendix Eq. 1 and Eq. 4)
// and the gather microbenchmark that bounds the score path.
//
// A CTA owns a brick of 8 x 8 x 4 vertices.  It streams the receptor atoms in
// index order, keeps those within the cutoff of the brick's bounding box
// (ballot compaction into shared memory, order preserved, so the sums are
// deterministic), then every thread sums the pair score and its gradient
// for all 8 ligand types at its vertex.  The 8 types share 4 atomic radii:
// the gauss / repulsion terms are summed once per radius (packed FP32x2, two
// radii per operation), and the hydrophobic and H-bond terms, which only some
// receptor atoms carry and only at short range, in five sums of their own;
// each type's map is its radius sum plus its own term at the end.
#include "launch.h"

namespace dsdp {
namespace {

constexpr int kBX = 8, kBY = 8, kBZ = 4, kThreads = kBX * kBY * kBZ;
constexpr int kChunk = 1536;

// hydrophobic term of surface distance d (1 below 0.5, linear to 0 at 1.5),
// added to e and de/dd
__device__ __forceinline__ void hydrophobic(float d, float& e, float& de) {
  if (d < 0.5f) {
    e += kWHydrophobic;
  } else if (d < 1.5f) {
    e += kWHydrophobic * (1.5f - d);
    de -= kWHydrophobic;
  }
}
// H-bond term (1 below -0.7, linear to 0 at 0)
__device__ __forceinline__ void hbond(float d, float& e, float& de) {
  if (d < -0.7f) {
    e += kWHBond;
  } else if (d < 0.f) {
    e += kWHBond * (-d * (1.0f / 0.7f));
    de -= kWHBond * (1.0f / 0.7f);
  }
}

// a (e, de/dd) pair term projected on the unit vector u, added to (E, G)
__device__ __forceinline__ void add_term(float4& acc, float e, float de, float ux, float uy, float uz) {
  acc.x += e;
  acc.y = fmaf(de, ux, acc.y);
  acc.z = fmaf(de, uy, acc.z);
  acc.w = fmaf(de, uz, acc.w);
}

template <int FMT>
__device__ __forceinline__ void store_node(void* maps, size_t idx, float e, float gx, float gy, float gz) {
  if (FMT == 0) {
    reinterpret_cast<float4*>(maps)[idx] = make_float4(e, gx, gy, gz);
  } else if (FMT == 1) {
    __nv_bfloat162 a = __floats2bfloat162_rn(e, gx), b = __floats2bfloat162_rn(gy, gz);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&a);
    raw.y = *reinterpret_cast<uint32_t*>(&b);
    reinterpret_cast<uint2*>(maps)[idx] = raw;
  } else if (FMT == 2) {
    __half2 a = __floats2half2_rn(e, gx), b = __floats2half2_rn(gy, gz);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&a);
    raw.y = *reinterpret_cast<uint32_t*>(&b);
    reinterpret_cast<uint2*>(maps)[idx] = raw;
  } else if (FMT == 3) {
    reinterpret_cast<float*>(maps)[idx] = e;
  } else if (FMT == 4) {
    reinterpret_cast<unsigned short*>(maps)[idx] = __bfloat16_as_ushort(__float2bfloat16_rn(e));
  } else {
    reinterpret_cast<unsigned short*>(maps)[idx] = __half_as_ushort(__float2half_rn(e));
  }
}

template <int FMT>
__global__ void __launch_bounds__(kThreads) grid_build_kernel(int n_rec, const float* __restrict__ xyz,
                                                              const uint8_t* __restrict__ type, int nx, int ny,
                                                              int nz, float ox, float oy, float oz, float h,
                                                              void* __restrict__ maps) {
  __shared__ float4 s_atom[kChunk];
  __shared__ int s_count[kThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bx0 = blockIdx.x * kBX, by0 = blockIdx.y * kBY, bz0 = blockIdx.z * kBZ;
  const int ix = bx0 + (tid & 7), iy = by0 + ((tid >> 3) & 7), iz = bz0 + (tid >> 6);
  const bool active = ix < nx && iy < ny && iz < nz;
  const float mx = ox + h * (float)ix, my = oy + h * (float)iy, mz = oz + h * (float)iz;
  const float lox = ox + h * (float)bx0, loy = oy + h * (float)by0, loz = oz + h * (float)bz0;
  const float hix = ox + h * (float)min(bx0 + kBX - 1, nx - 1), hiy = oy + h * (float)min(by0 + kBY - 1, ny - 1),
              hiz = oz + h * (float)min(bz0 + kBZ - 1, nz - 1);
  const float reach2 = (kCutoff + 0.01f) * (kCutoff + 0.01f);
  // gauss / repulsion sums per radius, packed (1.9, 1.8) and (1.7, 2.0): energy and gradient
  float2 Ea = make_float2(0.f, 0.f), Eb = Ea, Xa = Ea, Xb = Ea, Ya = Ea, Yb = Ea, Za = Ea, Zb = Ea;
  // hydrophobic term of C_H; H-bond terms of N_D (with receptor acceptors), N_A
  // and O_A (with receptor donors), O_DA (with donors or acceptors): (e, gx, gy, gz)
  float4 Hch = make_float4(0.f, 0.f, 0.f, 0.f), Hnd = Hch, Hna = Hch, Hoa = Hch, Hoda = Hch;
  int base = 0;
  while (base < n_rec) {
    int count = 0;
    while (base < n_rec && count <= kChunk - kThreads) {
      const int j = base + tid;
      bool keep = false;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < n_rec) {
        a.x = __ldg(xyz + 3 * j);
        a.y = __ldg(xyz + 3 * j + 1);
        a.z = __ldg(xyz + 3 * j + 2);
        a.w = __int_as_float((int)__ldg(type + j));
        const float dx = fmaxf(fmaxf(lox - a.x, a.x - hix), 0.f);
        const float dy = fmaxf(fmaxf(loy - a.y, a.y - hiy), 0.f);
        const float dz = fmaxf(fmaxf(loz - a.z, a.z - hiz), 0.f);
        keep = dx * dx + dy * dy + dz * dz < reach2;
      }
      const unsigned bal = __ballot_sync(kFull, keep);
      if (lane == 0) s_count[warp] = __popc(bal);
      __syncthreads();
      int off = count, total = 0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        const int c = s_count[w];
        if (w < warp) off += c;
        total += c;
      }
      if (keep) s_atom[off + __popc(bal & ((1u << lane) - 1u))] = a;
      count += total;
      base += kThreads;
      __syncthreads();
    }
    if (active) {
      for (int k = 0; k < count; ++k) {
        const float4 a = s_atom[k];
        const float dx = mx - a.x, dy = my - a.y, dz = mz - a.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < kCutoff * kCutoff)) continue;
        // a vertex on an atom (r = 0) takes no gradient from it: ir is finite there and d* = 0
        const float ir = rsqrt_ftz(fmaxf(r2, 1e-30f));
        const float r = r2 * ir;
        const int tj = min(__float_as_int(a.w), 8);
        const float Rj = c_xs_radius[tj];
        const int bj = c_xs_bits[tj];  // the same for every thread: the branches below do not diverge on it
        const float2 sa = make_float2(r - (1.9f + Rj), r - (1.8f + Rj));
        const float2 sb = make_float2(r - (1.7f + Rj), r - (2.0f + Rj));
        float2 ea, da, eb, db;
        steric_x2(sa, ea, da);
        steric_x2(sb, eb, db);
        const float ux = dx * ir, uy = dy * ir, uz = dz * ir;
        Ea = __fadd2_rn(Ea, ea);
        Eb = __fadd2_rn(Eb, eb);
        Xa = __ffma2_rn(da, splat2(ux), Xa);
        Xb = __ffma2_rn(db, splat2(ux), Xb);
        Ya = __ffma2_rn(da, splat2(uy), Ya);
        Yb = __ffma2_rn(db, splat2(uy), Yb);
        Za = __ffma2_rn(da, splat2(uz), Za);
        Zb = __ffma2_rn(db, splat2(uz), Zb);
        if ((bj & 1) && sa.x < 1.5f) {  // hydrophobic receptor atom: C_H (radius 1.9)
          float e = 0.f, de = 0.f;
          hydrophobic(sa.x, e, de);
          add_term(Hch, e, de, ux, uy, uz);
        }
        if ((bj & 6) && sa.y < 0.f) {  // donor and/or acceptor within H-bond range (d of radius 1.8 < 0)
          if (bj & 4) {  // receptor acceptor: N_D (1.8)
            float e = 0.f, de = 0.f;
            hbond(sa.y, e, de);
            add_term(Hnd, e, de, ux, uy, uz);
          }
          if (bj & 2) {  // receptor donor: N_A (1.8), O_A (1.7)
            float e = 0.f, de = 0.f;
            hbond(sa.y, e, de);
            add_term(Hna, e, de, ux, uy, uz);
            e = de = 0.f;
            hbond(sb.x, e, de);
            add_term(Hoa, e, de, ux, uy, uz);
          }
          float e = 0.f, de = 0.f;  // O_DA (1.7) with either
          hbond(sb.x, e, de);
          add_term(Hoda, e, de, ux, uy, uz);
        }
      }
    }
    __syncthreads();
  }
  if (!active) return;
  const size_t nxyz = (size_t)nx * ny * nz;
  const size_t v = ((size_t)iz * ny + iy) * nx + ix;
  store_node<FMT>(maps, 0 * nxyz + v, Ea.x + Hch.x, Xa.x + Hch.y, Ya.x + Hch.z, Za.x + Hch.w);     // C_H
  store_node<FMT>(maps, 1 * nxyz + v, Ea.x, Xa.x, Ya.x, Za.x);                                     // C_P
  store_node<FMT>(maps, 2 * nxyz + v, Ea.y, Xa.y, Ya.y, Za.y);                                     // N_P
  store_node<FMT>(maps, 3 * nxyz + v, Ea.y + Hnd.x, Xa.y + Hnd.y, Ya.y + Hnd.z, Za.y + Hnd.w);     // N_D
  store_node<FMT>(maps, 4 * nxyz + v, Ea.y + Hna.x, Xa.y + Hna.y, Ya.y + Hna.z, Za.y + Hna.w);     // N_A
  store_node<FMT>(maps, 5 * nxyz + v, Eb.x + Hoa.x, Xb.x + Hoa.y, Yb.x + Hoa.z, Zb.x + Hoa.w);     // O_A
  store_node<FMT>(maps, 6 * nxyz + v, Eb.x + Hoda.x, Xb.x + Hoda.y, Yb.x + Hoda.z, Zb.x + Hoda.w); // O_DA
  store_node<FMT>(maps, 7 * nxyz + v, Eb.y, Xb.y, Yb.y, Zb.y);                                     // S_P
}

// 32-bit mixing hash (multiply-xorshift; the finaliser of MurmurHash3) for the
// microbenchmark's pseudo-random sample points.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// Each thread samples `repeats` points: the first is its input point, each later
// one an independent pseudo-random position in the grid (hash of the point
// index and the repeat) with a pseudo-random map type, so that consecutive
// samples share no cell and the corner reads are the random 8-corner gathers of
// the scoring path, with none of its arithmetic.
template <int FMT>
__global__ void __launch_bounds__(256) gather_bench_kernel(MapView M, const float* __restrict__ pts,
                                                           const uint8_t* __restrict__ types, int n, int repeats,
                                                           float* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  const float ex = (M.nx - 1) * M.h, ey = (M.ny - 1) * M.h, ez = (M.nz - 1) * M.h;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float3 p = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    int t = types[i];
    float acc = 0.f;
    for (int r = 0; r < repeats; ++r) {
      float3 g;
      const float e = sample_map<FMT>(M, t, p, g);
      acc += e + g.x + g.y + g.z;
      const uint32_t h0 = mix32((uint32_t)i * 0x9E3779B9u + (uint32_t)r + 1u);
      const uint32_t h1 = mix32(h0 ^ 0x68E31DA4u), h2 = mix32(h1 ^ 0xB5297A4Du);
      p = make_float3(M.ox + ex * ((h0 >> 8) * (1.f / 16777216.f)), M.oy + ey * ((h1 >> 8) * (1.f / 16777216.f)),
                      M.oz + ez * ((h2 >> 8) * (1.f / 16777216.f)));
      t = (int)(h2 & 7u);
    }
    out[i] = acc;
  }
}

template <int FMT>
cudaError_t launch_grid(const dsdp_receptor* rec, int nx, int ny, int nz, float ox, float oy, float oz, float h,
                        void* maps, cudaStream_t st) {
  const dim3 grid((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY, (nz + kBZ - 1) / kBZ);
  grid_build_kernel<FMT><<<grid, kThreads, 0, st>>>(rec->n, rec->xyz, rec->xs_type, nx, ny, nz, ox, oy, oz, h, maps);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t launch_gather(const MapView& M, const float* pts, const uint8_t* types, int n, int repeats, float* out,
                          cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = min((n + 255) / 256, sms * 8);
  gather_bench_kernel<FMT><<<blocks, 256, 0, st>>>(M, pts, types, n, repeats, out);
  return cudaGetLastError();
}

}  // namespace

void grid_geometry(const dsdp_box* box, int n[3], double origin[3]) {
  for (int a = 0; a < 3; ++a) {
    n[a] = (int)ceil(box->size[a] / box->spacing);
    origin[a] = box->center[a] - (n[a] - 1) * box->spacing / 2.0;
  }
}

dsdp_status validate_box(const dsdp_box* box) {
  if (!box) return set_error(DSDP_ERR_INVALID_ARG, "box is NULL");
  if (!(box->spacing > 0.0) || !isfinite(box->spacing))
    return set_error(DSDP_ERR_INVALID_ARG, "box spacing must be positive");
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(box->center[a]) || !isfinite(box->size[a]))
      return set_error(DSDP_ERR_INVALID_ARG, "box center/size not finite");
    if (!(box->size[a] > box->spacing))
      return set_error(DSDP_ERR_INVALID_ARG, "box size %g must exceed the spacing %g", box->size[a], box->spacing);
    if (box->size[a] / box->spacing > 4096.0) return set_error(DSDP_ERR_INVALID_ARG, "box has > 4096 vertices per axis");
  }
  int n[3];
  double o[3];
  grid_geometry(box, n, o);
  if ((double)DSDP_NUM_MAP_TYPES * n[0] * n[1] * n[2] >= 2147483648.0)
    return set_error(DSDP_ERR_INVALID_ARG, "grid of %d x %d x %d x 8 nodes exceeds 2^31 (32-bit map indices)", n[0],
                     n[1], n[2]);
  return DSDP_OK;
}

dsdp_status check_cuda(int err, const char* what) {
  if (err == cudaSuccess) return DSDP_OK;
  return set_error(DSDP_ERR_DEVICE, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
}

}  // namespace dsdp

using namespace dsdp;

extern "C" uint64_t dsdp_grid_map_bytes(const dsdp_box* box, dsdp_map_dtype dtype, dsdp_grid_mode mode) {
  if (validate_box(box) != DSDP_OK || (int)dtype < 0 || (int)dtype > 2 || (int)mode < 0 || (int)mode > 1) return 0;
  int n[3];
  double o[3];
  grid_geometry(box, n, o);
  const int fmt = map_fmt((int)dtype, (int)mode);
  return (uint64_t)DSDP_NUM_MAP_TYPES * n[0] * n[1] * n[2] * fmt_channels(fmt) * fmt_elem_bytes(fmt);
}

extern "C" dsdp_status dsdp_grid_build_device(const dsdp_receptor* rec, const dsdp_box* box, dsdp_map_dtype dtype,
                                              dsdp_grid_mode mode, void* d_maps, uint64_t maps_bytes,
                                              void* stream) {
  dsdp_status s = validate_box(box);
  if (s != DSDP_OK) return s;
  if (!rec || rec->n < 0 || (rec->n > 0 && (!rec->xyz || !rec->xs_type)))
    return set_error(DSDP_ERR_INVALID_ARG, "receptor arrays invalid");
  if ((int)dtype < 0 || (int)dtype > 2 || (int)mode < 0 || (int)mode > 1)
    return set_error(DSDP_ERR_INVALID_ARG, "bad map dtype/mode");
  const uint64_t need = dsdp_grid_map_bytes(box, dtype, mode);
  if (!d_maps || maps_bytes < need)
    return set_error(DSDP_ERR_INVALID_ARG, "maps buffer %llu bytes < %llu", (unsigned long long)maps_bytes,
                     (unsigned long long)need);
  int n[3];
  double o[3];
  grid_geometry(box, n, o);
  const float h = (float)box->spacing;
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (map_fmt((int)dtype, (int)mode)) {
    case 0: e = launch_grid<0>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
    case 1: e = launch_grid<1>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
    case 2: e = launch_grid<2>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
    case 3: e = launch_grid<3>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
    case 4: e = launch_grid<4>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
    default: e = launch_grid<5>(rec, n[0], n[1], n[2], (float)o[0], (float)o[1], (float)o[2], h, d_maps, st); break;
  }
  return check_cuda(e, "grid_build_kernel launch");
}

MapView dsdp::map_view_of(const dsdp_grid_view* g) {
  MapView M;
  M.maps = g->d_maps;
  M.nx = g->n[0];
  M.ny = g->n[1];
  M.nz = g->n[2];
  M.ox = (float)g->origin[0];
  M.oy = (float)g->origin[1];
  M.oz = (float)g->origin[2];
  M.h = (float)g->spacing;
  M.inv_h = (float)(1.0 / g->spacing);
  return M;
}

extern "C" dsdp_status dsdp_gather_bench_device(const dsdp_grid_view* grid, const float* d_points,
                                                const uint8_t* d_types, int32_t n_points, int32_t repeats,
                                                float* d_out, void* stream) {
  if (!grid || !grid->d_maps || !d_points || !d_types || !d_out || n_points <= 0 || repeats <= 0)
    return set_error(DSDP_ERR_INVALID_ARG, "gather bench arguments invalid");
  if (grid->n[0] < 2 || grid->n[1] < 2 || grid->n[2] < 2) return set_error(DSDP_ERR_INVALID_ARG, "grid too small");
  const MapView M = map_view_of(grid);
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  switch (map_fmt(grid->dtype, grid->mode)) {
    case 0: e = launch_gather<0>(M, d_points, d_types, n_points, repeats, d_out, st); break;
    case 1: e = launch_gather<1>(M, d_points, d_types, n_points, repeats, d_out, st); break;
    case 2: e = launch_gather<2>(M, d_points, d_types, n_points, repeats, d_out, st); break;
    case 3: e = launch_gather<3>(M, d_points, d_types, n_points, repeats, d_out, st); break;
    case 4: e = launch_gather<4>(M, d_points, d_types, n_points, repeats, d_out, st); break;
    default: e = launch_gather<5>(M, d_points, d_types, n_points, repeats, d_out, st); break;
  }
  return check_cuda(e, "gather_bench_kernel launch");
}
