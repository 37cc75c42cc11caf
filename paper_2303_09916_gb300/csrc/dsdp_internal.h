// Internal layouts shared by the host code and the kernels of libdsdp.
#pragma once
#include <stdint.h>

#include "../../include/dsdp.h"

namespace dsdp {

constexpr uint32_t kBlobMagic = 0x50445344u;  // "DSDP"
constexpr int kMaxAtoms = DSDP_MAX_LIGAND_ATOMS;
constexpr int kMaxBodies = DSDP_MAX_TORSIONS + 1;
constexpr int kMaxDim = 6 + DSDP_MAX_TORSIONS;  // gradient / step dimension
// Atoms per lane of a warp holding one conformation: up to 32 atoms internal
// atom i sits in lane i; above, each lane has two slots and the blob's lane map
// says which atom sits where.
__host__ __device__ constexpr int atoms_per_lane(int n_atoms) { return n_atoms <= 32 ? 1 : 2; }

// Intra-pair step table: the pairs are split into steps in which every lane
// computes at most one pair (its "active" atom against a partner lane's
// "passive" atom) and receives at most one reaction force.  One entry per lane
// per step (uint2):
//   x bits 0-4   partner lane (the passive atom's lane; own lane when inactive)
//        5-9    lane whose force this lane receives (the active atom's lane when
//               this lane is passive, otherwise a lane inactive in this step)
//        10     slot of the active atom in this lane, 11 slot of the passive atom
//        12, 13 the active pair carries the hydrophobic / H-bond term
//        14, 15 some pair of this step carries the hydrophobic / H-bond term
//               (the same in every lane of the step)
//   y    -(R_a + R_b) of the active pair as a float; kStepIdleNrs when inactive
constexpr float kStepIdleNrs = 1.0e4f;  // surface distance where every term and slope is zero

// Packed ligand (dsdp_ligand_pack).  Internal atom order: rigid bodies in
// depth-first pre-order from the root (children by torsion index), atoms of a
// body in ascending input index.  Every subtree is then one contiguous atom
// range, which the kernels use for the torsion gradients.
struct BlobHeader {
  uint32_t magic;
  uint32_t bytes;          // whole blob, multiple of 16
  int32_t n_atoms;
  int32_t n_torsions;
  int32_t n_bodies;
  int32_t n_pairs;
  int32_t rounds;          // pointer-jumping rounds: ceil(log2(max depth + 1))
  float gyration_radius;   // of the reference pose about the root origin atom
  float root_ref[3];       // input coordinates of the root origin atom
  int32_t root_user_atom;
  uint32_t off_atom;       // float4[n_atoms]: local xyz (reference frame, relative to the body origin);
                           //   w = int bits: map type | body << 8
  uint32_t off_atom_user;  // int32[n_atoms]: input index of internal atom i
  uint32_t off_body;       // BodyRec[n_bodies]
  uint32_t off_pairs;      // uint2[n_pairs] intra pair records (internal indices i < j):
                           //   x = 16 i | 16 j << 16, y = float -(R_i + R_j)  (after the staged prefix)
  uint32_t off_steps;      // uint2[n_steps][32] intra-pair step table (see kStepIdleNrs)
  int32_t n_steps;         // even
  uint32_t off_torsion_body;  // int32[n_torsions]: body driven by torsion k
  uint32_t off_atom64;     // double[n_atoms][3]: local xyz in FP64 (rescoring)
  uint32_t off_body64;     // double[n_bodies][6]: origin offset and unit axis in FP64 (rescoring)
  int32_t pair_hyd_begin;  // pairs [pair_hyd_begin, pair_hb_begin) carry the hydrophobic term,
  uint32_t stage_bytes;    // prefix the FP32 kernels stage into shared memory (the FP64 geometry follows it)
  int32_t pair_hb_begin;   //   pairs [pair_hb_begin, n_pairs) the H-bond term, the others neither
  uint32_t off_lane_map;   // int16[32][2]: internal atom in slot s of lane l (-1: empty); atom i in lane i
                           //   up to 32 atoms, a degree-balanced assignment above (see assign_lanes)
  uint32_t pad_[3];
};
static_assert(sizeof(BlobHeader) % 16 == 0, "blob header alignment");

struct BodyRec {
  float off[3];       // origin minus parent origin, reference frame
  int32_t parent;     // -1 for the root
  float axis[3];      // unit torsion axis (parent-side atom -> child-side atom), reference frame
  int32_t torsion;    // torsion index, -1 for the root
  int32_t atom_begin; // subtree atoms [atom_begin, atom_end)
  int32_t atom_end;
  int32_t depth;
  int32_t pad;
};
static_assert(sizeof(BodyRec) == 48, "body record size");

// One job as the kernels see it.
struct DevJob {
  const uint8_t* blob;
  const void* maps;
  int32_t n[3];
  float origin[3];
  float spacing;
  float inv_spacing;
  int32_t dtype;
  int32_t mode;
  int32_t n_chains;
  int32_t n_steps;
  int32_t n_opt_iters;
  int32_t optimizer;
  float temperature;
  uint32_t seed_lo, seed_hi;
  float box_lo[3];
  float box_size[3];
  const float* sites;  // adaptive search space: [n_sites][3] predicted binding-site points
  int32_t n_sites;     // 0: initial positions uniform in the box
  float site_r2;       // site radius squared (FP32)
  float* chain_best_conf;
  float* chain_best_e;
  uint32_t* chain_evals;
  float* trace;
  int32_t trace_starts;  // trace row 0: the initial conformation (not the state after the first optimisation)
  // rescoring
  int32_t n_rec;
  const float* rec_xyz;
  const uint8_t* rec_type;
  double* chain_score;   // scratch [n_chains]
  double* chain_inter;   // scratch [n_chains]
  double* chain_intra;   // scratch [n_chains]
  double* chain_coords;  // scratch [n_chains][n_atoms][3] (internal atom order)
  int32_t top_k;
  float rmsd_dedup;
  int32_t* out_n;
  int32_t* out_chain;
  double* out_score;
  double* out_inter;
  double* out_intra;
  double* out_conf;
  float* out_coords;
};

struct Tile {
  int32_t job;
  int32_t chain0;
  int32_t count;
  int32_t pad;
};

// Vina constants of the kernels (the scoring function DSDP keeps, Sec. 2).
constexpr float kWGauss1 = -0.0356f;
constexpr float kWGauss2 = -0.00516f;
constexpr float kWRepulsion = 0.840f;
constexpr float kWHydrophobic = -0.0351f;
constexpr float kWHBond = -0.587f;
constexpr double kWRot = 0.0585;
constexpr float kCutoff = 8.0f;
constexpr float kWallSlope = 10.0f;

// The same constants in double precision, for the FP64 rescoring.
constexpr double kWGauss1D = -0.0356;
constexpr double kWGauss2D = -0.00516;
constexpr double kWRepulsionD = 0.840;
constexpr double kWHydrophobicD = -0.0351;
constexpr double kWHBondD = -0.587;
constexpr double kCutoffD = 8.0;

// Optimiser constants (BFGS: Armijo backtracking; BB: BB1 step with clamps).
constexpr float kArmijoC1 = 1e-4f;
constexpr float kShrink = 0.5f;
constexpr int kMaxTrials = 10;
constexpr float kMinCurvature = 1e-10f;
constexpr float kBBAlpha0 = 1e-3f;
constexpr float kBBAlphaMin = 1e-4f;
constexpr float kBBAlphaMax = 0.1f;
constexpr float kMutationAmplitude = 2.0f;

}  // namespace dsdp

// Host-side helpers implemented in the library's .cpp / .cu files.
namespace dsdp {
dsdp_status set_error(dsdp_status s, const char* fmt, ...);
const char* last_error();
dsdp_status check_cuda(int err, const char* what);
void grid_geometry(const dsdp_box* box, int n[3], double origin[3]);
dsdp_status validate_box(const dsdp_box* box);
// dock parameters with the documented defaults filled in; INVALID_ARG if out of range
dsdp_status normalize_params(const dsdp_dock_params* in, dsdp_dock_params* out);
// context allocator (ctx may be NULL: plain cudaMalloc / cudaFree)
void* ctx_alloc(dsdp_ctx* ctx, size_t bytes, void* stream);
void ctx_free(dsdp_ctx* ctx, void* p, size_t bytes, void* stream);
int ctx_sm_count(dsdp_ctx* ctx);
}  // namespace dsdp
