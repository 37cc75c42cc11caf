// DSDP docking hot path -- FP64 CPU ORACLE.  TEST INFRASTRUCTURE ONLY.
//
// Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
// legs may load this library.  It shares no code with the CUDA path: its own
// constants, its own kinematics (3x3 matrices, not quaternions), its own tree
// builder, its own Philox.  Everything is written for a reader checking it
// against the method by eye: plain loops, FP64, no blocking or fusion.
//
// What it computes (section / equation of "DSDP: A Blind Docking Strategy
// Accelerated by GPUs", arXiv 2303.09916):
//   * Vina-form pair score (Sec. 2 "Binding pose search": DSDP keeps the
//     scoring function of AutoDock Vina, ref. 6; terms and constants are the
//     Vina reading listed in pair_term below -- not printed in the paper).
//   * Receptor grid maps holding, per vertex and ligand atom type, the summed
//     pair score and its gradient (Sec. 2 first modification; Appendix Eq. 1
//     and the gradient maps of Eq. 4).
//   * Trilinear interpolation of the score (Eq. 2) and of the gradient, either
//     as the derivative of the interpolant (Eq. 3) or by interpolating the
//     gradient maps (Eq. 4, DSDP's choice).
//   * Torsion-tree forward kinematics and the chain rule from atom gradients to
//     (position, orientation, torsion) gradients (Vina's search space, Sec. 2).
//   * BFGS with Armijo backtracking (Vina's optimiser, ref. 36) and
//     Barzilai-Borwein (DSDP's second modification, Sec. 2, ref. 37).
//   * Monte Carlo chains (Sec. 2, many short independent copies).
//   * Gridless FP64 rescoring, RMSD de-duplication and top-k (Fig. 4 postprocess).
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
//     generator both sides implement from its published definition.
//   * Receptor voxel features, the binding-site network's input (Sec. 2,
//     "Protein-ligand binding site prediction": 36^3 voxels over 70 A, 18
//     channels with S and Se merged and one surface channel), with surface
//     atoms by the Shrake-Rupley test.
//
// Parity status per function is stated in the header comment of each section.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Atom types (Vina "XS" types restricted to C/N/O/S heavy atoms).
// Ligand map types are indices 0..7; N_DA (8) occurs on receptor atoms only.
// ---------------------------------------------------------------------------
enum XsType { C_H = 0, C_P, N_P, N_D, N_A, O_A, O_DA, S_P, N_DA, NUM_XS };
const int kNumMapTypes = 8;

const double kXsRadius[NUM_XS] = {1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0, 1.8};
const bool kXsHydrophobic[NUM_XS] = {true, false, false, false, false, false, false, false, false};
const bool kXsDonor[NUM_XS] = {false, false, false, true, false, false, true, false, true};
const bool kXsAcceptor[NUM_XS] = {false, false, false, false, true, true, true, false, true};

// Vina weights (ref. 6; the paper adopts "the same scoring function", Sec. 2).
const double kWGauss1 = -0.0356;
const double kWGauss2 = -0.00516;
const double kWRepulsion = 0.840;
const double kWHydrophobic = -0.0351;
const double kWHBond = -0.587;
const double kWRot = 0.0585;       // torsion normalisation of the reported score
const double kCutoff = 8.0;        // pair cutoff, Angstrom
const double kWallSlope = 10.0;    // out-of-grid restraint, energy per Angstrom

// Pair score f(t_i, t_j, r) and df/dr.  Surface distance d = r - (R_i + R_j).
//   gauss1      exp(-(d/0.5)^2)
//   gauss2      exp(-((d-3)/2)^2)
//   repulsion   d^2 for d < 0
//   hydrophobic 1 for d < 0.5, 0 for d >= 1.5, linear between (both hydrophobic)
//   H-bond      1 for d < -0.7, 0 for d >= 0, linear between (donor/acceptor pair)
// Zero for r >= cutoff.  Parity: pinned by closed-form values in the tests.
void pair_term(int ti, int tj, double r, double cutoff, double* e, double* dedr) {
  *e = 0.0;
  *dedr = 0.0;
  if (!(r < cutoff)) return;
  const double d = r - (kXsRadius[ti] + kXsRadius[tj]);
  const double g1 = std::exp(-(d / 0.5) * (d / 0.5));
  const double g2 = std::exp(-((d - 3.0) / 2.0) * ((d - 3.0) / 2.0));
  double energy = kWGauss1 * g1 + kWGauss2 * g2;
  double slope = kWGauss1 * g1 * (-2.0 * d / 0.25) + kWGauss2 * g2 * (-2.0 * (d - 3.0) / 4.0);
  if (d < 0.0) {
    energy += kWRepulsion * d * d;
    slope += kWRepulsion * 2.0 * d;
  }
  if (kXsHydrophobic[ti] && kXsHydrophobic[tj]) {
    if (d < 0.5) {
      energy += kWHydrophobic * 1.0;
    } else if (d < 1.5) {
      energy += kWHydrophobic * (1.5 - d);
      slope += kWHydrophobic * (-1.0);
    }
  }
  const bool hbond = (kXsDonor[ti] && kXsAcceptor[tj]) || (kXsAcceptor[ti] && kXsDonor[tj]);
  if (hbond) {
    if (d < -0.7) {
      energy += kWHBond * 1.0;
    } else if (d < 0.0) {
      energy += kWHBond * (-d / 0.7);
      slope += kWHBond * (-1.0 / 0.7);
    }
  }
  *e = energy;
  *dedr = slope;
}

// ---------------------------------------------------------------------------
// Small vector / matrix helpers (FP64).
// ---------------------------------------------------------------------------
struct V3 {
  double x, y, z;
};
V3 v3(double x, double y, double z) { return V3{x, y, z}; }
V3 add(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
V3 sub(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
V3 scale(V3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct M3 {
  double m[3][3];
};
M3 identity3() {
  M3 r{};
  for (int i = 0; i < 3; ++i) r.m[i][i] = 1.0;
  return r;
}
M3 matmul(const M3& a, const M3& b) {
  M3 r{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) r.m[i][j] += a.m[i][k] * b.m[k][j];
  return r;
}
V3 matvec(const M3& a, V3 v) {
  return v3(a.m[0][0] * v.x + a.m[0][1] * v.y + a.m[0][2] * v.z,
            a.m[1][0] * v.x + a.m[1][1] * v.y + a.m[1][2] * v.z,
            a.m[2][0] * v.x + a.m[2][1] * v.y + a.m[2][2] * v.z);
}
// Rotation matrix of a unit quaternion (w, x, y, z), Hamilton convention.
M3 quat_to_matrix(const double q[4]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  M3 r;
  r.m[0][0] = 1 - 2 * (y * y + z * z);
  r.m[0][1] = 2 * (x * y - w * z);
  r.m[0][2] = 2 * (x * z + w * y);
  r.m[1][0] = 2 * (x * y + w * z);
  r.m[1][1] = 1 - 2 * (x * x + z * z);
  r.m[1][2] = 2 * (y * z - w * x);
  r.m[2][0] = 2 * (x * z - w * y);
  r.m[2][1] = 2 * (y * z + w * x);
  r.m[2][2] = 1 - 2 * (x * x + y * y);
  return r;
}
// Rodrigues' rotation about unit axis a by angle t (right-hand rule).
M3 axis_angle_matrix(V3 a, double t) {
  const double c = std::cos(t), s = std::sin(t), C = 1 - c;
  M3 r;
  r.m[0][0] = c + a.x * a.x * C;
  r.m[0][1] = a.x * a.y * C - a.z * s;
  r.m[0][2] = a.x * a.z * C + a.y * s;
  r.m[1][0] = a.y * a.x * C + a.z * s;
  r.m[1][1] = c + a.y * a.y * C;
  r.m[1][2] = a.y * a.z * C - a.x * s;
  r.m[2][0] = a.z * a.x * C - a.y * s;
  r.m[2][1] = a.z * a.y * C + a.x * s;
  r.m[2][2] = c + a.z * a.z * C;
  return r;
}
// Hamilton product a (x) b.
void quat_mul(const double a[4], const double b[4], double out[4]) {
  double r[4];
  r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  r[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  r[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  r[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  for (int i = 0; i < 4; ++i) out[i] = r[i];
}
// Unit quaternion of the rotation vector w (angle |w| about w/|w|).
void quat_from_rotvec(V3 w, double out[4]) {
  const double angle = norm(w);
  if (angle == 0.0) {
    out[0] = 1.0;
    out[1] = out[2] = out[3] = 0.0;
    return;
  }
  const double s = std::sin(angle / 2.0) / angle;
  out[0] = std::cos(angle / 2.0);
  out[1] = w.x * s;
  out[2] = w.y * s;
  out[3] = w.z * s;
}
void quat_normalize(double q[4]) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] /= n;
}
const double kPi = 3.14159265358979323846;
// Wrap an angle to (-pi, pi].
double wrap_angle(double t) { return t - 2.0 * kPi * std::ceil((t - kPi) / (2.0 * kPi)); }

// ---------------------------------------------------------------------------
// Grid maps (Sec. 2 first modification; Appendix Eq. 1 and Eq. 4).
// n[a] = ceil(size[a] / h) vertices per axis, origin = center - (n-1) h / 2,
// vertex (ix, iy, iz) at origin + h (ix, iy, iz).  maps layout:
// [type][iz][iy][ix][channel], channel 0 = sum_j f, channels 1..3 = its
// gradient with respect to the vertex position.  Parity: pinned (closed-form
// single-atom values, superposition, FD of channel 0, integer-node shifts).
// ---------------------------------------------------------------------------
struct Grid {
  int n[3];
  double origin[3];
  double h;
  const double* maps;  // borrowed
};

inline size_t map_index(const Grid& g, int t, int ix, int iy, int iz) {
  return ((((size_t)t * g.n[2] + iz) * g.n[1] + iy) * g.n[0] + ix) * 4;
}

// Score and gradient at point m for a ligand atom of type t: the plain sum over
// every receptor atom (Eq. 1 evaluated at a vertex).
void receptor_field(int n_rec, const double* rec_xyz, const int* rec_type, int t, V3 m, double cutoff,
                    double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  for (int j = 0; j < n_rec; ++j) {
    const V3 rj = v3(rec_xyz[3 * j], rec_xyz[3 * j + 1], rec_xyz[3 * j + 2]);
    const V3 dv = sub(m, rj);
    const double r = norm(dv);
    if (!(r < cutoff)) continue;
    double e, dedr;
    pair_term(t, rec_type[j], r, cutoff, &e, &dedr);
    out[0] += e;
    if (r > 0.0) {
      out[1] += dedr * dv.x / r;
      out[2] += dedr * dv.y / r;
      out[3] += dedr * dv.z / r;
    }
  }
}

void grid_dims(const double* size, double h, int n[3]) {
  for (int a = 0; a < 3; ++a) n[a] = (int)std::ceil(size[a] / h);
}

// ---------------------------------------------------------------------------
// Trilinear interpolation (Appendix Eq. 2, 3, 4) plus the out-of-grid wall.
// u = (x - origin)/h clamped to [0, n-1]; cell i = min(floor(u), n-2);
// p = u - i.  An atom outside the grid is evaluated at its clamped point and
// pays kWallSlope per Angstrom of excess along each axis (L1); along an axis
// where it is outside, its gradient is the wall slope alone.
// mode 0 = Eq. 4 (interpolated gradient maps), mode 1 = Eq. 3 (derivative of
// the interpolated score).  Parity: pinned (multilinear fields are reproduced
// exactly; Eq. 3 equals a finite difference of Eq. 2).
// ---------------------------------------------------------------------------
void interpolate(const Grid& g, int mode, int t, V3 x, double* e_out, V3* g_out) {
  const double xs[3] = {x.x, x.y, x.z};
  double p[3];
  int cell[3];
  double excess[3];
  for (int a = 0; a < 3; ++a) {
    double u = (xs[a] - g.origin[a]) / g.h;
    const double umax = (double)(g.n[a] - 1);
    excess[a] = 0.0;  // signed Angstrom outside the grid along axis a
    if (u < 0.0) {
      excess[a] = u * g.h;
      u = 0.0;
    } else if (u > umax) {
      excess[a] = (u - umax) * g.h;
      u = umax;
    }
    int i = (int)std::floor(u);
    if (i > g.n[a] - 2) i = g.n[a] - 2;
    if (i < 0) i = 0;
    cell[a] = i;
    p[a] = u - i;
  }
  double energy = 0.0;
  double grad[3] = {0.0, 0.0, 0.0};
  for (int l = 0; l <= 1; ++l)
    for (int m = 0; m <= 1; ++m)
      for (int n = 0; n <= 1; ++n) {
        const double wx = l ? p[0] : 1.0 - p[0];
        const double wy = m ? p[1] : 1.0 - p[1];
        const double wz = n ? p[2] : 1.0 - p[2];
        const double* node = g.maps + map_index(g, t, cell[0] + l, cell[1] + m, cell[2] + n);
        energy += wx * wy * wz * node[0];  // Eq. 2
        if (mode == 0) {                   // Eq. 4
          grad[0] += wx * wy * wz * node[1];
          grad[1] += wx * wy * wz * node[2];
          grad[2] += wx * wy * wz * node[3];
        } else {  // Eq. 3
          grad[0] += (2 * l - 1) / g.h * wy * wz * node[0];
          grad[1] += wx * (2 * m - 1) / g.h * wz * node[0];
          grad[2] += wx * wy * (2 * n - 1) / g.h * node[0];
        }
      }
  for (int a = 0; a < 3; ++a) {
    if (excess[a] != 0.0) {
      energy += kWallSlope * std::fabs(excess[a]);
      grad[a] = excess[a] > 0.0 ? kWallSlope : -kWallSlope;
    }
  }
  *e_out = energy;
  *g_out = v3(grad[0], grad[1], grad[2]);
}

// ---------------------------------------------------------------------------
// Ligand: rigid bodies, torsion tree, intra pair list.
// Bodies are the connected components left after cutting the rotatable bonds.
// Root = body with most atoms (ties: the body holding the lowest atom index).
// Torsion k is the k-th bond flagged rotatable, in input order.  The child
// body of torsion k rotates by theta_k about the axis from the parent-side
// atom to the child-side atom (right-hand rule), relative to the input
// (reference) geometry.  Intra pairs: i < j in different bodies and more than
// three bonds apart.  Parity: pinned (identity conformation, invariants,
// gradient vs central differences).
// ---------------------------------------------------------------------------
struct Ligand {
  int n_atoms = 0;
  std::vector<V3> ref;          // reference coordinates
  std::vector<int> type;        // XS type per atom
  std::vector<int> body_of;     // body index per atom
  int n_bodies = 0;
  int root = 0;
  int T = 0;
  // per body
  std::vector<int> parent;      // parent body (-1 for root)
  std::vector<int> origin_atom; // root: its lowest atom; child: child-side atom of its bond
  std::vector<int> axis_from;   // parent-side atom of the bond (-1 root)
  std::vector<int> torsion_of;  // torsion index driving the body (-1 root)
  std::vector<int> order;       // bodies parents-before-children (BFS from root)
  std::vector<int> torsion_body;  // body driven by torsion k
  std::vector<std::pair<int, int>> pairs;
  double gyration_radius = 1.0;
  bool ok = false;
};

bool build_ligand(Ligand& L, int n_atoms, const double* xyz, const int* types, int n_bonds, const int* bonds,
                  const int* rotatable) {
  L.n_atoms = n_atoms;
  if (n_atoms <= 0) return false;
  L.ref.resize(n_atoms);
  L.type.assign(types, types + n_atoms);
  for (int i = 0; i < n_atoms; ++i) {
    L.ref[i] = v3(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
    if (L.type[i] < 0 || L.type[i] >= kNumMapTypes) return false;
  }
  std::vector<std::vector<int>> adj(n_atoms), rigid_adj(n_atoms);
  for (int b = 0; b < n_bonds; ++b) {
    const int i = bonds[2 * b], j = bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= n_atoms || j >= n_atoms || i == j) return false;
    adj[i].push_back(j);
    adj[j].push_back(i);
    if (!rotatable[b]) {
      rigid_adj[i].push_back(j);
      rigid_adj[j].push_back(i);
    }
  }
  // bodies: connected components over non-rotatable bonds, numbered by lowest atom
  L.body_of.assign(n_atoms, -1);
  L.n_bodies = 0;
  for (int s = 0; s < n_atoms; ++s) {
    if (L.body_of[s] >= 0) continue;
    std::vector<int> stack{s};
    L.body_of[s] = L.n_bodies;
    while (!stack.empty()) {
      const int a = stack.back();
      stack.pop_back();
      for (int b : rigid_adj[a])
        if (L.body_of[b] < 0) {
          L.body_of[b] = L.n_bodies;
          stack.push_back(b);
        }
    }
    ++L.n_bodies;
  }
  // every rotatable bond must join two different bodies
  std::vector<int> rot_bonds;
  for (int b = 0; b < n_bonds; ++b)
    if (rotatable[b]) {
      if (L.body_of[bonds[2 * b]] == L.body_of[bonds[2 * b + 1]]) return false;
      rot_bonds.push_back(b);
    }
  L.T = (int)rot_bonds.size();
  if (L.T != L.n_bodies - 1) return false;  // body graph must be a tree
  // root body
  std::vector<int> count(L.n_bodies, 0);
  for (int i = 0; i < n_atoms; ++i) ++count[L.body_of[i]];
  L.root = 0;
  for (int b = 1; b < L.n_bodies; ++b)
    if (count[b] > count[L.root]) L.root = b;  // bodies numbered by lowest atom: ties keep the lower
  // BFS over the body tree
  L.parent.assign(L.n_bodies, -2);
  L.origin_atom.assign(L.n_bodies, -1);
  L.axis_from.assign(L.n_bodies, -1);
  L.torsion_of.assign(L.n_bodies, -1);
  L.torsion_body.assign(L.T, -1);
  L.order.clear();
  L.parent[L.root] = -1;
  for (int i = 0; i < n_atoms; ++i)
    if (L.body_of[i] == L.root) {
      L.origin_atom[L.root] = i;
      break;
    }
  std::vector<int> queue{L.root};
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    const int b = queue[qi];
    L.order.push_back(b);
    for (int k = 0; k < L.T; ++k) {
      const int bi = bonds[2 * rot_bonds[k]], bj = bonds[2 * rot_bonds[k] + 1];
      int near = -1, far = -1;
      if (L.body_of[bi] == b) near = bi, far = bj;
      else if (L.body_of[bj] == b) near = bj, far = bi;
      if (near < 0) continue;
      const int c = L.body_of[far];
      if (L.parent[c] != -2) continue;  // already reached (this bond leads to b's parent)
      L.parent[c] = b;
      L.origin_atom[c] = far;
      L.axis_from[c] = near;
      L.torsion_of[c] = k;
      L.torsion_body[k] = c;
      queue.push_back(c);
    }
  }
  if ((int)L.order.size() != L.n_bodies) return false;
  // topological (bond-count) distances for the intra pair rule
  std::vector<int> dist(n_atoms);
  L.pairs.clear();
  for (int i = 0; i < n_atoms; ++i) {
    std::fill(dist.begin(), dist.end(), -1);
    std::vector<int> q{i};
    dist[i] = 0;
    for (size_t qi = 0; qi < q.size(); ++qi)
      for (int b : adj[q[qi]])
        if (dist[b] < 0) {
          dist[b] = dist[q[qi]] + 1;
          q.push_back(b);
        }
    for (int j = i + 1; j < n_atoms; ++j) {
      const bool far_apart = dist[j] < 0 || dist[j] > 3;
      if (L.body_of[i] != L.body_of[j] && far_apart) L.pairs.push_back({i, j});
    }
  }
  // gyration radius of the reference geometry about the root origin
  double s2 = 0.0;
  const V3 o = L.ref[L.origin_atom[L.root]];
  for (int i = 0; i < n_atoms; ++i) {
    const V3 d = sub(L.ref[i], o);
    s2 += dot(d, d);
  }
  L.gyration_radius = std::sqrt(s2 / n_atoms);
  L.ok = true;
  return true;
}

// Conformation: c[0..2] = position of the root origin atom, c[3..6] = unit
// quaternion (w, x, y, z), c[7 + k] = theta_k.
struct Pose {
  std::vector<V3> atom;        // world coordinates
  std::vector<M3> R;           // body rotation
  std::vector<V3> origin;      // body origin (world)
  std::vector<V3> axis;        // world torsion axis per body (unit), zero for root
};

void forward_kinematics(const Ligand& L, const double* c, Pose& P) {
  P.R.assign(L.n_bodies, identity3());
  P.origin.assign(L.n_bodies, v3(0, 0, 0));
  P.axis.assign(L.n_bodies, v3(0, 0, 0));
  P.atom.assign(L.n_atoms, v3(0, 0, 0));
  double q[4] = {c[3], c[4], c[5], c[6]};
  quat_normalize(q);
  for (int b : L.order) {
    if (L.parent[b] < 0) {
      P.R[b] = quat_to_matrix(q);
      P.origin[b] = v3(c[0], c[1], c[2]);
    } else {
      const int pb = L.parent[b];
      const V3 axis_ref = scale(sub(L.ref[L.origin_atom[b]], L.ref[L.axis_from[b]]),
                                1.0 / norm(sub(L.ref[L.origin_atom[b]], L.ref[L.axis_from[b]])));
      P.origin[b] = add(P.origin[pb], matvec(P.R[pb], sub(L.ref[L.origin_atom[b]], L.ref[L.origin_atom[pb]])));
      P.R[b] = matmul(P.R[pb], axis_angle_matrix(axis_ref, c[7 + L.torsion_of[b]]));
      P.axis[b] = matvec(P.R[pb], axis_ref);
    }
  }
  for (int i = 0; i < L.n_atoms; ++i) {
    const int b = L.body_of[i];
    P.atom[i] = add(P.origin[b], matvec(P.R[b], sub(L.ref[i], L.ref[L.origin_atom[b]])));
  }
}

// Chain rule from atom gradients g_i = dE/dr_i to the conformation gradient
// [dE/dp (3), dE/domega (3, world rotation vector about p), dE/dtheta (T)].
void conf_gradient(const Ligand& L, const Pose& P, const std::vector<V3>& g, double* out) {
  const int root = L.root;
  const V3 p = P.origin[root];
  V3 f = v3(0, 0, 0), tau = v3(0, 0, 0);
  for (int i = 0; i < L.n_atoms; ++i) {
    f = add(f, g[i]);
    tau = add(tau, cross(sub(P.atom[i], p), g[i]));
  }
  out[0] = f.x, out[1] = f.y, out[2] = f.z;
  out[3] = tau.x, out[4] = tau.y, out[5] = tau.z;
  for (int k = 0; k < L.T; ++k) {
    const int b = L.torsion_body[k];
    // subtree of b: bodies whose ancestor chain passes through b
    V3 t = v3(0, 0, 0);
    for (int i = 0; i < L.n_atoms; ++i) {
      int a = L.body_of[i];
      bool inside = false;
      while (a >= 0) {
        if (a == b) {
          inside = true;
          break;
        }
        a = L.parent[a];
      }
      if (inside) t = add(t, cross(sub(P.atom[i], P.origin[b]), g[i]));
    }
    out[6 + k] = dot(P.axis[b], t);
  }
}

struct Receptor {
  int n = 0;
  const double* xyz = nullptr;
  const int* type = nullptr;
};

// Energy terms selected by flags: bit 0 inter (grid or exact), bit 1 intra.
struct Terms {
  double inter = 0.0, intra = 0.0;
};

// Search objective on grid maps (grid != null) or gridless exact (rec != null).
Terms evaluate(const Ligand& L, const Grid* grid, int mode, const Receptor* rec, const double* c, int flags,
               double* grad_out, Pose* pose_out = nullptr) {
  Pose P;
  forward_kinematics(L, c, P);
  std::vector<V3> g(L.n_atoms, v3(0, 0, 0));
  Terms T;
  if (flags & 1) {
    for (int i = 0; i < L.n_atoms; ++i) {
      if (grid) {
        double e;
        V3 gi;
        interpolate(*grid, mode, L.type[i], P.atom[i], &e, &gi);
        T.inter += e;
        g[i] = add(g[i], gi);
      } else {
        double f[4];
        receptor_field(rec->n, rec->xyz, rec->type, L.type[i], P.atom[i], kCutoff, f);
        T.inter += f[0];
        g[i] = add(g[i], v3(f[1], f[2], f[3]));
      }
    }
  }
  if (flags & 2) {
    for (const auto& pr : L.pairs) {
      const int i = pr.first, j = pr.second;
      const V3 dv = sub(P.atom[i], P.atom[j]);
      const double r = norm(dv);
      double e, dedr;
      pair_term(L.type[i], L.type[j], r, kCutoff, &e, &dedr);
      T.intra += e;
      if (r > 0.0) {
        const V3 gi = scale(dv, dedr / r);
        g[i] = add(g[i], gi);
        g[j] = sub(g[j], gi);
      }
    }
  }
  if (grad_out) conf_gradient(L, P, g, grad_out);
  if (pose_out) *pose_out = P;
  return T;
}

// Apply a step s (6 + T) to conformation c (7 + T) in place: translate,
// rotate by the world rotation vector s[3..5] (q <- quat(s) (x) q), add torsions.
void apply_step(const Ligand& L, double* c, const double* s) {
  c[0] += s[0], c[1] += s[1], c[2] += s[2];
  double dq[4], q[4] = {c[3], c[4], c[5], c[6]};
  quat_from_rotvec(v3(s[3], s[4], s[5]), dq);
  quat_mul(dq, q, q);
  quat_normalize(q);
  for (int i = 0; i < 4; ++i) c[3 + i] = q[i];
  for (int k = 0; k < L.T; ++k) c[7 + k] = wrap_angle(c[7 + k] + s[6 + k]);
}

// ---------------------------------------------------------------------------
// Optimisers.  A generic objective works on x (dim nx) and a tangent step of
// dim nd; the docking objective has nx = 7 + T, nd = 6 + T; the Euclidean
// test objectives have nx = nd.
// ---------------------------------------------------------------------------
struct Objective {
  int nx, nd;
  virtual double eval(const double* x, double* g) = 0;   // returns E, fills g[nd]
  virtual void step(double* x, const double* s) = 0;     // x <- x (+) s
  virtual ~Objective() {}
};

// A decision the search takes by comparing two computed quantities, with its
// margin: the quantity whose sign selects the branch.  Recorded (optionally)
// so that a test can tell a near tie -- a branch FP32 and FP64 arithmetic may
// take differently -- from a real disagreement.  kind and margin:
//   0 Armijo test of a BFGS trial (Nocedal & Wright Alg. 6.1 with backtracking):
//     E(x + alpha d) - (E(x) + c1 alpha g.d); the trial is accepted iff <= 0
//   1 Barzilai-Borwein best iterate: E_new - E_best; a new best iff < 0
//   2 Metropolis acceptance of an MC candidate: (E' - E) + T ln u; accepted iff < 0
//     (equivalent to E' < E or u < exp(-(E' - E) / T) for u in [0, 1))
//   3 BFGS curvature condition: y.s - min_curvature; H is updated iff > 0
//   4 Barzilai-Borwein curvature: s.y; the BB1 step is taken iff > 0
//   5 cell choice of an Eq. 3 evaluation: the smallest distance (A) of an atom
//     inside the grid to a face of its cell, where Eq. 3's gradient jumps (one
//     record per evaluation on Eq. 3 maps; Eq. 4's gradient is continuous there)
// scale: |s|_1 (|g|_inf + |g'|_inf) for kinds 3 and 4 -- the bound on how far
// s.y moves when each gradient component moves by a fraction of its norm --,
// 0 otherwise (the energies' own scale applies).
struct Decision {
  int kind;
  double margin;
  double scale;
};

struct OptSettings {
  std::vector<Decision>* log = nullptr;  // decisions taken, appended in order (recording only)
  int max_iters = 100;
  // BFGS (Nocedal & Wright, Algorithm 6.1 with backtracking Armijo search)
  double c1 = 1e-4;
  double shrink = 0.5;
  int max_trials = 10;
  double min_curvature = 1e-10;
  // Barzilai-Borwein (paper Sec. 2 second modification, ref. 37): BB1 step
  double bb_alpha0 = 1e-3;
  double bb_alpha_min = 1e-4;
  double bb_alpha_max = 0.1;
  // Every step the optimisers take is multiplied by this factor; 1 (exact) by
  // default.  Tests set it to 1 +- 2^-24 to measure the search's own response
  // to a one-ulp FP32 rounding of its steps (a sensitivity probe, not part of
  // the method).
  double step_scale = 1.0;
  // Every gradient the optimisers see gets delta |g|_inf p_i added, p_i =
  // ((7 i + 3) mod 5 - 2) / 2; 0 (exact) by default.  Tests set it to the FP32
  // gradient error measured on the GPU to measure the search's own response to
  // gradients of that accuracy (a sensitivity probe, not part of the method).
  double grad_perturb = 0.0;
};

// The gradient probe of OptSettings::grad_perturb (no-op at 0).
void perturb_gradient(const OptSettings& st, int n, double* g) {
  if (st.grad_perturb == 0.0) return;
  double gm = 0.0;
  for (int i = 0; i < n; ++i) gm = std::max(gm, std::fabs(g[i]));
  for (int i = 0; i < n; ++i) g[i] += st.grad_perturb * gm * (double)((7 * i + 3) % 5 - 2) * 0.5;
}

struct OptResult {
  double e;
  long evals;
  int iters;
};

// BFGS inverse-Hessian update (Nocedal & Wright Eq. 6.17):
// H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / (y^T s).
void bfgs_update(int n, std::vector<double>& H, const double* s, const double* y) {
  double sy = 0.0;
  for (int i = 0; i < n; ++i) sy += s[i] * y[i];
  const double rho = 1.0 / sy;
  std::vector<double> A(n * n), tmp(n * n, 0.0), out(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = (i == j ? 1.0 : 0.0) - rho * s[i] * y[j];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) tmp[i * n + j] += A[i * n + k] * H[k * n + j];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      for (int k = 0; k < n; ++k) out[i * n + j] += tmp[i * n + k] * A[j * n + k];  // times A^T
      out[i * n + j] += rho * s[i] * s[j];
    }
  H = out;
}

// BFGS from x (updated in place to the final iterate).  Each iteration takes
// the direction d = -H g and backtracks alpha = 1, shrink, shrink^2, ... until
// E(x (+) alpha d) <= E + c1 alpha g.d; if no trial passes, the search stops.
// H is updated only when y.s > min_curvature.
OptResult bfgs(Objective& f, double* x, const OptSettings& st) {
  const int nx = f.nx, n = f.nd;
  std::vector<double> H(n * n, 0.0), g(n), d(n), gt(n), xt(nx), s(n), y(n);
  for (int i = 0; i < n; ++i) H[i * n + i] = 1.0;
  OptResult R{0.0, 0, 0};
  double e = f.eval(x, g.data());
  perturb_gradient(st, n, g.data());
  R.evals = 1;
  for (int it = 0; it < st.max_iters; ++it) {
    for (int i = 0; i < n; ++i) {
      d[i] = 0.0;
      for (int j = 0; j < n; ++j) d[i] -= H[i * n + j] * g[j];
    }
    double gd = 0.0;
    for (int i = 0; i < n; ++i) gd += g[i] * d[i];
    double alpha = 1.0, et = 0.0;
    bool accepted = false;
    for (int trial = 0; trial < st.max_trials; ++trial) {
      for (int i = 0; i < nx; ++i) xt[i] = x[i];
      for (int i = 0; i < n; ++i) s[i] = alpha * d[i] * st.step_scale;
      f.step(xt.data(), s.data());
      et = f.eval(xt.data(), gt.data());
      perturb_gradient(st, n, gt.data());
      ++R.evals;
      if (st.log) st.log->push_back(Decision{0, et - (e + st.c1 * alpha * gd), 0.0});
      if (et <= e + st.c1 * alpha * gd) {
        accepted = true;
        break;
      }
      alpha *= st.shrink;
    }
    if (!accepted) break;
    for (int i = 0; i < n; ++i) y[i] = gt[i] - g[i];
    double sy = 0.0;
    for (int i = 0; i < n; ++i) sy += s[i] * y[i];
    for (int i = 0; i < nx; ++i) x[i] = xt[i];
    for (int i = 0; i < n; ++i) g[i] = gt[i];
    e = et;
    R.iters = it + 1;
    if (st.log) {  // g is already the new gradient; the old one is g - y
      double s1 = 0.0, gi = 0.0, go = 0.0;
      for (int i = 0; i < n; ++i)
        s1 += std::fabs(s[i]), gi = std::max(gi, std::fabs(g[i])), go = std::max(go, std::fabs(g[i] - y[i]));
      st.log->push_back(Decision{3, sy - st.min_curvature, s1 * (gi + go)});
    }
    if (sy > st.min_curvature) bfgs_update(n, H, s.data(), y.data());
  }
  R.e = e;
  return R;
}

// Barzilai-Borwein: x_{k+1} = x_k (+) (-alpha_k g_k) with the BB1 step
// alpha_{k+1} = s.s / s.y (alpha_max when s.y <= 0), clamped to
// [alpha_min, alpha_max]; no line search; returns the best iterate seen.
OptResult barzilai_borwein(Objective& f, double* x, const OptSettings& st) {
  const int nx = f.nx, n = f.nd;
  std::vector<double> g(n), gn(n), s(n), xbest(x, x + nx);
  OptResult R{0.0, 0, 0};
  double e = f.eval(x, g.data());
  perturb_gradient(st, n, g.data());
  R.evals = 1;
  double ebest = e;
  double alpha = st.bb_alpha0;
  for (int it = 0; it < st.max_iters; ++it) {
    for (int i = 0; i < n; ++i) s[i] = -alpha * g[i] * st.step_scale;
    f.step(x, s.data());
    const double en = f.eval(x, gn.data());
    perturb_gradient(st, n, gn.data());
    ++R.evals;
    double sy = 0.0, ss = 0.0;
    for (int i = 0; i < n; ++i) {
      sy += s[i] * (gn[i] - g[i]);
      ss += s[i] * s[i];
    }
    if (st.log) {
      double s1 = 0.0, gi = 0.0, go = 0.0;
      for (int i = 0; i < n; ++i)
        s1 += std::fabs(s[i]), gi = std::max(gi, std::fabs(gn[i])), go = std::max(go, std::fabs(g[i]));
      st.log->push_back(Decision{4, sy, s1 * (gi + go)});
    }
    if (sy > 0.0) {
      alpha = ss / sy;
      if (alpha < st.bb_alpha_min) alpha = st.bb_alpha_min;
      if (alpha > st.bb_alpha_max) alpha = st.bb_alpha_max;
    } else {
      alpha = st.bb_alpha_max;
    }
    for (int i = 0; i < n; ++i) g[i] = gn[i];
    e = en;
    R.iters = it + 1;
    if (st.log) st.log->push_back(Decision{1, e - ebest, 0.0});
    if (e < ebest) {
      ebest = e;
      for (int i = 0; i < nx; ++i) xbest[i] = x[i];
    }
  }
  for (int i = 0; i < nx; ++i) x[i] = xbest[i];
  R.e = ebest;
  return R;
}

struct DockObjective : Objective {
  const Ligand* L;
  const Grid* grid;
  int mode;
  std::vector<Decision>* log = nullptr;  // kind 5 records on Eq. 3 maps (recording only)
  DockObjective(const Ligand* l, const Grid* g, int m) : L(l), grid(g), mode(m) {
    nx = 7 + l->T;
    nd = 6 + l->T;
  }
  double eval(const double* x, double* g) override {
    Pose P;
    const Terms t = evaluate(*L, grid, mode, nullptr, x, 3, g, log && mode == 1 ? &P : nullptr);
    if (log && mode == 1) {
      double dmin = 1e300;
      for (const V3& a : P.atom) {
        const double r[3] = {a.x, a.y, a.z};
        for (int k = 0; k < 3; ++k) {
          const double u = (r[k] - grid->origin[k]) / grid->h;
          if (!(u > 0.0 && u < grid->n[k] - 1)) continue;  // on the wall: no cell face
          const double f = u - std::floor(u);
          dmin = std::min(dmin, std::min(f, 1.0 - f) * grid->h);
        }
      }
      log->push_back(Decision{5, dmin, 0.0});
    }
    return t.inter + t.intra;
  }
  void step(double* x, const double* s) override { apply_step(*L, x, s); }
};

// Euclidean quadratic 0.5 x^T A x - b^T x (test objective for the optimisers).
struct QuadObjective : Objective {
  const double* A;
  const double* b;
  QuadObjective(int n, const double* a, const double* bb) : A(a), b(bb) { nx = nd = n; }
  double eval(const double* x, double* g) override {
    double e = 0.0;
    for (int i = 0; i < nx; ++i) {
      double ax = 0.0;
      for (int j = 0; j < nx; ++j) ax += A[i * nx + j] * x[j];
      g[i] = ax - b[i];
      e += 0.5 * x[i] * ax - b[i] * x[i];
    }
    return e;
  }
  void step(double* x, const double* s) override {
    for (int i = 0; i < nx; ++i) x[i] += s[i];
  }
};

// Rosenbrock sum_i 100 (x_{i+1} - x_i^2)^2 + (1 - x_i)^2 (minimum at all ones).
struct RosenObjective : Objective {
  explicit RosenObjective(int n) { nx = nd = n; }
  double eval(const double* x, double* g) override {
    double e = 0.0;
    for (int i = 0; i < nx; ++i) g[i] = 0.0;
    for (int i = 0; i + 1 < nx; ++i) {
      const double a = x[i + 1] - x[i] * x[i], b = 1.0 - x[i];
      e += 100.0 * a * a + b * b;
      g[i] += -400.0 * a * x[i] - 2.0 * b;
      g[i + 1] += 200.0 * a;
    }
    return e;
  }
  void step(double* x, const double* s) override {
    for (int i = 0; i < nx; ++i) x[i] += s[i];
  }
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. SC'11): 10 rounds of the 4x32 Philox round with
// multipliers 0xD2511F53, 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
// 0xBB67AE85.  Parity: pinned to a library implementation of the same
// generator (tests).
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Random stream of one chain at one MC step: word w of block b comes from
// Philox(counter = (chain, step, b, 0), key = (seed_lo, seed_hi)).
struct ChainRng {
  uint32_t key[2];
  uint32_t chain;
  uint32_t word(uint32_t step, uint32_t block, int w) const {
    const uint32_t ctr[4] = {chain, step, block, 0u};
    uint32_t out[4];
    philox4x32_10(ctr, key, out);
    return out[w];
  }
  // uniform in [0, 1): top 24 bits times 2^-24 (exact in FP32 and FP64)
  double uniform(uint32_t step, uint32_t block, int w) const {
    return (double)(word(step, block, w) >> 8) * (1.0 / 16777216.0);
  }
};

// Uniform point in the unit ball by rejection: attempt a (0..15) uses block
// 1 + a; each coordinate is (word >> 8) - 2^23, accepted when the integer sum
// of squares is <= 2^46; the point is v / 2^23.  After 16 rejections: origin.
V3 unit_ball(const ChainRng& rng, uint32_t step) {
  for (int a = 0; a < 16; ++a) {
    int64_t v[3];
    for (int w = 0; w < 3; ++w) v[w] = (int64_t)(rng.word(step, 1 + a, w) >> 8) - (int64_t)(1 << 23);
    const int64_t s2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (s2 <= ((int64_t)1 << 46)) return v3(v[0] / 8388608.0, v[1] / 8388608.0, v[2] / 8388608.0);
  }
  return v3(0, 0, 0);
}

// ---------------------------------------------------------------------------
// Monte Carlo chain (Sec. 2: many short independent copies; Vina's mutation
// and Metropolis rules, ref. 6).
//   init (step 0): p uniform in the search box (uniform words 0..2 of the
//     step-0 stream), q from words 3..5 (Shoemake's uniform rotation),
//     theta_k = pi - 2 pi u (word 6 + k); word n is word n%4 of block n/4.
//   then local optimisation; the result is the current and best state.
//   step s >= 1: mode m = floor(u0 * (2 + T)) by integer arithmetic on word 0;
//     m = 0: p += 2 * ball; m = 1: q <- quat((2 / R_gyr) * ball) (x) q;
//     m = 2 + k: theta_k = pi - 2 pi u2; then local optimisation; accept when
//     E' < E or u1 < exp(-(E' - E) / T_mc); an accepted state better than the
//     best becomes the best.
// Parity: unpinned against the paper (it does not print the MC rules); pinned
// by determinism, batch independence and self-docking sanity in the tests, and
// the mutations against the moves stated here (mode uniform over 2 + T, move
// sizes by their unit-ball distribution, one coordinate group per move).
// ---------------------------------------------------------------------------
struct DockSettings {
  int n_mc_steps = 40;
  int optimizer = 0;  // 0 BFGS, 1 BB
  double temperature = 1.2;
  double box_lo[3], box_size[3];
  // adaptive search space: n_sites predicted binding-site points [3 n_sites]
  // (values representable in FP32) and the ball radius; n_sites = 0: the box
  int n_sites = 0;
  const double* sites = nullptr;
  double site_radius = 7.0;
  OptSettings opt;
};

struct StepRecord {
  int mode;
  int accepted;
  double e_candidate;
  double e_current;
  long evals;
};

OptResult local_opt(DockObjective& obj, double* x, const DockSettings& ds) {
  return ds.optimizer == 0 ? bfgs(obj, x, ds.opt) : barzilai_borwein(obj, x, ds.opt);
}

// Adaptive search space (Sec. 2, third modification; Fig. 3): the search
// region is the box intersected with the union of balls of radius R around the
// predicted binding-site points, and the initial positions are drawn uniformly
// from it.  Reading: rejection from the box -- attempt a uses the uniforms of
// block 0 (a = 0) or block 64 + a (a >= 1) of step 0, words 0-2; the candidate
// is lo + size u and it is accepted when its squared distance to some point is
// at most R^2; after 64 rejections the first point is taken.  The accept
// decision is made in FP32 (candidate by one fused multiply-add per axis,
// distance ((dx dx + dy dy) + dz dz) with every operation rounded), as the GPU
// makes it, so both take the same branch; the accepted position itself is
// lo + size u in FP64.  Parity: pinned by the tests (every start inside the
// region, the box case unchanged when the balls cover the box, uniformity in a
// ball).
bool site_accepts_f32(const DockSettings& ds, const double* u) {
  float c[3];
  for (int a = 0; a < 3; ++a) c[a] = std::fmaf((float)ds.box_size[a], (float)u[a], (float)ds.box_lo[a]);
  const float r2 = (float)ds.site_radius * (float)ds.site_radius;
  for (int k = 0; k < ds.n_sites; ++k) {
    const float dx = c[0] - (float)ds.sites[3 * k], dy = c[1] - (float)ds.sites[3 * k + 1],
                dz = c[2] - (float)ds.sites[3 * k + 2];
    const float d2 = (dx * dx + dy * dy) + dz * dz;
    if (d2 <= r2) return true;
  }
  return false;
}

void initial_position(const ChainRng& rng, const DockSettings& ds, double* c) {
  double u[3] = {rng.uniform(0, 0, 0), rng.uniform(0, 0, 1), rng.uniform(0, 0, 2)};
  if (ds.n_sites > 0) {
    bool found = false;
    for (int a = 0; a < 64 && !found; ++a) {
      if (a > 0)
        for (int w = 0; w < 3; ++w) u[w] = rng.uniform(0, 64 + a, w);
      found = site_accepts_f32(ds, u);
    }
    if (!found) {
      for (int a = 0; a < 3; ++a) c[a] = (double)(float)ds.sites[a];
      return;
    }
  }
  for (int a = 0; a < 3; ++a) c[a] = ds.box_lo[a] + ds.box_size[a] * u[a];
}

void chain_init(const Ligand& L, const ChainRng& rng, const DockSettings& ds, double* c) {
  auto U = [&](int n) { return rng.uniform(0, n / 4, n % 4); };
  initial_position(rng, ds, c);
  const double u1 = U(3), u2 = U(4), u3 = U(5);
  c[3] = std::sqrt(u1) * std::cos(2 * kPi * u3);
  c[4] = std::sqrt(1 - u1) * std::sin(2 * kPi * u2);
  c[5] = std::sqrt(1 - u1) * std::cos(2 * kPi * u2);
  c[6] = std::sqrt(u1) * std::sin(2 * kPi * u3);
  for (int k = 0; k < L.T; ++k) c[7 + k] = kPi - 2 * kPi * U(6 + k);
}

int mutation_mode(const ChainRng& rng, uint32_t step, int T) {
  const uint64_t u24 = rng.word(step, 0, 0) >> 8;
  return (int)((u24 * (uint64_t)(2 + T)) >> 24);
}

void mutate(const Ligand& L, const ChainRng& rng, uint32_t step, double* c, int mode) {
  if (mode == 0) {
    const V3 b = unit_ball(rng, step);
    c[0] += 2.0 * b.x, c[1] += 2.0 * b.y, c[2] += 2.0 * b.z;
  } else if (mode == 1) {
    const V3 b = scale(unit_ball(rng, step), 2.0 / L.gyration_radius);
    double dq[4], q[4] = {c[3], c[4], c[5], c[6]};
    quat_from_rotvec(b, dq);
    quat_mul(dq, q, q);
    quat_normalize(q);
    for (int i = 0; i < 4; ++i) c[3 + i] = q[i];
  } else {
    c[7 + (mode - 2)] = kPi - 2 * kPi * rng.uniform(step, 0, 2);
  }
}

// One MC step from (cur, e_cur): returns the record; cur/e_cur updated.
StepRecord mc_step(const Ligand& L, DockObjective& obj, const ChainRng& rng, const DockSettings& ds, uint32_t step,
                   double* cur, double* e_cur, double* best, double* e_best) {
  const int nx = 7 + L.T;
  std::vector<double> cand(cur, cur + nx);
  StepRecord rec;
  rec.mode = mutation_mode(rng, step, L.T);
  mutate(L, rng, step, cand.data(), rec.mode);
  const OptResult r = local_opt(obj, cand.data(), ds);
  rec.evals = r.evals;
  rec.e_candidate = r.e;
  const double u = rng.uniform(step, 0, 1);
  rec.accepted = (r.e < *e_cur) || (u < std::exp(-(r.e - *e_cur) / ds.temperature));
  if (ds.opt.log)
    ds.opt.log->push_back(Decision{2, u > 0.0 ? (r.e - *e_cur) + ds.temperature * std::log(u) : -1e300, 0.0});
  if (rec.accepted) {
    for (int i = 0; i < nx; ++i) cur[i] = cand[i];
    *e_cur = r.e;
    if (r.e < *e_best) {
      for (int i = 0; i < nx; ++i) best[i] = cand[i];
      *e_best = r.e;
    }
  }
  rec.e_current = *e_cur;
  return rec;
}

long run_chain(const Ligand& L, const Grid& grid, int mode, const DockSettings& ds, uint64_t seed, uint32_t chain,
               double* best, double* e_best, double* trace_conf, StepRecord* trace) {
  const int nx = 7 + L.T;
  DockObjective obj(&L, &grid, mode);
  ChainRng rng{{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}, chain};
  std::vector<double> cur(nx);
  chain_init(L, rng, ds, cur.data());
  OptResult r0 = local_opt(obj, cur.data(), ds);
  double e_cur = r0.e;
  long evals = r0.evals;
  for (int i = 0; i < nx; ++i) best[i] = cur[i];
  *e_best = e_cur;
  if (trace_conf)
    for (int i = 0; i < nx; ++i) trace_conf[i] = cur[i];
  if (trace) trace[0] = StepRecord{-1, 1, e_cur, e_cur, r0.evals};
  for (int s = 1; s <= ds.n_mc_steps; ++s) {
    StepRecord rec = mc_step(L, obj, rng, ds, (uint32_t)s, cur.data(), &e_cur, best, e_best);
    evals += rec.evals;
    if (trace_conf)
      for (int i = 0; i < nx; ++i) trace_conf[(size_t)s * nx + i] = cur[i];
    if (trace) trace[s] = rec;
  }
  return evals;
}

double rmsd(const std::vector<V3>& a, const std::vector<V3>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const V3 d = sub(a[i], b[i]);
    s += dot(d, d);
  }
  return std::sqrt(s / a.size());
}

}  // namespace

// ===========================================================================
// C interface for the tests (ctypes).  All arrays are host memory owned by the
// caller; ligand handles are owned by the caller until orc_ligand_free.
// ===========================================================================

// ---------------------------------------------------------------------------
// Receptor voxel features (Sec. 2, "Protein-ligand binding site prediction"):
// the protein as 36 x 36 x 36 voxels with 18 features, centred on the protein
// and 70 A on a side; DSDP merges the S and Se channels and uses the freed
// channel for the protein surface.  Reading (the paper gives the grid, the
// span, the channel count and the two changes, not the per-atom features):
//   * the cube [c - 35, c + 35)^3 is cut into 36^3 voxels of edge 70/36 A; an
//     atom belongs to voxel k = floor((x - (c - 35)) * (36/70)) per axis when
//     0 <= k < 36 on every axis (atoms outside are dropped); this decision is
//     taken in FP32, subtraction then multiplication, as the kernel takes it;
//   * channels 0..16 are the sums over the voxel's atoms of 17 per-atom
//     features supplied by the caller (the feature list is the site network's,
//     an input here);
//   * channel 17 counts the voxel's surface atoms: atom i is on the surface
//     when some test point x_i + (r_i + 1.4) u_k of its solvent-accessible
//     sphere (probe radius 1.4 A) lies outside every other atom's sphere of
//     radius r_j + 1.4 (Shrake & Rupley, J. Mol. Biol. 79, 351 (1973)).  The
//     98 test directions u_k are the integer vectors (a, b, c) in {-2..2}^3
//     with gcd(|a|, |b|, |c|) = 1, normalised; the point and distance tests are
//     FP32 with a fixed operation order (the kernel's), so both take the same
//     decisions;
//   * sums are exact: each feature is rounded to a multiple of 2^-24 and
//     accumulated as a 64-bit integer, so the result does not depend on the
//     order of the atoms; a channel is the sum times 2^-24 rounded to FP32.
// Parity: pinned by the tests (hand-placed atoms, an isolated atom and a
// buried one, the exposed fraction of two overlapping spheres, and a
// brute-force recount).
// ---------------------------------------------------------------------------
constexpr int kVoxN = 36;
constexpr int kVoxFeatures = 17;
constexpr int kVoxChannels = 18;

// The 98 test directions, FP32 (sqrt and division are correctly rounded).
static int sas_directions(float* u) {
  int m = 0;
  for (int a = -2; a <= 2; ++a)
    for (int b = -2; b <= 2; ++b)
      for (int c = -2; c <= 2; ++c) {
        if (a == 0 && b == 0 && c == 0) continue;
        int g = std::abs(a);
        for (int v : {std::abs(b), std::abs(c)}) {
          int x = g, y = v;
          while (y) {
            const int t = x % y;
            x = y;
            y = t;
          }
          g = x;
        }
        if (g != 1) continue;
        const float len = std::sqrt((float)(a * a + b * b + c * c));
        u[3 * m] = (float)a / len, u[3 * m + 1] = (float)b / len, u[3 * m + 2] = (float)c / len;
        ++m;
      }
  return m;
}

// Exposed test points of every atom (out[n]); xyz, radius FP32-representable.
static void sas_exposed(int n, const float* xyz, const float* radius, int* exposed) {
  float u[3 * 98];
  const int m = sas_directions(u);
  for (int i = 0; i < n; ++i) {
    const float Ri = radius[i] + 1.4f;
    int count = 0;
    for (int k = 0; k < m; ++k) {
      const float p[3] = {xyz[3 * i] + Ri * u[3 * k], xyz[3 * i + 1] + Ri * u[3 * k + 1],
                          xyz[3 * i + 2] + Ri * u[3 * k + 2]};
      bool buried = false;
      for (int j = 0; j < n && !buried; ++j) {
        if (j == i) continue;
        const float dx = p[0] - xyz[3 * j], dy = p[1] - xyz[3 * j + 1], dz = p[2] - xyz[3 * j + 2];
        const float d2 = (dx * dx + dy * dy) + dz * dz;
        const float Rj = radius[j] + 1.4f;
        buried = d2 < Rj * Rj;
      }
      count += !buried;
    }
    exposed[i] = count;
  }
}

extern "C" {

int orc_num_map_types() { return kNumMapTypes; }

void orc_pair(int ti, int tj, double r, double* e, double* dedr) { pair_term(ti, tj, r, kCutoff, e, dedr); }

void orc_constants(double* out) {
  out[0] = kWGauss1, out[1] = kWGauss2, out[2] = kWRepulsion, out[3] = kWHydrophobic, out[4] = kWHBond;
  out[5] = kWRot, out[6] = kCutoff, out[7] = kWallSlope;
}

void orc_grid_dims(const double* size, double h, int* n) { grid_dims(size, h, n); }

// Field at arbitrary points: out[p*4 + c] for point p (receptor sum, Eq. 1).
void orc_receptor_field(int n_rec, const double* rec_xyz, const int* rec_type, int t, int n_pts, const double* pts,
                        double cutoff, double* out) {
  for (int p = 0; p < n_pts; ++p)
    receptor_field(n_rec, rec_xyz, rec_type, t, v3(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]), cutoff,
                   out + 4 * p);
}

// Scale of the receptor sum at points, for tolerances: out[p*2] = sum_j |f|,
// out[p*2 + 1] = sum_j |df/dr| over receptor atoms within the cutoff.
void orc_receptor_field_abs(int n_rec, const double* rec_xyz, const int* rec_type, int t, int n_pts,
                            const double* pts, double cutoff, double* out) {
  for (int p = 0; p < n_pts; ++p) {
    const V3 m = v3(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]);
    double se = 0.0, sg = 0.0;
    for (int j = 0; j < n_rec; ++j) {
      const double r = norm(sub(m, v3(rec_xyz[3 * j], rec_xyz[3 * j + 1], rec_xyz[3 * j + 2])));
      if (!(r < cutoff)) continue;
      double e, dedr;
      pair_term(t, rec_type[j], r, cutoff, &e, &dedr);
      se += std::fabs(e);
      sg += std::fabs(dedr);
    }
    out[2 * p] = se;
    out[2 * p + 1] = sg;
  }
}

// Full maps [K][nz][ny][nx][4]; vertices split over n_threads (same arithmetic per vertex).
void orc_grid_build(int n_rec, const double* rec_xyz, const int* rec_type, const double* center,
                    const double* size, double h, double cutoff, int n_threads, double* maps) {
  int n[3];
  grid_dims(size, h, n);
  double origin[3];
  for (int a = 0; a < 3; ++a) origin[a] = center[a] - (n[a] - 1) * h / 2.0;
  const long total = (long)kNumMapTypes * n[2];
  std::atomic<long> next(0);
  auto work = [&]() {
    for (;;) {
      const long job = next.fetch_add(1);
      if (job >= total) break;
      const int t = (int)(job / n[2]), iz = (int)(job % n[2]);
      for (int iy = 0; iy < n[1]; ++iy)
        for (int ix = 0; ix < n[0]; ++ix) {
          const V3 m = v3(origin[0] + h * ix, origin[1] + h * iy, origin[2] + h * iz);
          double* out = maps + ((((size_t)t * n[2] + iz) * n[1] + iy) * n[0] + ix) * 4;
          receptor_field(n_rec, rec_xyz, rec_type, t, m, cutoff, out);
        }
    }
  };
  if (n_threads < 1) n_threads = 1;
  std::vector<std::thread> th;
  for (int i = 1; i < n_threads; ++i) th.emplace_back(work);
  work();
  for (auto& x : th) x.join();
}

// Interpolate maps at points: e[p], g[3p..3p+2].
void orc_interpolate(const double* maps, const int* n, const double* origin, double h, int mode, int t, int n_pts,
                     const double* pts, double* e, double* g) {
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, h, maps};
  for (int p = 0; p < n_pts; ++p) {
    V3 gv;
    interpolate(G, mode, t, v3(pts[3 * p], pts[3 * p + 1], pts[3 * p + 2]), &e[p], &gv);
    g[3 * p] = gv.x, g[3 * p + 1] = gv.y, g[3 * p + 2] = gv.z;
  }
}

void* orc_ligand_new(int n_atoms, const double* xyz, const int* types, int n_bonds, const int* bonds,
                     const int* rotatable) {
  Ligand* L = new Ligand();
  if (!build_ligand(*L, n_atoms, xyz, types, n_bonds, bonds, rotatable)) {
    delete L;
    return nullptr;
  }
  return L;
}
void orc_ligand_free(void* h) { delete (Ligand*)h; }

// info: [n_atoms, T, n_bodies, root_body, root_origin_atom, n_pairs]
void orc_ligand_info(void* h, int* info, double* gyration_radius) {
  const Ligand& L = *(Ligand*)h;
  info[0] = L.n_atoms, info[1] = L.T, info[2] = L.n_bodies, info[3] = L.root;
  info[4] = L.origin_atom[L.root], info[5] = (int)L.pairs.size();
  *gyration_radius = L.gyration_radius;
}
void orc_ligand_pairs(void* h, int* out) {
  const Ligand& L = *(Ligand*)h;
  for (size_t i = 0; i < L.pairs.size(); ++i) out[2 * i] = L.pairs[i].first, out[2 * i + 1] = L.pairs[i].second;
}
void orc_ligand_bodies(void* h, int* body_of, int* parent, int* torsion_body) {
  const Ligand& L = *(Ligand*)h;
  for (int i = 0; i < L.n_atoms; ++i) body_of[i] = L.body_of[i];
  for (int b = 0; b < L.n_bodies; ++b) parent[b] = L.parent[b];
  for (int k = 0; k < L.T; ++k) torsion_body[k] = L.torsion_body[k];
}

void orc_ligand_coords(void* h, const double* conf, double* xyz) {
  const Ligand& L = *(Ligand*)h;
  Pose P;
  forward_kinematics(L, conf, P);
  for (int i = 0; i < L.n_atoms; ++i) xyz[3 * i] = P.atom[i].x, xyz[3 * i + 1] = P.atom[i].y, xyz[3 * i + 2] = P.atom[i].z;
}

// Score on maps.  terms[0] = inter, terms[1] = intra; grad (6 + T) of the selected terms.
void orc_score_grid(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                    const double* conf, int flags, double* terms, double* grad) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  const Terms t = evaluate(L, &G, mode, nullptr, conf, flags, grad);
  terms[0] = t.inter, terms[1] = t.intra;
}

// Gridless (exact pairwise) score.
void orc_score_exact(void* h, int n_rec, const double* rec_xyz, const int* rec_type, const double* conf, int flags,
                     double* terms, double* grad) {
  const Ligand& L = *(Ligand*)h;
  Receptor R{n_rec, rec_xyz, rec_type};
  const Terms t = evaluate(L, nullptr, 0, &R, conf, flags, grad);
  terms[0] = t.inter, terms[1] = t.intra;
}

void orc_apply_step(void* h, double* conf, const double* s) { apply_step(*(Ligand*)h, conf, s); }

// opt_params: [max_iters, c1, shrink, max_trials, min_curvature, bb_alpha0, bb_alpha_min, bb_alpha_max,
//              step_scale, grad_perturb]
static OptSettings opt_from(const double* p) {
  OptSettings s;
  s.max_iters = (int)p[0];
  s.c1 = p[1];
  s.shrink = p[2];
  s.max_trials = (int)p[3];
  s.min_curvature = p[4];
  s.bb_alpha0 = p[5];
  s.bb_alpha_min = p[6];
  s.bb_alpha_max = p[7];
  s.step_scale = p[8];
  s.grad_perturb = p[9];
  return s;
}

// Local optimisation of a docking conformation on maps (optimizer 0 BFGS, 1 BB).
// out: [E, evals, iters]
void orc_local_opt(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                   int optimizer, const double* opt_params, double* conf, double* out) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  DockObjective obj(&L, &G, mode);
  const OptSettings st = opt_from(opt_params);
  const OptResult r = optimizer == 0 ? bfgs(obj, conf, st) : barzilai_borwein(obj, conf, st);
  out[0] = r.e, out[1] = (double)r.evals, out[2] = r.iters;
}

// Copies a decision log into [cap][3] rows (kind, margin, scale); returns the
// number of decisions taken (rows beyond cap are dropped).
static int copy_log(const std::vector<Decision>& log, double* out, int cap) {
  for (int i = 0; i < (int)log.size() && i < cap; ++i)
    out[3 * i] = log[i].kind, out[3 * i + 1] = log[i].margin, out[3 * i + 2] = log[i].scale;
  return (int)log.size();
}

// orc_local_opt with the decisions it takes (see Decision); *n_log = their count.
void orc_local_opt_log(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                       int optimizer, const double* opt_params, double* conf, double* out, double* log_out,
                       int log_cap, int* n_log) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  DockObjective obj(&L, &G, mode);
  OptSettings st = opt_from(opt_params);
  std::vector<Decision> log;
  st.log = &log;
  obj.log = &log;
  const OptResult r = optimizer == 0 ? bfgs(obj, conf, st) : barzilai_borwein(obj, conf, st);
  out[0] = r.e, out[1] = (double)r.evals, out[2] = r.iters;
  *n_log = copy_log(log, log_out, log_cap);
}

// Optimisers on test objectives.  kind 0: quadratic 0.5 x^T A x - b^T x; kind 1: Rosenbrock.
// orc_opt_test_log also returns the decisions taken (see Decision).
void orc_opt_test_log(int kind, int optimizer, int n, const double* A, const double* b, const double* opt_params,
                      double* x, double* out, double* log_out, int log_cap, int* n_log);
void orc_opt_test(int kind, int optimizer, int n, const double* A, const double* b, const double* opt_params,
                  double* x, double* out) {
  int n_log = 0;
  orc_opt_test_log(kind, optimizer, n, A, b, opt_params, x, out, nullptr, 0, &n_log);
}

void orc_opt_test_log(int kind, int optimizer, int n, const double* A, const double* b, const double* opt_params,
                      double* x, double* out, double* log_out, int log_cap, int* n_log) {
  OptSettings st = opt_from(opt_params);
  std::vector<Decision> log;
  st.log = &log;
  OptResult r;
  if (kind == 0) {
    QuadObjective q(n, A, b);
    r = optimizer == 0 ? bfgs(q, x, st) : barzilai_borwein(q, x, st);
  } else {
    RosenObjective q(n);
    r = optimizer == 0 ? bfgs(q, x, st) : barzilai_borwein(q, x, st);
  }
  out[0] = r.e, out[1] = (double)r.evals, out[2] = r.iters;
  *n_log = copy_log(log, log_out, log_cap);
}

void orc_bfgs_update(int n, double* H, const double* s, const double* y) {
  std::vector<double> h(H, H + n * n);
  bfgs_update(n, h, s, y);
  for (int i = 0; i < n * n; ++i) H[i] = h[i];
}

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

void orc_unit_ball(uint64_t seed, uint32_t chain, uint32_t step, double* out) {
  ChainRng rng{{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}, chain};
  const V3 b = unit_ball(rng, step);
  out[0] = b.x, out[1] = b.y, out[2] = b.z;
}

// dock_params: [n_mc_steps, optimizer, temperature, box_lo x3, box_size x3,
//               site_radius, n_sites, sites x 3 n_sites]
static DockSettings dock_from(const double* dp, const double* op) {
  DockSettings ds;
  ds.n_mc_steps = (int)dp[0];
  ds.optimizer = (int)dp[1];
  ds.temperature = dp[2];
  for (int a = 0; a < 3; ++a) ds.box_lo[a] = dp[3 + a], ds.box_size[a] = dp[6 + a];
  ds.site_radius = dp[9];
  ds.n_sites = (int)dp[10];
  ds.sites = ds.n_sites > 0 ? dp + 11 : nullptr;
  ds.opt = opt_from(op);
  return ds;
}

void orc_chain_init(void* h, const double* dock_params, const double* opt_params, uint64_t seed, uint32_t chain,
                    double* conf) {
  const Ligand& L = *(Ligand*)h;
  const DockSettings ds = dock_from(dock_params, opt_params);
  ChainRng rng{{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}, chain};
  chain_init(L, rng, ds, conf);
}

// Whole chain.  best (7+T), out: [e_best, evals]; optional trace_conf
// ((S+1) x (7+T), the current state after each step) and trace_rec
// ((S+1) x 5: mode, accepted, e_candidate, e_current, evals).
void orc_run_chain(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                   const double* dock_params, const double* opt_params, uint64_t seed, uint32_t chain, double* best,
                   double* out, double* trace_conf, double* trace_rec) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  const DockSettings ds = dock_from(dock_params, opt_params);
  std::vector<StepRecord> tr(ds.n_mc_steps + 1);
  double eb;
  const long evals = run_chain(L, G, mode, ds, seed, chain, best, &eb, trace_conf, trace_rec ? tr.data() : nullptr);
  out[0] = eb, out[1] = (double)evals;
  if (trace_rec)
    for (int s = 0; s <= ds.n_mc_steps; ++s) {
      trace_rec[5 * s + 0] = tr[s].mode, trace_rec[5 * s + 1] = tr[s].accepted;
      trace_rec[5 * s + 2] = tr[s].e_candidate, trace_rec[5 * s + 3] = tr[s].e_current;
      trace_rec[5 * s + 4] = (double)tr[s].evals;
    }
}

// One MC step (replay): cur/e_cur in, updated in place; rec out (5 values as above).
// best/e_best are not tracked here.
void orc_mc_step(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                 const double* dock_params, const double* opt_params, uint64_t seed, uint32_t chain, uint32_t step,
                 double* cur, double* e_cur, double* rec_out) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  const DockSettings ds = dock_from(dock_params, opt_params);
  DockObjective obj(&L, &G, mode);
  ChainRng rng{{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}, chain};
  std::vector<double> best(7 + L.T);
  double e_best = -1e300;  // never improved: best is not tracked in a replay
  const StepRecord r = mc_step(L, obj, rng, ds, step, cur, e_cur, best.data(), &e_best);
  rec_out[0] = r.mode, rec_out[1] = r.accepted, rec_out[2] = r.e_candidate, rec_out[3] = r.e_current;
  rec_out[4] = (double)r.evals;
}

// orc_mc_step with the decisions it takes (local optimisation, then Metropolis).
void orc_mc_step_log(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
                     const double* dock_params, const double* opt_params, uint64_t seed, uint32_t chain,
                     uint32_t step, double* cur, double* e_cur, double* rec_out, double* log_out, int log_cap,
                     int* n_log) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  DockSettings ds = dock_from(dock_params, opt_params);
  std::vector<Decision> log;
  ds.opt.log = &log;
  DockObjective obj(&L, &G, mode);
  obj.log = &log;
  ChainRng rng{{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}, chain};
  std::vector<double> best(7 + L.T);
  double e_best = -1e300;
  const StepRecord r = mc_step(L, obj, rng, ds, step, cur, e_cur, best.data(), &e_best);
  rec_out[0] = r.mode, rec_out[1] = r.accepted, rec_out[2] = r.e_candidate, rec_out[3] = r.e_current;
  rec_out[4] = (double)r.evals;
  *n_log = copy_log(log, log_out, log_cap);
}


// A whole docking job: chains [chain0, chain0 + n_chains) split over n_threads.
// best (n_chains x (7+T)), e_best (n_chains), evals (n_chains).
void orc_dock(void* h, const double* maps, const int* n, const double* origin, double hh, int mode,
              const double* dock_params, const double* opt_params, uint64_t seed, int chain0, int n_chains,
              int n_threads, double* best, double* e_best, double* evals) {
  const Ligand& L = *(Ligand*)h;
  Grid G{{n[0], n[1], n[2]}, {origin[0], origin[1], origin[2]}, hh, maps};
  const DockSettings ds = dock_from(dock_params, opt_params);
  const int nx = 7 + L.T;
  std::atomic<int> next(0);
  auto work = [&]() {
    for (;;) {
      const int c = next.fetch_add(1);
      if (c >= n_chains) break;
      evals[c] = (double)run_chain(L, G, mode, ds, seed, (uint32_t)(chain0 + c), best + (size_t)c * nx, &e_best[c],
                                   nullptr, nullptr);
    }
  };
  if (n_threads < 1) n_threads = 1;
  std::vector<std::thread> th;
  for (int i = 1; i < n_threads; ++i) th.emplace_back(work);
  work();
  for (auto& x : th) x.join();
}

// FP64 gridless rescoring + RMSD de-duplication + top-k (Fig. 4 postprocess).
// For each pose: exact inter and intra; score = inter / (1 + w_rot T).
// Sorted by score ascending, ties by lower pose index; a pose within
// rmsd_cut of an already kept pose is dropped; at most k kept.
// scores_all (n) receives every pose's score; out_idx (k) the kept pose
// indices, out_terms (k x 3) [score, inter, intra]; returns the number kept.
int orc_rescore_topk(void* h, int n_rec, const double* rec_xyz, const int* rec_type, int n_poses,
                     const double* confs, int k, double rmsd_cut, double* scores_all, int* out_idx,
                     double* out_terms) {
  const Ligand& L = *(Ligand*)h;
  Receptor R{n_rec, rec_xyz, rec_type};
  const int nx = 7 + L.T;
  std::vector<Terms> terms(n_poses);
  std::vector<Pose> poses(n_poses);
  for (int p = 0; p < n_poses; ++p) {
    terms[p] = evaluate(L, nullptr, 0, &R, confs + (size_t)p * nx, 3, nullptr, &poses[p]);
    scores_all[p] = terms[p].inter / (1.0 + kWRot * L.T);
  }
  std::vector<int> idx(n_poses);
  for (int p = 0; p < n_poses; ++p) idx[p] = p;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return scores_all[a] < scores_all[b]; });
  int kept = 0;
  for (int p : idx) {
    if (kept >= k) break;
    bool dup = false;
    for (int q = 0; q < kept; ++q)
      if (rmsd(poses[p].atom, poses[out_idx[q]].atom) < rmsd_cut) {
        dup = true;
        break;
      }
    if (dup) continue;
    out_idx[kept] = p;
    out_terms[3 * kept] = scores_all[p], out_terms[3 * kept + 1] = terms[p].inter;
    out_terms[3 * kept + 2] = terms[p].intra;
    ++kept;
  }
  return kept;
}


int orc_sas_directions(float* u) { return sas_directions(u); }

// Exposed test points per atom (see the voxel features section).
void orc_sas_exposed(int n, const float* xyz, const float* radius, int* exposed) {
  sas_exposed(n, xyz, radius, exposed);
}

// Voxel features: out [36][36][36][18] (z, y, x, channel); features [n][17];
// center: the cube's centre (the lower corner c - 35 is taken in FP64, then
// rounded to FP32).  Returns the number of atoms inside the cube.
int orc_voxelize(int n, const float* xyz, const float* radius, const float* features, const double* center,
                 float* out) {
  std::vector<int> exposed(n);
  sas_exposed(n, xyz, radius, exposed.data());
  float lo[3];
  for (int a = 0; a < 3; ++a) lo[a] = (float)(center[a] - 35.0);
  const float inv = 36.0f / 70.0f;
  std::vector<int64_t> acc((size_t)kVoxN * kVoxN * kVoxN * kVoxChannels, 0);
  int inside = 0;
  for (int i = 0; i < n; ++i) {
    int k[3];
    bool in = true;
    for (int a = 0; a < 3; ++a) {
      const float u = (xyz[3 * i + a] - lo[a]) * inv;
      k[a] = (int)std::floor(u);
      in = in && k[a] >= 0 && k[a] < kVoxN;
    }
    if (!in) continue;
    ++inside;
    int64_t* v = &acc[(((size_t)k[2] * kVoxN + k[1]) * kVoxN + k[0]) * kVoxChannels];
    for (int c = 0; c < kVoxFeatures; ++c) v[c] += std::llrint((double)features[(size_t)kVoxFeatures * i + c] * 16777216.0);
    v[kVoxFeatures] += (exposed[i] > 0 ? 1 : 0) * (int64_t)16777216;
  }
  for (size_t q = 0; q < acc.size(); ++q) out[q] = (float)((double)acc[q] * (1.0 / 16777216.0));
  return inside;
}

}  // extern "C"
