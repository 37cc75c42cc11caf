// Ligand preparation on the host (the paper prepares the copies on the CPU,
// Sec. 2 / Fig. 4): rigid bodies, torsion tree, internal atom order, intra
// pair list, packed into one position-independent blob the kernels read.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dsdp_internal.h"

namespace dsdp {

static thread_local char g_last_error[512] = "";

dsdp_status set_error(dsdp_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return s;
}

const char* last_error() { return g_last_error; }

namespace {

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Prepared {
  int n = 0, T = 0, B = 0, P = 0, rounds = 0, root_atom = 0;
  int hyd_begin = 0, hb_begin = 0;  // class boundaries of the grouped pair list
  float gyr = 1.0f;
  std::vector<int> user_of;         // internal -> input index
  std::vector<float> local;         // [n][3]
  std::vector<double> local64;      // [n][3]
  std::vector<double> body64;       // [B][6]: offset, axis
  std::vector<int> type, body;      // per internal atom
  std::vector<BodyRec> bodies;      // DFS pre-order
  std::vector<uint32_t> pairs;      // i | j << 8 | (type_i * 8 + type_j) << 16
  std::vector<uint32_t> steps;       // [n_steps][32][2] step table (see kStepIdleNrs)
  int n_steps = 0;
  std::vector<int16_t> lane_map;     // [32][2] internal atom in slot s of lane l, -1 empty
  std::vector<int> torsion_body;
  float root_ref[3];
};

// Intra-pair step schedule.  Each pair is computed by one lane (its "active"
// atom) against an atom of a partner lane ("passive"), which receives the
// reaction force by a shuffle.  A step may give each lane at most one active
// and one passive role, so the pairs form a bipartite multigraph between lanes
// as active and lanes as passive.  Its edges are oriented first so that every
// lane is active about as often as it is passive (Euler circuits through an
// extra vertex joined to the lanes of odd degree: |out - in| <= 1), then
// coloured with max(out, in) colours by alternating-path recolouring (Konig's
// edge-colouring theorem for bipartite multigraphs); a colour is a step.
// Atoms to lanes.  Up to 32 atoms: atom i in lane i.  Above (two slots per
// lane), the lane's pair count bounds the schedule (half of the busiest lane's
// pairs), so the 64 - n atoms with the most intra pairs get a lane of their own
// and the others share lanes two by two, the one with the most pairs left with
// the one with the fewest (ties by atom index); slot 0 holds the first.
void assign_lanes(int n, const std::vector<int>& pi, const std::vector<int>& pj, std::vector<int16_t>& lane_map,
                  std::vector<int>& lane_of, std::vector<int>& slot_of) {
  lane_map.assign(64, (int16_t)-1);
  lane_of.assign(n, 0);
  slot_of.assign(n, 0);
  if (atoms_per_lane(n) == 1) {
    for (int a = 0; a < n; ++a) lane_map[2 * a] = (int16_t)a, lane_of[a] = a;
    return;
  }
  std::vector<int> deg(n, 0), order(n);
  for (size_t p = 0; p < pi.size(); ++p) ++deg[pi[p]], ++deg[pj[p]];
  for (int a = 0; a < n; ++a) order[a] = a;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg[a] > deg[b]; });
  const int singles = 64 - n;
  int lane = 0;
  for (int k = 0; k < singles; ++k, ++lane) lane_map[2 * lane] = (int16_t)order[k];
  for (int lo = singles, hi = n - 1; lo < hi; ++lo, --hi, ++lane) {
    lane_map[2 * lane] = (int16_t)order[lo];
    lane_map[2 * lane + 1] = (int16_t)order[hi];
  }
  for (int l = 0; l < 32; ++l)
    for (int s = 0; s < 2; ++s)
      if (lane_map[2 * l + s] >= 0) lane_of[lane_map[2 * l + s]] = l, slot_of[lane_map[2 * l + s]] = s;
}

void build_pair_steps(int n, const std::vector<int>& pi, const std::vector<int>& pj, const std::vector<int>& pc,
                      const std::vector<float>& pn, const std::vector<int>& lane_of_atom,
                      const std::vector<int>& slot_of_atom, std::vector<uint32_t>& table, int& n_steps) {
  const int P = (int)pi.size(), V = 32, X = 32;  // X: the extra vertex
  auto lane_of = [&](int a) { return lane_of_atom[a]; };
  // ---- orientation: act[p] = the active atom of pair p
  std::vector<int> act(P, -1);
  {
    struct E {
      int u, v, pair;  // pair < 0: edge to the extra vertex
    };
    std::vector<E> edges;
    std::vector<int> deg(V + 1, 0);
    for (int p = 0; p < P; ++p) {
      const int u = lane_of(pi[p]), v = lane_of(pj[p]);
      if (u == v) {
        act[p] = pi[p];  // both atoms in one lane: the lane is active and passive once
        continue;
      }
      edges.push_back(E{u, v, p});
      ++deg[u];
      ++deg[v];
    }
    for (int v = 0; v < V; ++v)
      if (deg[v] & 1) edges.push_back(E{v, X, -1});
    std::vector<std::vector<int>> inc(V + 1);
    for (int e = 0; e < (int)edges.size(); ++e) {
      inc[edges[e].u].push_back(e);
      inc[edges[e].v].push_back(e);
    }
    std::vector<char> used(edges.size(), 0);
    std::vector<size_t> next(V + 1, 0);
    for (int s0 = 0; s0 <= V; ++s0) {
      std::vector<int> stack{s0};
      while (!stack.empty()) {
        const int x = stack.back();
        while (next[x] < inc[x].size() && used[inc[x][next[x]]]) ++next[x];
        if (next[x] == inc[x].size()) {
          stack.pop_back();
          continue;
        }
        const int e = inc[x][next[x]];
        used[e] = 1;
        const int y = edges[e].u == x ? edges[e].v : edges[e].u;
        const int p = edges[e].pair;
        if (p >= 0) act[p] = lane_of(pi[p]) == x ? pi[p] : pj[p];  // walked x -> y: x's atom is active
        stack.push_back(y);
      }
    }
  }
  // ---- colouring
  int delta = 0;
  {
    std::vector<int> out_d(V, 0), in_d(V, 0);
    for (int p = 0; p < P; ++p) {
      const int a = act[p], b = a == pi[p] ? pj[p] : pi[p];
      ++out_d[lane_of(a)];
      ++in_d[lane_of(b)];
    }
    for (int v = 0; v < V; ++v) delta = std::max(delta, std::max(out_d[v], in_d[v]));
  }
  std::vector<int> colour(P, -1);
  std::vector<int> at_act((size_t)V * std::max(delta, 1), -1), at_pas((size_t)V * std::max(delta, 1), -1);
  auto A = [&](int lane, int c) -> int& { return at_act[(size_t)lane * delta + c]; };
  auto B = [&](int lane, int c) -> int& { return at_pas[(size_t)lane * delta + c]; };
  auto ends = [&](int p, int& u, int& v) {
    const int a = act[p], b = a == pi[p] ? pj[p] : pi[p];
    u = lane_of(a);
    v = lane_of(b);
  };
  // Pairs with a hydrophobic or H-bond term ("ramp" pairs) are coloured first,
  // from the top of the palette, the others from the bottom: the ramp pairs then
  // gather in a few steps, and the kernels skip those terms in the other steps.
  std::vector<int> order;
  for (int p = 0; p < P; ++p)
    if (pc[p] != 0) order.push_back(p);
  const size_t n_ramp = order.size();
  for (int p = 0; p < P; ++p)
    if (pc[p] == 0) order.push_back(p);
  for (size_t oi = 0; oi < order.size(); ++oi) {
    const int p = order[oi];
    int u, v;
    ends(p, u, v);
    int c1, c2;
    if (oi < n_ramp) {
      c1 = c2 = delta - 1;
      while (A(u, c1) >= 0) --c1;
      while (B(v, c2) >= 0) --c2;
    } else {
      c1 = c2 = 0;
      while (A(u, c1) >= 0) ++c1;
      while (B(v, c2) >= 0) ++c2;
    }
    if (B(v, c1) >= 0) {
      // swap c1 / c2 along the path from v (passive side) that starts with colour c1
      std::vector<int> path;
      int x = v, col = c1;
      bool passive_side = true;
      for (;;) {
        const int q = passive_side ? B(x, col) : A(x, col);
        if (q < 0) break;
        path.push_back(q);
        int qu, qv;
        ends(q, qu, qv);
        x = passive_side ? qu : qv;
        passive_side = !passive_side;
        col = col == c1 ? c2 : c1;
      }
      for (int q : path) {
        int qu, qv;
        ends(q, qu, qv);
        A(qu, colour[q]) = -1;
        B(qv, colour[q]) = -1;
      }
      for (int q : path) {
        int qu, qv;
        ends(q, qu, qv);
        colour[q] = colour[q] == c1 ? c2 : c1;
        A(qu, colour[q]) = q;
        B(qv, colour[q]) = q;
      }
    }
    colour[p] = c1;
    A(u, c1) = p;
    B(v, c1) = p;
  }
  // ---- table: steps holding ramp pairs first (they are processed two at a time)
  std::vector<int> col_order;
  for (int pass = 0; pass < 2; ++pass)
    for (int c = delta - 1; c >= 0; --c) {
      bool ramp = false;
      for (int v = 0; v < V; ++v) ramp |= A(v, c) >= 0 && pc[A(v, c)] != 0;
      if (ramp == (pass == 0)) col_order.push_back(c);
    }
  n_steps = (delta + 1) & ~1;
  table.assign((size_t)n_steps * V * 2, 0u);
  for (int st = 0; st < n_steps; ++st) {
    const int c = st < delta ? col_order[st] : delta;  // delta: the empty padding step
    uint32_t step_bits = 0;
    int idle = -1;
    for (int v = 0; v < V && c < delta; ++v) {
      if (A(v, c) < 0 && idle < 0) idle = v;
      if (A(v, c) >= 0) step_bits |= (pc[A(v, c)] == 1 ? 1u << 14 : 0u) | (pc[A(v, c)] == 2 ? 1u << 15 : 0u);
    }
    for (int v = 0; v < V; ++v) {
      uint32_t x = (uint32_t)v | ((uint32_t)(idle >= 0 ? idle : v) << 5);
      float nrs = kStepIdleNrs;
      if (c < delta && A(v, c) >= 0) {
        const int p = A(v, c), a = act[p], b = a == pi[p] ? pj[p] : pi[p];
        x = (x & ~31u) | (uint32_t)lane_of(b);
        x |= (uint32_t)slot_of_atom[a] << 10;
        x |= pc[p] == 1 ? 1u << 12 : 0u;
        x |= pc[p] == 2 ? 1u << 13 : 0u;
        nrs = pn[p];
      }
      if (c < delta && B(v, c) >= 0) {
        const int p = B(v, c), a = act[p], b = a == pi[p] ? pj[p] : pi[p];
        x = (x & ~(31u << 5)) | ((uint32_t)lane_of(a) << 5);
        x |= (uint32_t)slot_of_atom[b] << 11;
      }
      x |= step_bits;
      table[((size_t)st * V + v) * 2] = x;
      memcpy(&table[((size_t)st * V + v) * 2 + 1], &nrs, 4);
    }
  }
}

dsdp_status prepare(const dsdp_ligand* L, Prepared& out) {
  if (!L) return set_error(DSDP_ERR_INVALID_ARG, "ligand is NULL");
  const int n = L->n_atoms;
  if (n < 1 || n > kMaxAtoms) return set_error(DSDP_ERR_INVALID_ARG, "ligand n_atoms %d outside 1..%d", n, kMaxAtoms);
  if (!L->xyz || !L->xs_type) return set_error(DSDP_ERR_INVALID_ARG, "ligand xyz/xs_type NULL");
  if (L->n_bonds < 0 || (L->n_bonds > 0 && (!L->bonds || !L->rotatable)))
    return set_error(DSDP_ERR_INVALID_ARG, "ligand bonds/rotatable NULL");
  for (int i = 0; i < n; ++i) {
    if (L->xs_type[i] >= DSDP_NUM_MAP_TYPES)
      return set_error(DSDP_ERR_INVALID_ARG, "ligand atom %d has type %d; ligands use map types 0..7", i,
                       (int)L->xs_type[i]);
    for (int a = 0; a < 3; ++a)
      if (!isfinite(L->xyz[3 * i + a])) return set_error(DSDP_ERR_INVALID_ARG, "ligand atom %d not finite", i);
  }
  std::vector<std::vector<int>> adj(n), rigid(n);
  std::vector<int> rot_bonds;
  for (int b = 0; b < L->n_bonds; ++b) {
    const int i = L->bonds[2 * b], j = L->bonds[2 * b + 1];
    if (i < 0 || j < 0 || i >= n || j >= n || i == j)
      return set_error(DSDP_ERR_INVALID_ARG, "bond %d (%d, %d) invalid", b, i, j);
    adj[i].push_back(j);
    adj[j].push_back(i);
    if (L->rotatable[b]) rot_bonds.push_back(b);
    else {
      rigid[i].push_back(j);
      rigid[j].push_back(i);
    }
  }
  const int T = (int)rot_bonds.size();
  if (T > DSDP_MAX_TORSIONS) return set_error(DSDP_ERR_INVALID_ARG, "%d rotatable bonds > %d", T, DSDP_MAX_TORSIONS);
  // bodies numbered by their lowest atom
  std::vector<int> comp(n, -1);
  int B = 0;
  for (int s = 0; s < n; ++s) {
    if (comp[s] >= 0) continue;
    std::vector<int> st{s};
    comp[s] = B;
    while (!st.empty()) {
      const int a = st.back();
      st.pop_back();
      for (int c : rigid[a])
        if (comp[c] < 0) comp[c] = B, st.push_back(c);
    }
    ++B;
  }
  if (B != T + 1)
    return set_error(DSDP_ERR_INVALID_ARG,
                     "ligand must be one molecule whose rotatable bonds each split it (bodies %d, torsions %d)", B, T);
  for (int k = 0; k < T; ++k) {
    const int b = rot_bonds[k];
    if (comp[L->bonds[2 * b]] == comp[L->bonds[2 * b + 1]])
      return set_error(DSDP_ERR_INVALID_ARG, "rotatable bond %d lies in a ring", b);
  }
  std::vector<int> count(B, 0);
  for (int i = 0; i < n; ++i) ++count[comp[i]];
  int root = 0;
  for (int b = 1; b < B; ++b)
    if (count[b] > count[root]) root = b;
  // body tree by BFS from the root
  std::vector<int> parent(B, -2), origin(B, -1), near_atom(B, -1), tors(B, -1), depth(B, 0);
  std::vector<std::vector<int>> children(B);
  parent[root] = -1;
  for (int i = 0; i < n; ++i)
    if (comp[i] == root) {
      origin[root] = i;
      break;
    }
  std::vector<int> queue{root};
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    const int b = queue[qi];
    for (int k = 0; k < T; ++k) {
      const int i = L->bonds[2 * rot_bonds[k]], j = L->bonds[2 * rot_bonds[k] + 1];
      int nr = -1, fr = -1;
      if (comp[i] == b) nr = i, fr = j;
      else if (comp[j] == b) nr = j, fr = i;
      if (nr < 0) continue;
      const int c = comp[fr];
      if (parent[c] != -2) continue;
      parent[c] = b;
      origin[c] = fr;
      near_atom[c] = nr;
      tors[c] = k;
      depth[c] = depth[b] + 1;
      children[b].push_back(c);
      queue.push_back(c);
    }
  }
  if ((int)queue.size() != B) return set_error(DSDP_ERR_INVALID_ARG, "ligand is not connected");
  for (auto& ch : children) std::sort(ch.begin(), ch.end(), [&](int a, int b) { return tors[a] < tors[b]; });
  // DFS pre-order of bodies
  std::vector<int> dfs;
  std::vector<int> st{root};
  while (!st.empty()) {
    const int b = st.back();
    st.pop_back();
    dfs.push_back(b);
    for (int c = (int)children[b].size() - 1; c >= 0; --c) st.push_back(children[b][c]);
  }
  std::vector<int> new_body(B);
  for (int i = 0; i < B; ++i) new_body[dfs[i]] = i;
  // internal atom order
  out.user_of.clear();
  std::vector<int> body_first(B), internal_of(n);
  for (int bi = 0; bi < B; ++bi) {
    body_first[bi] = (int)out.user_of.size();
    for (int i = 0; i < n; ++i)
      if (comp[i] == dfs[bi]) {
        internal_of[i] = (int)out.user_of.size();
        out.user_of.push_back(i);
      }
  }
  // subtree end = begin of the next body in pre-order that is not a descendant
  std::vector<int> subtree_end(B, n);
  for (int bi = 0; bi < B; ++bi) {
    for (int bj = bi + 1; bj < B; ++bj) {
      // bj is a descendant of bi iff bi is on bj's ancestor chain
      int a = dfs[bj];
      bool desc = false;
      while (a >= 0) {
        if (a == dfs[bi]) {
          desc = true;
          break;
        }
        a = parent[a];
      }
      if (!desc) {
        subtree_end[bi] = body_first[bj];
        break;
      }
    }
  }
  auto ref = [&](int i, int a) { return (double)L->xyz[3 * i + a]; };
  out.bodies.assign(B, BodyRec{});
  out.body64.assign(6 * (size_t)B, 0.0);
  int max_depth = 0;
  for (int bi = 0; bi < B; ++bi) {
    const int b = dfs[bi];
    BodyRec& r = out.bodies[bi];
    r.parent = parent[b] < 0 ? -1 : new_body[parent[b]];
    r.torsion = tors[b];
    r.atom_begin = body_first[bi];
    r.atom_end = subtree_end[bi];
    r.depth = depth[b];
    max_depth = std::max(max_depth, depth[b]);
    if (parent[b] >= 0) {
      double ax[3], len = 0.0;
      for (int a = 0; a < 3; ++a) {
        r.off[a] = (float)(ref(origin[b], a) - ref(origin[parent[b]], a));
        ax[a] = ref(origin[b], a) - ref(near_atom[b], a);
        len += ax[a] * ax[a];
      }
      len = sqrt(len);
      if (!(len > 1e-6)) return set_error(DSDP_ERR_INVALID_ARG, "rotatable bond %d has zero length", rot_bonds[tors[b]]);
      for (int a = 0; a < 3; ++a) {
        r.axis[a] = (float)(ax[a] / len);
        out.body64[6 * bi + a] = ref(origin[b], a) - ref(origin[parent[b]], a);
        out.body64[6 * bi + 3 + a] = ax[a] / len;
      }
    }
  }
  out.rounds = 0;
  while ((1 << out.rounds) < max_depth + 1) ++out.rounds;
  out.torsion_body.assign(T, 0);
  for (int bi = 0; bi < B; ++bi)
    if (out.bodies[bi].torsion >= 0) out.torsion_body[out.bodies[bi].torsion] = bi;
  // atoms
  out.local.assign(3 * n, 0.0f);
  out.local64.assign(3 * n, 0.0);
  out.type.assign(n, 0);
  out.body.assign(n, 0);
  for (int ii = 0; ii < n; ++ii) {
    const int i = out.user_of[ii];
    const int b = comp[i];
    out.type[ii] = L->xs_type[i];
    out.body[ii] = new_body[b];
    for (int a = 0; a < 3; ++a) {
      out.local64[3 * ii + a] = ref(i, a) - ref(origin[b], a);
      out.local[3 * ii + a] = (float)out.local64[3 * ii + a];
    }
  }
  // pairs: different bodies and more than three bonds apart (internal indices)
  std::vector<int> dist(n);
  out.pairs.clear();
  std::vector<std::vector<int>> topo(n, std::vector<int>(n, 1 << 20));
  for (int i = 0; i < n; ++i) {
    std::fill(dist.begin(), dist.end(), -1);
    std::vector<int> q{i};
    dist[i] = 0;
    for (size_t qi = 0; qi < q.size(); ++qi)
      for (int c : adj[q[qi]])
        if (dist[c] < 0) dist[c] = dist[q[qi]] + 1, q.push_back(c);
    for (int j = 0; j < n; ++j) topo[i][j] = dist[j] < 0 ? (1 << 20) : dist[j];
  }
  // Pairs grouped by which optional terms they carry (none, hydrophobic, H-bond),
  // each group in (i, j) order: a warp taking 32 consecutive pairs then mostly
  // sees one group and can skip the terms none of its pairs has.
  {
    static const int xs_bits[8] = {1, 0, 0, 2, 4, 4, 6, 0};  // 1 hydrophobic, 2 donor, 4 acceptor
    std::vector<uint32_t> by_class[4];
    for (int ii = 0; ii < n; ++ii)
      for (int jj = ii + 1; jj < n; ++jj) {
        const int i = out.user_of[ii], j = out.user_of[jj];
        if (comp[i] == comp[j] || topo[i][j] <= 3) continue;
        const int a = xs_bits[out.type[ii]], b = xs_bits[out.type[jj]];
        const int cls = (a & b & 1) | ((((a & 2) && (b & 4)) || ((a & 4) && (b & 2))) ? 2 : 0);
        by_class[cls].push_back((uint32_t)ii | ((uint32_t)jj << 8) |
                                ((uint32_t)(out.type[ii] * DSDP_NUM_MAP_TYPES + out.type[jj]) << 16));
      }
    // a pair is never both (hydrophobic atoms are neither donors nor acceptors)
    if (!by_class[3].empty()) return set_error(DSDP_ERR_INTERNAL, "pair with both optional terms");
    out.pairs.clear();
    for (int c = 0; c < 3; ++c) out.pairs.insert(out.pairs.end(), by_class[c].begin(), by_class[c].end());
    out.hyd_begin = (int)by_class[0].size();
    out.hb_begin = out.hyd_begin + (int)by_class[1].size();
  }
  const int P = (int)out.pairs.size();
  {
    static const double radius[8] = {1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0};
    std::vector<int> pi(P), pj(P), pc(P);
    std::vector<float> pn(P);
    for (int p = 0; p < P; ++p) {
      pi[p] = out.pairs[p] & 0xff;
      pj[p] = (out.pairs[p] >> 8) & 0xff;
      pc[p] = p < out.hyd_begin ? 0 : (p < out.hb_begin ? 1 : 2);
      const int tp = out.pairs[p] >> 16;
      pn[p] = (float)-(radius[tp / DSDP_NUM_MAP_TYPES] + radius[tp % DSDP_NUM_MAP_TYPES]);
    }
    std::vector<int> lane_of, slot_of;
    assign_lanes(n, pi, pj, out.lane_map, lane_of, slot_of);
    build_pair_steps(n, pi, pj, pc, pn, lane_of, slot_of, out.steps, out.n_steps);
  }
  double s2 = 0.0;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      const double d = ref(i, a) - ref(origin[root], a);
      s2 += d * d;
    }
  out.gyr = (float)sqrt(s2 / n);
  if (!(out.gyr > 1e-3f)) out.gyr = 1.0f;
  out.n = n;
  out.T = T;
  out.B = B;
  out.P = P;
  out.root_atom = origin[root];
  for (int a = 0; a < 3; ++a) out.root_ref[a] = L->xyz[3 * origin[root] + a];
  return DSDP_OK;
}

}  // namespace
}  // namespace dsdp

using namespace dsdp;

extern "C" dsdp_status dsdp_ligand_pack(const dsdp_ligand* ligand, void* blob, uint64_t capacity,
                                        uint64_t* blob_bytes) {
  Prepared p;
  const dsdp_status s = prepare(ligand, p);
  if (s != DSDP_OK) return s;
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  size_t off = sizeof(BlobHeader);
  h.off_atom = (uint32_t)off;
  off = align16(off + 16 * (size_t)p.n);
  h.off_atom_user = (uint32_t)off;
  off = align16(off + 4 * (size_t)p.n);
  h.off_body = (uint32_t)off;
  off = align16(off + sizeof(BodyRec) * (size_t)p.B);
  h.off_torsion_body = (uint32_t)off;
  off = align16(off + 4 * (size_t)p.T);
  h.off_steps = (uint32_t)off;
  off = align16(off + 8 * 32 * (size_t)p.n_steps);
  h.off_lane_map = (uint32_t)off;
  off = align16(off + 2 * 64);
  h.stage_bytes = (uint32_t)off;  // the chain kernels stage only this prefix
  h.off_pairs = (uint32_t)off;
  off = align16(off + 8 * (size_t)p.P);
  h.off_atom64 = (uint32_t)off;
  off = align16(off + 8 * 3 * (size_t)p.n);
  h.off_body64 = (uint32_t)off;
  off = align16(off + 8 * 6 * (size_t)p.B);
  h.magic = kBlobMagic;
  h.bytes = (uint32_t)off;
  h.n_atoms = p.n;
  h.n_torsions = p.T;
  h.n_bodies = p.B;
  h.n_pairs = p.P;
  h.n_steps = p.n_steps;
  h.pair_hyd_begin = p.hyd_begin;
  h.pair_hb_begin = p.hb_begin;
  h.rounds = p.rounds;
  h.gyration_radius = p.gyr;
  for (int a = 0; a < 3; ++a) h.root_ref[a] = p.root_ref[a];
  h.root_user_atom = p.root_atom;
  if (blob_bytes) *blob_bytes = off;
  if (!blob) return DSDP_OK;
  if (capacity < off) return set_error(DSDP_ERR_INVALID_ARG, "blob capacity %llu < %llu bytes",
                                       (unsigned long long)capacity, (unsigned long long)off);
  uint8_t* b = (uint8_t*)blob;
  memset(b, 0, off);
  memcpy(b, &h, sizeof(h));
  float* atoms = (float*)(b + h.off_atom);
  for (int i = 0; i < p.n; ++i) {
    atoms[4 * i + 0] = p.local[3 * i + 0];
    atoms[4 * i + 1] = p.local[3 * i + 1];
    atoms[4 * i + 2] = p.local[3 * i + 2];
    const int32_t packed = p.type[i] | (p.body[i] << 8);
    memcpy(&atoms[4 * i + 3], &packed, 4);
  }
  memcpy(b + h.off_atom_user, p.user_of.data(), 4 * (size_t)p.n);
  memcpy(b + h.off_body, p.bodies.data(), sizeof(BodyRec) * (size_t)p.B);
  {
    // Vina XS radii of the 8 ligand map types
    static const double radius[8] = {1.9, 1.9, 1.8, 1.8, 1.8, 1.7, 1.7, 2.0};
    uint32_t* rec = (uint32_t*)(b + h.off_pairs);
    for (int k = 0; k < p.P; ++k) {
      const uint32_t pr = p.pairs[k], i = pr & 0xff, j = (pr >> 8) & 0xff, tp = pr >> 16;
      const float nrs = (float)-(radius[tp / DSDP_NUM_MAP_TYPES] + radius[tp % DSDP_NUM_MAP_TYPES]);
      rec[2 * k] = (i << 4) | (j << 20);
      memcpy(&rec[2 * k + 1], &nrs, 4);
    }
  }
  if (p.n_steps) memcpy(b + h.off_steps, p.steps.data(), 4 * p.steps.size());
  memcpy(b + h.off_lane_map, p.lane_map.data(), 2 * 64);
  if (p.T) memcpy(b + h.off_torsion_body, p.torsion_body.data(), 4 * (size_t)p.T);
  memcpy(b + h.off_atom64, p.local64.data(), 8 * 3 * (size_t)p.n);
  memcpy(b + h.off_body64, p.body64.data(), 8 * 6 * (size_t)p.B);
  return DSDP_OK;
}

extern "C" dsdp_status dsdp_ligand_blob_info(const void* blob, int32_t* n_atoms, int32_t* n_torsions,
                                             int32_t* n_pairs, int32_t* n_bodies) {
  if (!blob) return set_error(DSDP_ERR_INVALID_ARG, "blob is NULL");
  const BlobHeader* h = (const BlobHeader*)blob;
  if (h->magic != kBlobMagic) return set_error(DSDP_ERR_INVALID_ARG, "not a packed ligand blob");
  if (n_atoms) *n_atoms = h->n_atoms;
  if (n_torsions) *n_torsions = h->n_torsions;
  if (n_pairs) *n_pairs = h->n_pairs;
  if (n_bodies) *n_bodies = h->n_bodies;
  return DSDP_OK;
}
