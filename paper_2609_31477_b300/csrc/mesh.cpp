// Mesh analysis, run once per mesh on the host (Section 6, scaling study: the
// mesh and therefore the nonzero pattern never change, so the symbolic
// factorisation is computed once and reused by every Newton iteration).
//
//  1. unknown numbering (node-major inside nested-dissection supernodes)
//  2. CSR pattern of the Jacobian with the structural zeros of the block
//     structure of Section 3.2 (zero p-p and lambda-lambda blocks, pseudo-solid
//     rows independent of u, p, lambda)
//  3. element-to-nonzero map (e2nz) in the canonical pair order of the
//     element kernels, and an element colouring for a deterministic scatter
//  4. geometric nested dissection on element centroids, supernodes, front
//     index lists, assembly and extend-add maps, and the launch schedule of
//     the blocked numeric factorisation
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "viv_internal.h"

namespace viv {

void* DeviceArena::get(size_t n) {
  if (n == 0) n = 16;
  n = (n + 255) & ~size_t(255);
  void* p = nullptr;
  if (custom) {
    p = alloc.alloc(n, alloc.ctx);
    if (!p) throw Error{VIV_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed"};
  } else {
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{VIV_ERR_OOM, "cudaMalloc(" + std::to_string(n) + "): " + cudaGetErrorString(e)};
    }
  }
  blocks.push_back(p);
  bytes += n;
  return p;
}

void DeviceArena::release() {
  for (void* p : blocks) {
    if (custom)
      alloc.free(p, alloc.ctx);
    else
      cudaFree(p);
  }
  blocks.clear();
  bytes = 0;
}

namespace {

const int VERT[4] = {0, 2, 6, 8};
const int EDGE[4][3] = {{0, 3, 6}, {2, 5, 8}, {0, 1, 2}, {6, 7, 8}};
const int VERT3[8] = {0, 2, 6, 8, 18, 20, 24, 26};
const int VERT_TRI[3] = {0, 1, 2};
const int EDGE_TRI[3][3] = {{0, 3, 1}, {1, 4, 2}, {2, 5, 0}};   // (v_e, midpoint, v_{e+1})

// local node of position (s, t) on face f of a 27-node hexahedron: the face
// holds reference coordinate f / 2 at 0 (f even) or 1 (f odd); s runs along
// the first and t along the second of the other two directions
int hex_face_node(int f, int s, int t) {
  int idx[3];
  const int axis = f / 2;
  idx[axis] = 2 * (f % 2);
  int q = 0;
  for (int ax = 0; ax < 3; ++ax)
    if (ax != axis) idx[ax] = q++ == 0 ? s : t;
  return 9 * idx[2] + 3 * idx[1] + idx[0];
}

struct SN {
  std::vector<int> nodes;
  int parent = -1;
  std::vector<int> kids;
};

struct Dissector {
  const Mesh& m;
  int leaf;
  std::vector<double> cen[3];   // element centroids (seam-shifted coordinates)
  std::vector<int> owner, mark;
  int stamp = 0;
  std::vector<SN> sns;

  Dissector(const Mesh& mm, int leaf_) : m(mm), leaf(leaf_) {
    const int D = m.dim, P = m.npe;
    for (int d = 0; d < D; ++d) cen[d].resize(m.n_elems);
    for (int64_t e = 0; e < m.n_elems; ++e) {
      double sc[3] = {0, 0, 0};
      for (int a = 0; a < P; ++a) {
        int nd = m.conn[e * P + a];
        for (int d = 0; d < D; ++d) sc[d] += m.X[(int64_t)D * nd + d];
        if (D == 3 && (m.wrap[e] >> a & 1)) sc[2] += m.span;
      }
      for (int d = 0; d < D; ++d) cen[d][e] = sc[d] / P;
    }
    owner.assign(m.n_nodes, -1);
    mark.assign(m.n_nodes, 0);
  }

  int run(std::vector<int>& el, int lo, int hi) {
    const int P = m.npe;
    int cnt = hi - lo;
    if (cnt <= leaf) {
      int id = (int)sns.size();
      sns.emplace_back();
      for (int q = lo; q < hi; ++q)
        for (int a = 0; a < P; ++a) {
          int nd = m.conn[(int64_t)el[q] * P + a];
          if (owner[nd] < 0) {
            owner[nd] = id;
            sns[id].nodes.push_back(nd);
          }
        }
      return id;
    }
    // bisect at the median centroid along the longest extent
    int best = 0;
    double best_ext = -1;
    for (int d = 0; d < m.dim; ++d) {
      double c0 = 1e300, c1 = -1e300;
      for (int q = lo; q < hi; ++q) {
        c0 = std::min(c0, cen[d][el[q]]);
        c1 = std::max(c1, cen[d][el[q]]);
      }
      if (c1 - c0 > best_ext) {
        best_ext = c1 - c0;
        best = d;
      }
    }
    const std::vector<double>& key = cen[best];
    int mid = lo + cnt / 2;
    std::nth_element(el.begin() + lo, el.begin() + mid, el.begin() + hi, [&](int a, int b) {
      if (key[a] != key[b]) return key[a] < key[b];
      return a < b;
    });
    ++stamp;
    for (int q = lo; q < mid; ++q)
      for (int a = 0; a < P; ++a) mark[m.conn[(int64_t)el[q] * P + a]] = stamp;
    int id = (int)sns.size();
    sns.emplace_back();
    for (int q = mid; q < hi; ++q)
      for (int a = 0; a < P; ++a) {
        int nd = m.conn[(int64_t)el[q] * P + a];
        if (mark[nd] == stamp && owner[nd] < 0) {
          owner[nd] = id;
          sns[id].nodes.push_back(nd);
        }
      }
    int l = run(el, lo, mid);
    int r = run(el, mid, hi);
    sns[id].kids = {l, r};
    sns[l].parent = id;
    sns[r].parent = id;
    return id;
  }
};

// fn(begin, end) over [0, n) split among host threads; each index is handled
// by one thread, and the loops using it write disjoint outputs or sort
// afterwards, so the tables do not depend on the thread count
template <class Fn>
void parallel_for(int64_t n, Fn&& fn) {
  const int64_t hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const int64_t T = std::max<int64_t>(1, std::min<int64_t>(hw, n / 1024 + 1));
  if (T == 1) {
    fn((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (int64_t t = 0; t < T; ++t) th.emplace_back([&fn, n, t, T] { fn(n * t / T, n * (t + 1) / T); });
  for (auto& x : th) x.join();
}

int greedy_colour(const std::vector<int32_t>& items, int per, int64_t count, int64_t n_nodes,
                  std::vector<int32_t>& off, std::vector<int32_t>& order) {
  std::vector<uint64_t> used(n_nodes, 0);
  std::vector<int> col(count);
  int ncol = 0;
  for (int64_t e = 0; e < count; ++e) {
    uint64_t busy = 0;
    for (int a = 0; a < per; ++a) busy |= used[items[e * per + a]];
    int c = 0;
    while (c < 64 && (busy >> c & 1)) ++c;
    if (c >= 64) throw Error{VIV_ERR_ARG, "element colouring needs more than 64 colours"};
    col[e] = c;
    ncol = std::max(ncol, c + 1);
    for (int a = 0; a < per; ++a) used[items[e * per + a]] |= (uint64_t(1) << c);
  }
  off.assign(ncol + 1, 0);
  for (int64_t e = 0; e < count; ++e) off[col[e] + 1]++;
  for (int c = 0; c < ncol; ++c) off[c + 1] += off[c];
  order.assign(count, 0);
  std::vector<int32_t> pos(off.begin(), off.end() - 1);
  for (int64_t e = 0; e < count; ++e) order[pos[col[e]]++] = (int32_t)e;
  return ncol;
}

}  // namespace

void build_schedule(Mesh& m, int big_front);

// Build every host table of the mesh; see the file header.
void build_mesh(Mesh& m, const vivMeshDesc* d) {
  VIV_CHECK(d && d->X && d->conn && d->tags, VIV_ERR_ARG, "mesh description has NULL arrays");
  VIV_CHECK(d->n_nodes > 0 && d->n_elems > 0, VIV_ERR_ARG, "empty mesh");
  VIV_CHECK(d->n_nodes < (1LL << 30) && d->n_elems < (1LL << 28), VIV_ERR_ARG, "mesh too large");
  VIV_CHECK(d->n_gamma_faces == 0 || d->gamma_faces, VIV_ERR_ARG, "gamma_faces is NULL");
  VIV_CHECK(d->dim == 0 || d->dim == 2 || d->dim == 3, VIV_ERR_ARG, "dim must be 2 or 3");
  const int D = d->dim == 3 ? 3 : 2;
  VIV_CHECK(d->elem_type == VIV_ELEM_Q2 || (d->elem_type == VIV_ELEM_TRI_P2P1 && D == 2), VIV_ERR_ARG,
            "elem_type must be VIV_ELEM_Q2, or VIV_ELEM_TRI_P2P1 in two dimensions");
  const bool tri = d->elem_type == VIV_ELEM_TRI_P2P1;
  m.dim = D;
  m.tri = tri;
  m.npe = tri ? 6 : (D == 3 ? 27 : 9);
  m.nvert = tri ? 3 : (D == 3 ? 8 : 4);
  m.fpe = D == 3 ? 9 : 3;
  m.vol_pairs = tri ? TRI_PAIRS : (D == 3 ? VOL_PAIRS3 : VOL_PAIRS);
  m.face_pairs = D == 3 ? FACE_PAIRS3 : FACE_PAIRS;
  const int P = m.npe;
  const int* vert = tri ? VERT_TRI : (D == 3 ? VERT3 : VERT);
  const int64_t n = d->n_nodes, E = d->n_elems, F = d->n_gamma_faces;
  VIV_CHECK(D == 2 || E < (1LL << 31) / VOL_PAIRS3, VIV_ERR_ARG, "too many hexahedra for 32-bit element maps");
  m.n_nodes = n;
  m.n_elems = E;
  m.n_faces = F;
  m.X.assign(d->X, d->X + D * n);
  m.tags.assign(d->tags, d->tags + n);
  m.conn.resize(E * P);
  for (int64_t i = 0; i < E * P; ++i) {
    VIV_CHECK(d->conn[i] >= 0 && d->conn[i] < n, VIV_ERR_ARG, "connectivity out of range");
    m.conn[i] = (int32_t)d->conn[i];
  }
  m.span = D == 3 ? d->span : 0.0;
  m.wrap.assign(D == 3 ? E : 0, 0);
  if (D == 3 && d->wrap) {
    for (int64_t e = 0; e < E; ++e) {
      VIV_CHECK(d->wrap[e] >= 0 && d->wrap[e] < (1LL << 27), VIV_ERR_ARG, "wrap mask out of range");
      VIV_CHECK(d->wrap[e] == 0 || m.span > 0, VIV_ERR_ARG, "wrapped nodes need span > 0");
      m.wrap[e] = (int32_t)d->wrap[e];
    }
  }
  // every element positively oriented: the corner edge vectors at local node
  // 0 (quads and hexahedra: along xi, eta, zeta; triangles: to vertices 1, 2)
  // span a positive area / volume, wrapped nodes at their shifted position
  for (int64_t e = 0; e < E; ++e) {
    auto pt = [&](int a, double* v) {
      const int nd = m.conn[e * P + a];
      for (int i = 0; i < D; ++i) v[i] = m.X[(int64_t)D * nd + i];
      if (D == 3 && (m.wrap[e] >> a & 1)) v[2] += m.span;
    };
    double o[3], a[3], b[3], c[3] = {0, 0, 0};
    pt(0, o);
    pt(tri ? 1 : 2, a);
    pt(tri ? 2 : 6, b);
    if (D == 3) pt(18, c);
    for (int i = 0; i < D; ++i) {
      a[i] -= o[i];
      b[i] -= o[i];
      c[i] -= o[i];
    }
    const double vol = D == 2 ? a[0] * b[1] - a[1] * b[0]
                              : a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                                    a[2] * (b[0] * c[1] - b[1] * c[0]);
    VIV_CHECK(vol > 0, VIV_ERR_ARG, "element " + std::to_string(e) + " is not positively oriented");
  }
  std::vector<char> is_vertex(n, 0), cyl(n, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < m.nvert; ++c) is_vertex[m.conn[e * P + vert[c]]] = 1;
  for (int64_t a = 0; a < n; ++a) cyl[a] = (m.tags[a] & VIV_TAG_CYL) != 0;
  m.mid_parent.assign(tri ? 2 * n : 0, -1);
  if (tri) {   // midside nodes: their edge's end vertices, and straight edges
    double ext = 0;
    for (int64_t a = 0; a < 2 * n; ++a) ext = std::max(ext, std::fabs(m.X[a]));
    for (int64_t e = 0; e < E; ++e)
      for (int k = 0; k < 3; ++k) {
        const int mid = m.conn[e * 6 + 3 + k], va = m.conn[e * 6 + k], vb = m.conn[e * 6 + (k + 1) % 3];
        for (int i = 0; i < 2; ++i)
          VIV_CHECK(std::fabs(m.X[2 * mid + i] - 0.5 * (m.X[2 * va + i] + m.X[2 * vb + i])) <= 1e-12 * (1 + ext),
                    VIV_ERR_ARG, "a midside node is not at the midpoint of its edge");
        VIV_CHECK(!is_vertex[mid], VIV_ERR_ARG, "a node is a vertex of one triangle and a midside node of another");
        m.mid_parent[2 * mid] = va;
        m.mid_parent[2 * mid + 1] = vb;
      }
  }
  if (D == 3)
    for (int64_t a = 0; a < n; ++a)
      VIV_CHECK(!cyl[a] || (m.tags[a] & VIV_TAG_X_FIX_Z), VIV_ERR_ARG,
                "3-D Gamma nodes must hold their z position (VIV_TAG_X_FIX_Z)");
  m.faces.resize(F * m.fpe);
  m.face_elem.resize(F);
  m.face_wrap.assign(D == 3 ? F : 0, 0);
  for (int64_t f = 0; f < F; ++f) {
    int64_t e = d->gamma_faces[2 * f], ed = d->gamma_faces[2 * f + 1];
    VIV_CHECK(e >= 0 && e < E && ed >= 0 && ed < (tri ? 3 : 2 * D), VIV_ERR_ARG, "bad gamma face");
    m.face_elem[f] = (int32_t)e;
    for (int b = 0; b < m.fpe; ++b) {
      const int loc = D == 3 ? hex_face_node((int)ed, b % 3, b / 3) : (tri ? EDGE_TRI[ed][b] : EDGE[ed][b]);
      int nd = m.conn[e * P + loc];
      VIV_CHECK(cyl[nd], VIV_ERR_ARG, "gamma face node is not tagged CYL");
      m.faces[f * m.fpe + b] = nd;
      if (D == 3 && (m.wrap[e] >> loc & 1)) m.face_wrap[f] |= 1 << b;
    }
  }
  const bool has_body = F > 0;

  // ---- nested dissection -----------------------------------------------------
  int leaf = d->leaf_elems > 0 ? d->leaf_elems : (tri ? 8 : (D == 3 ? 2 : 4));
  Dissector ds(m, leaf);
  std::vector<int> el(E);
  std::iota(el.begin(), el.end(), 0);
  int root0 = ds.run(el, 0, (int)E);
  // splice out empty supernodes (keep the root)
  std::vector<SN>& sns = ds.sns;
  int S0 = (int)sns.size();
  std::vector<int> keep_parent(S0, -1);
  std::vector<char> kept(S0, 0);
  for (int s = 0; s < S0; ++s) kept[s] = !sns[s].nodes.empty() || s == root0;
  for (int s = 0; s < S0; ++s) {
    int p = sns[s].parent;
    while (p >= 0 && !kept[p]) p = sns[p].parent;
    keep_parent[s] = p;
  }
  // (delta is not a front unknown: it is numbered last and eliminated through
  // the FP64 border Schur complement after the fronts, see the border tables)
  // postorder over kept supernodes
  std::vector<std::vector<int>> kids(S0);
  for (int s = 0; s < S0; ++s)
    if (kept[s] && s != root0) kids[keep_parent[s]].push_back(s);
  std::vector<int> post;
  {
    std::vector<std::pair<int, int>> st{{root0, 0}};
    while (!st.empty()) {
      auto& [s, i] = st.back();
      if (i < (int)kids[s].size()) {
        int c = kids[s][i++];
        st.push_back({c, 0});
      } else {
        post.push_back(s);
        st.pop_back();
      }
    }
  }
  const int NF = (int)post.size();
  std::vector<int> pos_of(S0, -1);
  for (int i = 0; i < NF; ++i) pos_of[post[i]] = i;
  // front id of every node (n = delta)
  std::vector<int> front_of(n + 1, -1);
  for (int i = 0; i < NF; ++i)
    for (int nd : sns[post[i]].nodes) front_of[nd] = i;
  for (int64_t a = 0; a < n; ++a) VIV_CHECK(front_of[a] >= 0, VIV_ERR_ARG, "node outside every element");

  // ---- unknown numbering -----------------------------------------------------
  m.node_dof.assign(n * NSLOT, -1);
  m.delta_dof.assign(2, -1);
  m.f_first.resize(NF);
  m.f_p.resize(NF);
  m.f_parent.assign(NF, -1);
  std::vector<int32_t> node_first(n + 1, -1), node_cnt(n + 1, 0);
  int32_t next = 0;
  for (int i = 0; i < NF; ++i) {
    int s = post[i];
    std::vector<int>& nodes = sns[s].nodes;
    std::sort(nodes.begin(), nodes.end());
    m.f_first[i] = next;
    for (int nd : nodes) {
      node_first[nd] = next;
      if (nd == n) {
        m.delta_dof[0] = next++;
        m.delta_dof[1] = next++;
      } else {
        int32_t t = m.tags[nd];
        int32_t* sl = &m.node_dof[(int64_t)nd * NSLOT];
        static const int ufix[3] = {VIV_TAG_U_FIX_X, VIV_TAG_U_FIX_Y, VIV_TAG_U_FIX_Z};
        static const int xfix[3] = {VIV_TAG_X_FIX_X, VIV_TAG_X_FIX_Y, VIV_TAG_X_FIX_Z};
        for (int i = 0; i < D; ++i)
          if (!(t & ufix[i])) sl[S_UX + i] = next++;
        const bool has_x = !cyl[nd] && (!tri || is_vertex[nd]);   // triangles: P1 position
        for (int i = 0; i < D; ++i)
          if (has_x && !(t & xfix[i])) sl[S_XX + i] = next++;
        if (is_vertex[nd] && !(t & VIV_TAG_P_FIX)) sl[S_P] = next++;
        if (cyl[nd])
          for (int i = 0; i < D; ++i) sl[S_LX + i] = next++;
      }
      node_cnt[nd] = next - node_first[nd];
    }
    m.f_p[i] = next - m.f_first[i];
    if (s != root0) m.f_parent[i] = pos_of[keep_parent[s]];
  }
  m.n_front_dofs = next;   // unknowns of the fronts (everything but delta)
  if (has_body) {
    node_first[n] = next;
    m.delta_dof[0] = next++;
    m.delta_dof[1] = next++;
    node_cnt[n] = 2;
  }
  m.n_dofs = next;
  m.dof_node.assign(next, -1);
  m.dof_field.assign(next, -1);
  for (int64_t a = 0; a < n; ++a)
    for (int f = 0; f < NSLOT; ++f) {
      int dof = m.node_dof[a * NSLOT + f];
      if (dof >= 0) {
        m.dof_node[dof] = a;
        static const int code[NSLOT] = {VIV_F_UX, VIV_F_UY, VIV_F_UZ, VIV_F_XX, VIV_F_XY,
                                        VIV_F_XZ, VIV_F_P,  VIV_F_LX, VIV_F_LY, VIV_F_LZ};
        m.dof_field[dof] = code[f];
      }
    }
  if (has_body) {
    m.dof_node[m.delta_dof[0]] = n;
    m.dof_field[m.delta_dof[0]] = VIV_F_DX;
    m.dof_node[m.delta_dof[1]] = n;
    m.dof_field[m.delta_dof[1]] = VIV_F_DY;
  }

  // ---- element slot maps -------------------------------------------------------
  // element columns: cs = 2 D a + f (f < D: u_f of node a, else x_{f-D}), then
  // the pressure vertices at 2 D P + c; rows: u (D P), p, x (D P)
  const int NUX = 2 * D * P;          // u/x columns
  const int NCOL = NUX + m.nvert;     // all columns of a momentum row
  auto row_slot = [&](int64_t e, int cs) -> int32_t {
    if (cs < NUX) {
      int a = cs / (2 * D), f = cs % (2 * D);
      return m.node_dof[(int64_t)m.conn[e * P + a] * NSLOT + (f < D ? S_UX + f : S_XX + f - D)];
    }
    return m.node_dof[(int64_t)m.conn[e * P + vert[cs - NUX]] * NSLOT + S_P];
  };
  auto col_slot = [&](int64_t e, int cs) -> int32_t {
    if (cs < NUX) {
      int a = cs / (2 * D), f = cs % (2 * D);
      int nd = m.conn[e * P + a];
      if (f >= D && cyl[nd]) return f - D < 2 ? m.delta_dof[f - D] : -1;   // x = X + (delta, 0) on Gamma
      return m.node_dof[(int64_t)nd * NSLOT + (f < D ? S_UX + f : S_XX + f - D)];
    }
    return m.node_dof[(int64_t)m.conn[e * P + vert[cs - NUX]] * NSLOT + S_P];
  };
  // enumerate the structural pairs of an element in canonical order:
  // u rows x all columns, p rows x (u, x) columns, x rows x x columns
  // triangles: u columns 2 a + i, vertex position columns 12 + 2 v + k, pressure 18 + c
  auto tri_col = [&](int64_t e, int cs) -> int32_t {
    if (cs < 12) return m.node_dof[(int64_t)m.conn[e * 6 + cs / 2] * NSLOT + S_UX + cs % 2];
    if (cs < 18) {
      const int nd = m.conn[e * 6 + (cs - 12) / 2], k = (cs - 12) % 2;
      return cyl[nd] ? m.delta_dof[k] : m.node_dof[(int64_t)nd * NSLOT + S_XX + k];
    }
    return m.node_dof[(int64_t)m.conn[e * 6 + cs - 18] * NSLOT + S_P];
  };
  auto for_pairs = [&](int64_t e, auto&& fn) {
    if (tri) {
      auto nd = [&](int a) { return (int64_t)m.conn[e * 6 + a] * NSLOT; };
      for (int a = 0; a < 6; ++a)
        for (int i = 0; i < 2; ++i)
          for (int cs = 0; cs < 21; ++cs) fn(tpairA(a, i, cs), m.node_dof[nd(a) + S_UX + i], tri_col(e, cs));
      for (int c = 0; c < 3; ++c)
        for (int cs = 0; cs < 18; ++cs) fn(tpairB(c, cs), m.node_dof[nd(c) + S_P], tri_col(e, cs));
      for (int v = 0; v < 3; ++v)
        for (int i = 0; i < 2; ++i)
          for (int w = 0; w < 3; ++w)
            for (int k = 0; k < 2; ++k)
              fn(tpairC(v, i, w, k), m.node_dof[nd(v) + S_XX + i], tri_col(e, 12 + 2 * w + k));
      return;
    }
    int idx = 0;
    for (int a = 0; a < P; ++a)
      for (int i = 0; i < D; ++i)
        for (int cs = 0; cs < NCOL; ++cs) fn(idx++, row_slot(e, 2 * D * a + i), col_slot(e, cs));
    for (int c = 0; c < m.nvert; ++c)
      for (int cs = 0; cs < NUX; ++cs) fn(idx++, row_slot(e, NUX + c), col_slot(e, cs));
    for (int a = 0; a < P; ++a)
      for (int i = 0; i < D; ++i)
        for (int b = 0; b < P; ++b)
          for (int k = 0; k < D; ++k)
            fn(idx++, row_slot(e, 2 * D * a + D + i), col_slot(e, 2 * D * b + D + k));
  };
  auto for_face_pairs = [&](int64_t f, auto&& fn) {
    const int32_t* fn_ = &m.faces[f * m.fpe];
    auto nd_dof = [&](int b, int s) { return m.node_dof[(int64_t)fn_[b] * NSLOT + s]; };
    if (D == 2) {
      for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 2; ++i)
          for (int bp = 0; bp < 3; ++bp)
            for (int k = 0; k < 2; ++k) fn(fpairD(b, i, bp, k), nd_dof(b, S_UX + i), nd_dof(bp, S_LX + k));
      for (int b = 0; b < 3; ++b)
        for (int i = 0; i < 2; ++i)
          for (int cs = 0; cs < 12; ++cs) {
            int bp = (cs % 6) / 2, k = cs % 2;
            int32_t c = cs < 6 ? nd_dof(bp, S_UX + k) : m.delta_dof[k];
            fn(fpairE(b, i, cs), nd_dof(b, S_LX + i), c);
          }
      for (int i = 0; i < 2; ++i)
        for (int bp = 0; bp < 3; ++bp)
          for (int k = 0; k < 2; ++k) fn(fpairF(i, bp, k), m.delta_dof[i], nd_dof(bp, S_LX + k));
      return;
    }
    // 3-D: the face terms couple equal components only
    for (int b = 0; b < 9; ++b)
      for (int i = 0; i < 3; ++i)
        for (int bp = 0; bp < 9; ++bp) {
          fn(fpairD3(b, i, bp), nd_dof(b, S_UX + i), nd_dof(bp, S_LX + i));
          fn(fpairE3(b, i, bp), nd_dof(b, S_LX + i), nd_dof(bp, S_UX + i));
        }
    for (int b = 0; b < 9; ++b)
      for (int i = 0; i < 2; ++i) fn(fpairG3(b, i), nd_dof(b, S_LX + i), m.delta_dof[i]);
    for (int i = 0; i < 2; ++i)
      for (int bp = 0; bp < 9; ++bp) fn(fpairF3(i, bp), m.delta_dof[i], nd_dof(bp, S_LX + i));
  };

  // ---- CSR pattern -------------------------------------------------------------
  // every structural pair (element pairs, face pairs, the border diagonal) once
  // per occurrence, bucketed by row in two passes (count, fill), then each row
  // sorted and made unique
  {
    const int64_t N = m.n_dofs;
    std::vector<int64_t> off(N + 1, 0);
    parallel_for(E, [&](int64_t e0, int64_t e1) {
      for (int64_t e = e0; e < e1; ++e)
        for_pairs(e, [&](int, int32_t r, int32_t c) {
          if (r >= 0 && c >= 0) __atomic_fetch_add(&off[r + 1], (int64_t)1, __ATOMIC_RELAXED);
        });
    });
    for (int64_t f = 0; f < F; ++f)
      for_face_pairs(f, [&](int, int32_t r, int32_t c) {
        if (r >= 0 && c >= 0) ++off[r + 1];
      });
    if (has_body)
      for (int i = 0; i < 2; ++i) ++off[m.delta_dof[i] + 1];
    for (int64_t r = 0; r < N; ++r) off[r + 1] += off[r];
    std::vector<int32_t> buf(off[N]);
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    parallel_for(E, [&](int64_t e0, int64_t e1) {
      for (int64_t e = e0; e < e1; ++e)
        for_pairs(e, [&](int, int32_t r, int32_t c) {
          if (r >= 0 && c >= 0) buf[__atomic_fetch_add(&pos[r], (int64_t)1, __ATOMIC_RELAXED)] = c;
        });
    });
    for (int64_t f = 0; f < F; ++f)
      for_face_pairs(f, [&](int, int32_t r, int32_t c) {
        if (r >= 0 && c >= 0) buf[pos[r]++] = c;
      });
    if (has_body)
      for (int i = 0; i < 2; ++i) buf[pos[m.delta_dof[i]]++] = m.delta_dof[i];
    std::vector<int64_t> len(N);
    parallel_for(N, [&](int64_t r0, int64_t r1) {
      for (int64_t r = r0; r < r1; ++r) {
        auto b = buf.begin() + off[r], en = buf.begin() + off[r + 1];
        std::sort(b, en);
        len[r] = std::unique(b, en) - b;
      }
    });
    m.row_ptr.assign(N + 1, 0);
    for (int64_t r = 0; r < N; ++r) m.row_ptr[r + 1] = m.row_ptr[r] + len[r];
    VIV_CHECK(m.row_ptr[N] < (1LL << 31), VIV_ERR_ARG, "too many nonzeros for int32 CSR slots");
    m.col.resize(m.row_ptr[N]);
    parallel_for(N, [&](int64_t r0, int64_t r1) {
      for (int64_t r = r0; r < r1; ++r)
        std::copy(buf.begin() + off[r], buf.begin() + off[r] + len[r], m.col.begin() + m.row_ptr[r]);
    });
  }
  auto slot = [&](int32_t r, int32_t c) -> int32_t {
    if (r < 0 || c < 0) return -1;
    auto b = m.col.begin() + m.row_ptr[r], en = m.col.begin() + m.row_ptr[r + 1];
    auto it = std::lower_bound(b, en, c);
    return (int32_t)(it - m.col.begin());
  };
  const int VP = m.vol_pairs, FP = m.face_pairs;
  m.e2nz.assign(E * VP, -1);
  parallel_for(E, [&](int64_t e0, int64_t e1) {
    for (int64_t e = e0; e < e1; ++e)
      for_pairs(e, [&](int idx, int32_t r, int32_t c) { m.e2nz[e * VP + idx] = slot(r, c); });
  });
  m.f2nz.assign(F * FP, -1);
  for (int64_t f = 0; f < F; ++f)
    for_face_pairs(f, [&](int idx, int32_t r, int32_t c) { m.f2nz[f * FP + idx] = slot(r, c); });
  if (has_body)
    for (int i = 0; i < 2; ++i) m.dd_nz[i] = slot(m.delta_dof[i], m.delta_dof[i]);

  // ---- colours -------------------------------------------------------------------
  greedy_colour(m.conn, P, E, n, m.color_off, m.color_elems);
  if (F > 0)
    greedy_colour(m.faces, m.fpe, F, n, m.fcolor_off, m.fcolor_faces);
  else
    m.fcolor_off.assign(1, 0);

  // ---- symbolic factorisation on the node quotient graph ------------------------
  std::vector<std::vector<int32_t>> adj(n + 1);
  for (int64_t e = 0; e < E; ++e) {
    for (int a = 0; a < P; ++a) {
      int na = m.conn[e * P + a];
      for (int b = 0; b < P; ++b) adj[na].push_back(m.conn[e * P + b]);
    }
  }
  for (auto& v : adj) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  m.n_fronts = NF;
  std::vector<std::vector<int32_t>> cbn(NF);
  std::vector<int> mk(n + 1, -1);
  for (int i = 0; i < NF; ++i) {
    int s = post[i];
    for (int nd : sns[s].nodes) mk[nd] = i;
    std::vector<int32_t> set;
    auto consider = [&](int b) {
      if (mk[b] == i) return;
      if (front_of[b] <= i) return;
      mk[b] = i;
      set.push_back(b);
    };
    for (int nd : sns[s].nodes)
      for (int b : adj[nd]) consider(b);
    for (int c : kids[s])
      for (int b : cbn[pos_of[c]]) consider(b);
    std::sort(set.begin(), set.end(), [&](int a, int b) { return node_first[a] < node_first[b]; });
    cbn[i] = std::move(set);
  }
  // children lists in front ids
  m.f_child_off.assign(NF + 1, 0);
  for (int i = 0; i < NF; ++i) m.f_child_off[i + 1] = m.f_child_off[i] + (int)kids[post[i]].size();
  m.f_child.resize(m.f_child_off[NF]);
  for (int i = 0; i < NF; ++i)
    for (size_t j = 0; j < kids[post[i]].size(); ++j) m.f_child[m.f_child_off[i] + j] = pos_of[kids[post[i]][j]];
  // index lists, offsets
  m.f_m.resize(NF);
  m.f_off.resize(NF + 1);
  m.f_idx_off.resize(NF + 1);
  m.f_vec_off.resize(NF + 1);
  m.f_piv_off.resize(NF + 1);
  m.f_off[0] = m.f_idx_off[0] = m.f_vec_off[0] = 0;
  m.f_piv_off[0] = 0;
  m.f_idx.clear();
  m.factor_flops = 0;
  m.max_front = 0;
  m.max_p = 0;
  for (int i = 0; i < NF; ++i) {
    for (int32_t j = 0; j < m.f_p[i]; ++j) m.f_idx.push_back(m.f_first[i] + j);
    for (int b : cbn[i])
      for (int j = 0; j < node_cnt[b]; ++j) m.f_idx.push_back(node_first[b] + j);
    int64_t mm = (int64_t)m.f_idx.size() - m.f_idx_off[i];
    VIV_CHECK(mm < 46000, VIV_ERR_ARG, "front order exceeds the 32-bit local index range");
    m.f_m[i] = (int32_t)mm;
    m.max_front = std::max<int>(m.max_front, (int)mm);
    m.max_p = std::max<int>(m.max_p, m.f_p[i]);
    VIV_CHECK(2 * (int64_t)m.f_p[i] * 4 <= PERM_SMEM_MAX, VIV_ERR_ARG, "front pivot count exceeds the solve tables");
    m.f_idx_off[i + 1] = m.f_idx.size();
    m.f_off[i + 1] = m.f_off[i] + mm * mm;
    // solve workspace: the front vector, then the slice partial sums
    // (forward: ceil(p / SLICE) x (m - p); backward: ceil((m - p) / SLICE) x p)
    const int64_t pp = m.f_p[i], nn = mm - pp;
    const int64_t part = std::max((pp + SOLVE_SLICE - 1) / SOLVE_SLICE * nn, (nn + SOLVE_SLICE - 1) / SOLVE_SLICE * pp);
    m.f_vec_off[i + 1] = m.f_vec_off[i] + mm + part;
    m.f_piv_off[i + 1] = m.f_piv_off[i] + m.f_p[i];
    double p = m.f_p[i];
    for (int64_t j = 0; j < m.f_p[i]; ++j) {
      double r = (double)(mm - j - 1);
      m.factor_flops += r + 2.0 * r * r;
    }
    (void)p;
  }
  m.front_entries = m.f_off[NF];
  m.vec_entries = m.f_vec_off[NF];
  m.piv_entries = m.f_piv_off[NF];
  // local index lookup
  std::vector<int32_t> loc(m.n_dofs, -1);
  std::vector<int32_t> front_of_dof(m.n_dofs);
  for (int i = 0; i < NF; ++i)
    for (int j = 0; j < m.f_p[i]; ++j) front_of_dof[m.f_first[i] + j] = i;
  // original entries -> fronts (bucketed by the front of min(row, col))
  {
    const int64_t nnz = m.row_ptr[m.n_dofs];
    const int32_t nA = (int32_t)m.n_front_dofs;   // entries in a delta row or column are border entries
    std::vector<int64_t> cnt(NF + 1, 0);
    for (int64_t r = 0; r < nA; ++r)
      for (int64_t q = m.row_ptr[r]; q < m.row_ptr[r + 1]; ++q)
        if (m.col[q] < nA) cnt[front_of_dof[std::min<int32_t>(r, m.col[q])] + 1]++;
    for (int i = 0; i < NF; ++i) cnt[i + 1] += cnt[i];
    m.f_nz_off.assign(cnt.begin(), cnt.end());
    std::vector<int32_t> nz_row(nnz), nz_colv(nnz), nz_q(nnz);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t r = 0; r < nA; ++r)
      for (int64_t q = m.row_ptr[r]; q < m.row_ptr[r + 1]; ++q) {
        if (m.col[q] >= nA) continue;
        int f = front_of_dof[std::min<int32_t>(r, m.col[q])];
        int64_t at = fill[f]++;
        nz_row[at] = (int32_t)r;
        nz_colv[at] = m.col[q];
        nz_q[at] = (int32_t)q;
      }
    const int64_t nnz_fronts = m.f_nz_off[NF];
    m.f_nz_csr.resize(nnz_fronts);
    m.f_nz_pos.resize(nnz_fronts);
    m.f_col_nz_off.assign(NF + 1, 0);
    for (int i = 0; i < NF; ++i) {
      int mm = m.f_m[i];
      m.f_col_nz_off[i + 1] = m.f_col_nz_off[i] + (mm + ASM_COLS - 1) / ASM_COLS + 1;
    }
    m.f_col_nz.assign(m.f_col_nz_off[NF], 0);
    std::vector<std::pair<int32_t, int32_t>> tmp;
    for (int i = 0; i < NF; ++i) {
      int mm = m.f_m[i];
      for (int j = 0; j < mm; ++j) loc[m.f_idx[m.f_idx_off[i] + j]] = j;
      tmp.clear();
      for (int64_t at = m.f_nz_off[i]; at < m.f_nz_off[i + 1]; ++at) {
        int32_t lr = loc[nz_row[at]], lc = loc[nz_colv[at]];
        VIV_CHECK(lr >= 0 && lc >= 0, VIV_ERR_ARG, "symbolic: entry outside its front");
        tmp.push_back({lr + lc * mm, nz_q[at]});
      }
      std::sort(tmp.begin(), tmp.end(), [&](auto& a, auto& b) {
        int ca = a.first / mm, cb = b.first / mm;
        if (ca != cb) return ca < cb;
        return a.first < b.first;
      });
      int nch = (mm + ASM_COLS - 1) / ASM_COLS;
      int64_t base = m.f_nz_off[i];
      int ch = 0;
      for (size_t t = 0; t < tmp.size(); ++t) {
        m.f_nz_pos[base + t] = tmp[t].first;
        m.f_nz_csr[base + t] = tmp[t].second;
        int c = tmp[t].first / mm / ASM_COLS;
        while (ch <= c) m.f_col_nz[m.f_col_nz_off[i] + ch++] = (int32_t)t;
      }
      while (ch <= nch) m.f_col_nz[m.f_col_nz_off[i] + ch++] = (int32_t)tmp.size();
      // extend-add map of each child
      for (int j = 0; j < mm; ++j) loc[m.f_idx[m.f_idx_off[i] + j]] = -1;
    }
    m.f_ea_off.assign(NF + 1, 0);
    for (int i = 0; i < NF; ++i) m.f_ea_off[i + 1] = m.f_ea_off[i] + (m.f_m[i] - m.f_p[i]);
    m.f_ea.assign(m.f_ea_off[NF], -1);
    for (int i = 0; i < NF; ++i) {
      int par = m.f_parent[i];
      if (par < 0) {
        VIV_CHECK(m.f_m[i] == m.f_p[i], VIV_ERR_ARG, "symbolic: root front has a contribution block");
        continue;
      }
      int pm = m.f_m[par];
      for (int j = 0; j < pm; ++j) loc[m.f_idx[m.f_idx_off[par] + j]] = j;
      for (int j = m.f_p[i]; j < m.f_m[i]; ++j) {
        int32_t l = loc[m.f_idx[m.f_idx_off[i] + j]];
        VIV_CHECK(l >= 0, VIV_ERR_ARG, "symbolic: contribution block row missing in the parent");
        m.f_ea[m.f_ea_off[i] + (j - m.f_p[i])] = l;
      }
      for (int j = 0; j < pm; ++j) loc[m.f_idx[m.f_idx_off[par] + j]] = -1;
    }
  }
  // border tables: delta rows C (entries in front columns), delta columns B
  // (entries in front rows) and D, as CSR slots
  m.bc_off.assign(3, 0);
  m.bb_off.assign(3, 0);
  m.bc_col.clear();
  m.bc_q.clear();
  m.bb_row.clear();
  m.bb_q.clear();
  for (int i = 0; i < 4; ++i) m.bd_q[i] = -1;
  if (has_body) {
    const int32_t nA = (int32_t)m.n_front_dofs;
    for (int i = 0; i < 2; ++i) {
      const int32_t r = m.delta_dof[i];
      for (int64_t q = m.row_ptr[r]; q < m.row_ptr[r + 1]; ++q) {
        if (m.col[q] < nA) {
          m.bc_col.push_back(m.col[q]);
          m.bc_q.push_back((int32_t)q);
        } else {
          m.bd_q[2 * i + (m.col[q] - nA)] = (int32_t)q;
        }
      }
      m.bc_off[i + 1] = (int32_t)m.bc_col.size();
    }
    for (int j = 0; j < 2; ++j) {
      for (int32_t r = 0; r < nA; ++r)
        for (int64_t q = m.row_ptr[r]; q < m.row_ptr[r + 1]; ++q)
          if (m.col[q] == m.delta_dof[j]) {
            m.bb_row.push_back(r);
            m.bb_q.push_back((int32_t)q);
          }
      m.bb_off[j + 1] = (int32_t)m.bb_row.size();
    }
  }
  // levels (height above the leaves)
  m.f_level.assign(NF, 0);
  for (int i = 0; i < NF; ++i)   // postorder: children first
    for (int c = m.f_child_off[i]; c < m.f_child_off[i + 1]; ++c)
      m.f_level[i] = std::max(m.f_level[i], m.f_level[m.f_child[c]] + 1);
  m.n_levels = 0;
  for (int i = 0; i < NF; ++i) m.n_levels = std::max(m.n_levels, m.f_level[i] + 1);
  m.level_off.assign(m.n_levels + 1, 0);
  for (int i = 0; i < NF; ++i) m.level_off[m.f_level[i] + 1]++;
  for (int l = 0; l < m.n_levels; ++l) m.level_off[l + 1] += m.level_off[l];
  m.level_fronts.assign(NF, 0);
  m.level_maxm.assign(m.n_levels, 0);
  {
    std::vector<int32_t> fill(m.level_off.begin(), m.level_off.end() - 1);
    for (int i = 0; i < NF; ++i) {
      m.level_fronts[fill[m.f_level[i]]++] = i;
      m.level_maxm[m.f_level[i]] = std::max(m.level_maxm[m.f_level[i]], m.f_m[i]);
    }
  }
  // solve threads per front, by level: the chains update pivot rows only
  m.level_maxp.assign(m.n_levels, 0);
  for (int i = 0; i < NF; ++i) m.level_maxp[m.f_level[i]] = std::max(m.level_maxp[m.f_level[i]], m.f_p[i]);
  m.level_threads.assign(m.n_levels, 64);
  for (int l = 0; l < m.n_levels; ++l) {
    int t = ((m.level_maxp[l] + 31) / 32) * 32;
    m.level_threads[l] = std::min(1024, std::max(64, t));
  }
  // diagonal blocks to invert, and the slice items of the solves by level
  m.inv_items.clear();
  for (int i = 0; i < NF; ++i)
    for (int jb = 0; jb < m.f_p[i]; jb += 32) {
      m.inv_items.push_back(i);
      m.inv_items.push_back(jb);
    }
  m.fg_items.clear();
  m.bg_items.clear();
  m.fg_off.assign(m.n_levels + 1, 0);
  m.bg_off.assign(m.n_levels + 1, 0);
  m.solve_fused.assign(NF, 0);
  for (int l = 0; l < m.n_levels; ++l) {
    bool fuse_f = true, fuse_b = true;
    for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
      const int f = m.level_fronts[q];
      const int pp = m.f_p[f], nn = m.f_m[f] - pp;
      fuse_f = fuse_f && pp <= SOLVE_FUSE_F && nn <= 2 * SOLVE_SLICE;
      fuse_b = fuse_b && nn <= SOLVE_FUSE_B && pp <= SOLVE_SLICE;
    }
    for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
      const int f = m.level_fronts[q];
      const int pp = m.f_p[f], nn = m.f_m[f] - pp;
      m.solve_fused[f] = (fuse_f ? 1 : 0) | (fuse_b ? 2 : 0);
      if (!(m.solve_fused[f] & 1))
        for (int s0 = 0; s0 * SOLVE_SLICE < pp; ++s0)
          for (int r0 = 0; r0 < nn; r0 += SOLVE_ROWS) m.fg_items.insert(m.fg_items.end(), {f, r0, s0, 0});
      if (!(m.solve_fused[f] & 2))
        for (int s0 = 0; s0 * SOLVE_SLICE < nn; ++s0)
          for (int r0 = 0; r0 < pp; r0 += SOLVE_ROWS) m.bg_items.insert(m.bg_items.end(), {f, r0, s0, 0});
    }
    m.fg_off[l + 1] = (int32_t)(m.fg_items.size() / 4);
    m.bg_off[l + 1] = (int32_t)(m.bg_items.size() / 4);
  }
  // image chunks of the tensor-core operand split that a mixed case holds: an
  // upper bound for every schedule (each outer-block step of a level at most
  // splits the blocks of all its fronts; a smaller large-front threshold only
  // adds fronts), capped at TC_IMG_MAX_CHUNKS unless one front alone needs more
  {
    int64_t bound = 0, single = 0;
    for (int l = 0; l < m.n_levels; ++l) {
      int maxp = 0;
      for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) maxp = std::max(maxp, m.f_p[m.level_fronts[q]]);
      for (int k2 = 0; k2 < maxp; k2 += OUTER_NB) {
        int64_t sum = 0;
        for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
          const int f = m.level_fronts[q];
          const int be = std::min(k2 + OUTER_NB, m.f_p[f]);
          if (m.f_p[f] <= k2 || be >= m.f_m[f]) continue;
          // (+ 2 chunks of each K slice for the inverse triangles of the block path)
          const int64_t need = 2 * (int64_t)((m.f_m[f] - be + 127) / 128 + 1) * ((be - k2 + 31) / 32);
          sum += need;
          single = std::max(single, need);
        }
        bound = std::max(bound, sum);
      }
    }
    m.tc_img_chunks = std::min(bound, std::max(TC_IMG_MAX_CHUNKS, single));
  }
  build_schedule(m, BIG_FRONT);
}

// The 128-column block at pivot k2 of every large FP32 front of level l with
// windowed pivoting: block LU (one CTA per front: the diagonal block, its row
// permutations and the inverse triangles as operand images), the block rows'
// permutation on the other columns, then on the tensor cores L21 = A21 U11^-1
// and U12 = L11^-1 P A12, and the Schur update A22 -= L21 U12.  Fronts are
// grouped so that a group's operand images fit the case's image buffer:
// per front [A21 row blocks][P A12 column blocks][(I - L^-1)][(I - U^-1)],
// the L21 / U12 split reusing the first two.
// fronts of the block path: large, with more than one pivot window (a single
// window is factored faster by the per-panel kernels)
static bool block_front(const Mesh& m, int f, int big_front) {
  return m.f_m[f] >= big_front && m.f_p[f] > PANEL_NB && (m.level_block.empty() || m.level_block[m.f_level[f]]);
}

template <class Push, class Open, class Close, class Items>
static void emit_blocks(Mesh& m, int l, int k2, int big_front, Push& push, Open& open, Close& close, Items& items) {
  std::vector<int> fr;
  for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
    const int f = m.level_fronts[q];
    if (block_front(m, f, big_front) && m.f_p[f] > k2) fr.push_back(f);
  }
  auto geom = [&](int f, int& be, int& nb, int& nch, int& nbk) {
    be = std::min(k2 + OUTER_NB, m.f_p[f]);
    nb = be - k2;
    nch = (nb + 31) / 32;
    nbk = (m.f_m[f] - be + 127) / 128;
  };
  size_t g0 = 0;
  while (g0 < fr.size()) {
    // a group within the image capacity
    size_t g1 = g0;
    int64_t chunks = 0;
    while (g1 < fr.size()) {
      int be, nb, nch, nbk;
      geom(fr[g1], be, nb, nch, nbk);
      const int64_t need = nbk > 0 ? 2 * (int64_t)(nbk + 1) * nch : 0;
      if (g1 > g0 && chunks + need > m.tc_img_chunks) break;
      chunks += need;
      ++g1;
    }
    VIV_CHECK(chunks <= m.tc_img_chunks, VIV_ERR_ARG, "tensor-core operand images exceed the case buffer");
    std::vector<int64_t> a21(g1 - g0), pa12(g1 - g0), ainv(g1 - g0), binv(g1 - g0);
    int64_t blk = 0;
    for (size_t g = g0; g < g1; ++g) {
      int be, nb, nch, nbk;
      geom(fr[g], be, nb, nch, nbk);
      if (nbk == 0) {
        a21[g - g0] = pa12[g - g0] = ainv[g - g0] = binv[g - g0] = -1;
        continue;
      }
      a21[g - g0] = blk;
      blk += (int64_t)nbk * nch;
      pa12[g - g0] = blk;
      blk += (int64_t)nbk * nch;
      ainv[g - g0] = blk;
      blk += nch;
      binv[g - g0] = blk;
      blk += nch;
    }
    auto L1 = open(L_BLOCK_LU, l, k2);
    for (size_t g = g0; g < g1; ++g) {
      int be, nb, nch, nbk;
      geom(fr[g], be, nb, nch, nbk);
      push({fr[g], k2, (int)ainv[g - g0], (int)binv[g - g0], nch});
      L1.aux = std::max(L1.aux, 32 * nch);   // CTA size and shared memory of the launch
    }
    close(L1);
    auto L2 = open(L_BLOCK_PERM, l, k2);
    for (size_t g = g0; g < g1; ++g) {
      const int f = fr[g];
      int be, nb, nch, nbk;
      geom(f, be, nb, nch, nbk);
      if (m.f_m[f] > nb)
        for (int c0 = 0; c0 < m.f_m[f]; c0 += 256) push({f, k2, c0});
    }
    close(L2);
    // splits of A21 / P A12 (first) and of L21 / U12 (after the first update)
    auto split = [&](int check) {
      auto S = open(L_TC_SPLIT, l, k2);
      for (size_t g = g0; g < g1; ++g) {
        const int f = fr[g], mm = m.f_m[f];
        int be, nb, nch, nbk;
        geom(f, be, nb, nch, nbk);
        for (int i = 0; i < nbk; ++i)
          for (int ch = 0; ch < nch; ++ch)
            push({f, be + 128 * i, 0, k2 + 32 * ch, std::min(32, nb - 32 * ch), (int)(a21[g - g0] + i * nch + ch), mm,
                  check});
        for (int j = 0; j < nbk; ++j)
          for (int ch = 0; ch < nch; ++ch)
            push({f, be + 128 * j, 1, k2 + 32 * ch, std::min(32, nb - 32 * ch), (int)(pa12[g - g0] + j * nch + ch), mm});
      }
      close(S);
    };
    split(0);
    auto T1 = open(L_TC_GEMM, l, k2);   // L21 = A21 - A21 (I - U^-1), U12 = P A12 - (I - L^-1) P A12
    for (size_t g = g0; g < g1; ++g) {
      const int f = fr[g], mm = m.f_m[f];
      int be, nb, nch, nbk;
      geom(f, be, nb, nch, nbk);
      for (int i = 0; i < nbk; ++i)
        push({f, be + 128 * i, k2, mm, be, (int)(a21[g - g0] + i * nch), (int)binv[g - g0], nch});
      for (int j = 0; j < nbk; ++j)
        push({f, k2, be + 128 * j, be, mm, (int)ainv[g - g0], (int)(pa12[g - g0] + j * nch), nch});
    }
    close(T1);
    split(1);   // (and the threshold test of the multipliers L21)
    auto T2 = open(L_TC_GEMM, l, k2);   // A22 -= L21 U12
    for (size_t g = g0; g < g1; ++g) {
      const int f = fr[g], mm = m.f_m[f];
      int be, nb, nch, nbk;
      geom(f, be, nb, nch, nbk);
      for (int i = 0; i < nbk; ++i)
        for (int j = 0; j < nbk; ++j)
          push({f, be + 128 * i, be + 128 * j, mm, mm, (int)(a21[g - g0] + i * nch), (int)(pa12[g - g0] + j * nch),
                nch});
      const double rest = (double)(mm - be);
      m.window_tc_flops += 4.0 * nb * nb * rest + 2.0 * rest * rest * nb;
      // LU of the nb x nb block, and with rows below it the two triangle inverses
      double lu = 0;
      for (int j = 0; j < nb; ++j) lu += (double)(nb - j - 1) + 2.0 * (nb - j - 1) * (nb - j - 1);
      m.window_lu_flops += lu + (nbk > 0 ? 2.0 * nb * (double)nb * nb / 3.0 : 0.0);
    }
    close(T2);
    (void)items;
    g0 = g1;
  }
}

// Launch schedules of the numeric factorisation for a large-front threshold
// (fronts of order >= big_front use 128-column outer blocks).
void build_schedule(Mesh& m, int big_front) {
  m.big_front = big_front;
  // launch schedules of the numeric factorisation, one per front element size.
  // Fronts of order >= BIG_FRONT are factored in 128-column outer blocks: four
  // 32-column pivot panels update only the block's own columns; the outer
  // columns receive the block's row interchanges, then its TRSM, then one
  // K = 128 Schur update (tensor cores on the FP32 path).
  m.work.clear();
  m.gemm_flops = m.trsm_flops = m.panel_flops = m.outer_flops = 0;
  m.tc_split_chunks = m.tc_tiles = 0;
  m.window_tc_flops = m.window_lu_flops = m.window_gemm_flops = 0;
  m.blk_front.assign(m.n_fronts, 0);
  for (int f = 0; f < m.n_fronts; ++f) m.blk_front[f] = m.block_lu && block_front(m, f, big_front) ? 1 : 0;
  // multi-CTA chains: tasks per level, flags per block
  m.mc_fwd.clear();
  m.mc_bwd.clear();
  m.mc_off.assign(m.n_levels + 1, 0);
  m.mc_flags = 0;
  m.chain_flag_bound = 0;
  for (int f = 0; f < m.n_fronts; ++f)
    if (m.f_p[f] >= MULTI_CHAIN_P) m.chain_flag_bound += (m.f_p[f] + OUTER_NB - 1) / OUTER_NB;
  for (int l = 0; l < m.n_levels; ++l) {
    std::vector<std::array<int, 3>> fr;   // (front, blocks, first flag)
    for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
      const int f = m.level_fronts[q];
      if (m.blk_front[f] && m.f_p[f] >= MULTI_CHAIN_P) {
        m.blk_front[f] = 2;
        const int nblk = (m.f_p[f] + OUTER_NB - 1) / OUTER_NB;
        fr.push_back({f, nblk, m.mc_flags});
        m.mc_flags += nblk;
      }
    }
    int maxb = 0;
    for (auto& e : fr) maxb = std::max(maxb, e[1]);
    for (int d = 0; d < maxb; ++d)
      for (auto& e : fr)
        if (d < e[1]) {
          m.mc_fwd.insert(m.mc_fwd.end(), {e[0], d, e[2]});
          m.mc_bwd.insert(m.mc_bwd.end(), {e[0], e[1] - 1 - d, e[2]});
        }
    m.mc_off[l + 1] = (int)(m.mc_fwd.size() / 3);
  }
  m.inv_items_blk.clear();
  for (size_t q = 0; q + 1 < m.inv_items.size(); q += 2)
    if (!m.blk_front[m.inv_items[q]]) {
      m.inv_items_blk.push_back(m.inv_items[q]);
      m.inv_items_blk.push_back(m.inv_items[q + 1]);
    }
  auto push = [&](std::initializer_list<int> v) {
    int n = 0;
    for (int x : v) {
      m.work.push_back(x);
      ++n;
    }
    for (; n < WORK_STRIDE; ++n) m.work.push_back(0);
  };
  auto items = [&]() { return (int64_t)m.work.size() / WORK_STRIDE; };
  for (int var = 0; var < 4; ++var) {
    const int prec = var & 1;          // FP64 fronts
    const bool window = var >= 2;      // pivots restricted to the diagonal block
    const bool count = var == 0;
    const int esz = prec ? 8 : 4;
    const int rows_cta = PANEL_SMEM_BYTES / (PANEL_NB * esz);   // panel rows one CTA holds
    std::vector<Launch>& sched = m.sched[var];
    sched.clear();
    auto open = [&](int kind, int l, int k) { return Launch{kind, l, k, items(), 0}; };
    auto close = [&](Launch L) {
      L.count = items() - L.item0;
      if (L.count) sched.push_back(L);
    };
    // diag_tile: the tile at (r0, c0) also factors the next panel's diagonal block
    auto gemm_tiles = [&](int f, int r0, int r_end, int c0, int c_end, int kb, int kl, bool diag_tile = false) {
      for (int rb = r0; rb < r_end; rb += GEMM_TILE)
        for (int cb = c0; cb < c_end; cb += GEMM_TILE)
          push({f, rb, cb, r_end, c_end, kb, kl, (diag_tile && rb == r0 && cb == c0) ? 1 : 0});
      const double fl = 2.0 * std::max(0, r_end - r0) * std::max(0, c_end - c0) * kl;
      if (count) m.gemm_flops += fl;
      if (window && prec == 0) m.window_gemm_flops += fl;
    };
    // windowed pivoting: the diagonal block of panel k of front f is factored by
    // the Schur update of panel k - 32 when that update covers it (every panel
    // but the first, and but the first of each outer block of a large front)
    auto diag_fused = [&](int f, int k) {
      return window && k > 0 && k < m.f_p[f] && (m.f_m[f] < big_front || k % OUTER_NB != 0);
    };
    // FP32 fronts with windowed pivoting and 128-column blocks: each block is
    // factored by one CTA (block_lu_kernel) and its L21 / U12 and the Schur
    // update run on the tensor cores; these fronts take no per-panel launches
    const bool blockpath = window && prec == 0 && m.block_lu;
    auto newblk = [&](int f) { return blockpath && block_front(m, f, big_front); };
    for (int l = 0; l < m.n_levels; ++l) {
      Launch L = open(L_ASSEMBLE, l, 0);
      L.aux = m.level_maxm[l] >= 1024 ? 512 : 256;   // assembly threads per item
      int maxp = 0;
      for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
        int f = m.level_fronts[q];
        for (int c0 = 0; c0 < m.f_m[f]; c0 += ASM_COLS) push({f, c0});
        maxp = std::max(maxp, m.f_p[f]);
      }
      close(L);
      for (int k = 0; k < maxp; k += PANEL_NB) {
        const int k2 = (k / OUTER_NB) * OUTER_NB;
        auto big = [&](int f) { return m.f_m[f] >= big_front; };
        auto block_end = [&](int f) { return std::min(k2 + OUTER_NB, m.f_p[f]); };
        if (blockpath && k == k2) emit_blocks(m, l, k2, big_front, push, open, close, items);
        // panel kind of a front: 0 one CTA, 1 cluster, 2 global-memory fallback
        auto kind = [&](int f) {
          const int rows = m.f_m[f] - k;
          if (rows <= rows_cta) return 0;
          if ((rows + PANEL_CLUSTER - 1) / PANEL_CLUSTER <= rows_cta) return 1;
          return 2;
        };
        if (window) {
          // one warp per front factors the diagonal block; then, in one launch,
          // the rows below it (L21) and the columns outside the panel (row
          // permutation everywhere, U12 inside the block's column range)
          Launch D = open(L_DIAG, l, k);
          for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
            int f = m.level_fronts[q];
            if (m.f_p[f] > k && !diag_fused(f, k) && !newblk(f)) push({f});
          }
          close(D);
          Launch W = open(L_WINDOW, l, k);
          for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
            int f = m.level_fronts[q];
            if (m.f_p[f] <= k || newblk(f)) continue;
            const int nbe = std::min(PANEL_NB, m.f_p[f] - k);
            // U12 for every column right of the panel, the outer columns of a
            // large front included (their in-block rows are updated below)
            for (int r0 = k + nbe; r0 < m.f_m[f]; r0 += WINDOW_THREADS) push({0, f, r0});
            for (int c0 = 0; c0 < m.f_m[f]; c0 += WINDOW_THREADS) push({1, f, c0, m.f_m[f]});
          }
          close(W);
        }
        for (int pk = 0; pk < 2 && !window; ++pk) {
          Launch PC = open(pk == 0 ? L_PANEL_1 : L_PANEL_CL, l, k);
          int rows = 0;
          for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
            int f = m.level_fronts[q];
            if (m.f_p[f] > k && kind(f) == pk) {
              push({f});
              const int r = m.f_m[f] - k;
              rows = std::max(rows, pk == 0 ? r : (r + PANEL_CLUSTER - 1) / PANEL_CLUSTER);
            }
          }
          PC.aux = rows;
          close(PC);
        }
        if (!window) {
          Launch SW = open(L_LASWP, l, k);
          for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
            int f = m.level_fronts[q];
            if (m.f_p[f] > k && kind(f) < 2)
              for (int c0 = 0; c0 < m.f_m[f]; c0 += LASWP_COLS) push({f, c0});
          }
          close(SW);
          Launch P = open(L_PANEL, l, k);
          for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
            int f = m.level_fronts[q];
            if (m.f_p[f] > k && kind(f) == 2) push({f});
          }
          close(P);
        }
        // TRSM and GEMM of this panel (inside the outer block for large fronts)
        Launch T = open(L_TRSM, l, k);
        for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
          int f = m.level_fronts[q];
          if (m.f_p[f] <= k) continue;
          const int nbe = std::min(PANEL_NB, m.f_p[f] - k);
          const int c_end = big(f) ? block_end(f) : m.f_m[f];
          if (!window)
            for (int c0 = k + nbe; c0 < c_end; c0 += TRSM_COLS) push({f, c0, c_end, k});
          double pf = 0;   // the panel's LU flops (its rows below included)
          for (int j = k; j < k + nbe; ++j) {
            const double below = (double)(m.f_m[f] - j - 1);
            pf += below + 2.0 * below * (k + nbe - j - 1);
          }
          if (count) {
            m.trsm_flops += (double)nbe * (nbe - 1) * std::max(0, c_end - k - nbe);
            m.panel_flops += pf;
          }
          if (window && prec == 0 && !newblk(f)) m.window_lu_flops += pf;
        }
        close(T);
        Launch G = open(L_GEMM, l, k);
        for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
          int f = m.level_fronts[q];
          if (m.f_p[f] <= k || newblk(f)) continue;
          const int nbe = std::min(PANEL_NB, m.f_p[f] - k);
          const int r0 = k + nbe;
          const int c_end = big(f) ? block_end(f) : m.f_m[f];
          gemm_tiles(f, r0, m.f_m[f], r0, c_end, k, nbe, diag_fused(f, r0));
          // windowed schedule: the outer columns' rows inside the block, panel by panel
          if (window && big(f) && c_end < m.f_m[f]) gemm_tiles(f, r0, c_end, c_end, m.f_m[f], k, nbe);
        }
        close(G);
        // large fronts whose outer block ends with this panel: the outer columns
        std::vector<int> done;
        for (int q = m.level_off[l]; q < m.level_off[l + 1]; ++q) {
          int f = m.level_fronts[q];
          if (m.f_p[f] <= k || !big(f) || newblk(f)) continue;
          const int nbe = std::min(PANEL_NB, m.f_p[f] - k);
          if (k + nbe == block_end(f) && block_end(f) < m.f_m[f]) done.push_back(f);
        }
        if (done.empty()) continue;
        for (int s0 = k2; s0 <= k && !window; s0 += PANEL_NB) {
          Launch OT = open(L_TRSM, l, s0);
          for (int f : done) {
            const int be = block_end(f);
            if (s0 >= be) continue;
            const int nbe = std::min(PANEL_NB, m.f_p[f] - s0);
            for (int c0 = be; c0 < m.f_m[f]; c0 += TRSM_COLS) push({f, c0, m.f_m[f], s0});
            if (count) m.trsm_flops += (double)nbe * (nbe - 1) * (m.f_m[f] - be);
          }
          close(OT);
          Launch OG = open(L_GEMM, l, s0);
          for (int f : done) {
            const int be = block_end(f);
            const int nbe = std::min(PANEL_NB, m.f_p[f] - s0);
            if (s0 + nbe < be) gemm_tiles(f, s0 + nbe, be, be, m.f_m[f], s0, nbe);
          }
          close(OG);
        }
        if (prec == 0) {
          // tensor cores: the fronts' L21 / U12 chunks are split into hi/lo
          // TF32 images (one launch), then the 128 x 128 tiles are updated from
          // them (one persistent launch); fronts are grouped so that a group's
          // images fit the case's image buffer
          std::vector<int> group;
          int64_t group_chunks = 0;
          auto flush = [&]() {
            if (group.empty()) return;
            std::vector<int64_t> a_base(group.size()), b_base(group.size());
            int64_t blk = 0;
            Launch SP = open(L_TC_SPLIT, l, k2);
            for (size_t g = 0; g < group.size(); ++g) {
              const int f = group[g], be = block_end(f), mm = m.f_m[f], kl = be - k2;
              const int nch = (kl + 31) / 32;
              a_base[g] = blk;
              for (int rb = be; rb < mm; rb += 128)
                for (int ch = 0; ch < nch; ++ch)
                  push({f, rb, 0, k2 + 32 * ch, std::min(32, kl - 32 * ch), (int)blk++, mm});
              b_base[g] = blk;
              for (int cb = be; cb < mm; cb += 128)
                for (int ch = 0; ch < nch; ++ch)
                  push({f, cb, 1, k2 + 32 * ch, std::min(32, kl - 32 * ch), (int)blk++, mm});
            }
            close(SP);
            VIV_CHECK(blk <= m.tc_img_chunks, VIV_ERR_ARG, "tensor-core operand images exceed the case buffer");
            if (count) m.tc_split_chunks += blk;
            // tiles row block by row block: a CTA takes a contiguous range, so
            // its consecutive tiles mostly share the row block's A chunks
            Launch TC = open(L_TC_GEMM, l, k2);
            for (size_t g = 0; g < group.size(); ++g) {
              const int f = group[g], be = block_end(f), mm = m.f_m[f];
              const int nch = (be - k2 + 31) / 32, nb = (mm - be + 127) / 128;
              for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j)
                  push({f, be + 128 * i, be + 128 * j, mm, mm, (int)(a_base[g] + (int64_t)i * nch),
                        (int)(b_base[g] + (int64_t)j * nch), nch});
              if (count) m.tc_tiles += (int64_t)nb * nb;
            }
            close(TC);
            group.clear();
            group_chunks = 0;
          };
          for (int f : done) {
            const int be = block_end(f), mm = m.f_m[f];
            const int64_t need = 2 * (int64_t)((mm - be + 127) / 128) * ((be - k2 + 31) / 32);
            if (group_chunks + need > m.tc_img_chunks) flush();
            group.push_back(f);
            group_chunks += need;
            const double rest = (double)(mm - be);
            if (count) {
              m.gemm_flops += 2.0 * rest * rest * (be - k2);
              m.outer_flops += 2.0 * rest * rest * (be - k2);
            }
            if (window) m.window_tc_flops += 2.0 * rest * rest * (be - k2);
          }
          flush();
        } else {
          Launch OG = open(L_GEMM, l, k2);
          for (int f : done) {
            const int be = block_end(f), mm = m.f_m[f];
            for (int rb = be; rb < mm; rb += GEMM_TILE)
              for (int cb = be; cb < mm; cb += GEMM_TILE) push({f, rb, cb, mm, mm, k2, be - k2});
          }
          close(OG);
        }
      }
    }
  }
}

// (re)upload the work-item array of the schedules
void upload_work(Mesh& m, cudaStream_t s) {
  const size_t need = m.work.size() ? m.work.size() : 1;
  if (!m.ft.work || m.work_cap < need) {
    m.ft.work = m.arena.make<int32_t>(need);
    m.work_cap = need;
  }
  if (!m.work.empty())
    VIV_CUDA(cudaMemcpyAsync(m.ft.work, m.work.data(), m.work.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  if (!m.d_blk_front) {
    m.d_blk_front = m.arena.make<uint8_t>(std::max<size_t>(1, m.blk_front.size()));
    m.d_inv_items_blk = m.arena.make<int32_t>(std::max<size_t>(1, m.inv_items.size()));
  }
  if (!m.blk_front.empty())
    VIV_CUDA(cudaMemcpyAsync(m.d_blk_front, m.blk_front.data(), m.blk_front.size(), cudaMemcpyHostToDevice, s));
  if (!m.inv_items_blk.empty())
    VIV_CUDA(cudaMemcpyAsync(m.d_inv_items_blk, m.inv_items_blk.data(), m.inv_items_blk.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
  if (m.mc_cap < std::max<size_t>(1, m.mc_fwd.size())) {
    m.mc_cap = std::max<size_t>(1, m.mc_fwd.size());
    m.d_mc_fwd = m.arena.make<int32_t>(m.mc_cap);
    m.d_mc_bwd = m.arena.make<int32_t>(m.mc_cap);
  }
  if (!m.mc_fwd.empty()) {
    VIV_CUDA(cudaMemcpyAsync(m.d_mc_fwd, m.mc_fwd.data(), m.mc_fwd.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    VIV_CUDA(cudaMemcpyAsync(m.d_mc_bwd, m.mc_bwd.data(), m.mc_bwd.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  VIV_CUDA(cudaStreamSynchronize(s));
  m.sched_version += 1;
}

void upload_mesh(Mesh& m, cudaStream_t s) {
  DeviceArena& A = m.arena;
  m.d_X = A.upload(m.X, s);
  m.d_conn = A.upload(m.conn, s);
  m.d_wrap = A.upload(m.wrap, s);
  m.d_mid_parent = A.upload(m.mid_parent, s);
  m.d_face_wrap = A.upload(m.face_wrap, s);
  if (m.dim == 3) upload_hex_tables(m, s);
  m.d_tags = A.upload(m.tags, s);
  m.d_faces = A.upload(m.faces, s);
  m.d_node_dof = A.upload(m.node_dof, s);
  m.d_delta_dof = A.upload(m.delta_dof, s);
  m.d_row_ptr = A.upload(m.row_ptr, s);
  m.d_col = A.upload(m.col, s);
  m.d_e2nz = A.upload(m.e2nz, s);
  m.d_f2nz = A.upload(m.f2nz, s);
  m.d_color_elems = A.upload(m.color_elems, s);
  m.d_fcolor_faces = A.upload(m.fcolor_faces, s);
  m.d_level_fronts = A.upload(m.level_fronts, s);
  m.d_inv_items = A.upload(m.inv_items, s);
  m.d_solve_fused = A.upload(m.solve_fused, s);
  m.d_fg_items = A.upload(m.fg_items, s);
  m.d_bg_items = A.upload(m.bg_items, s);
  m.d_bc_col = A.upload(m.bc_col, s);
  m.d_bc_q = A.upload(m.bc_q, s);
  m.d_bb_row = A.upload(m.bb_row, s);
  m.d_bb_q = A.upload(m.bb_q, s);
  FrontTables& t = m.ft;
  t.n_fronts = m.n_fronts;
  t.off = A.upload(m.f_off, s);
  t.m = A.upload(m.f_m, s);
  t.p = A.upload(m.f_p, s);
  t.first = A.upload(m.f_first, s);
  t.idx_off = A.upload(m.f_idx_off, s);
  t.idx = A.upload(m.f_idx, s);
  t.nz_off = A.upload(m.f_nz_off, s);
  t.nz_csr = A.upload(m.f_nz_csr, s);
  t.nz_pos = A.upload(m.f_nz_pos, s);
  t.child_off = A.upload(m.f_child_off, s);
  t.child = A.upload(m.f_child, s);
  t.ea_off = A.upload(m.f_ea_off, s);
  t.ea = A.upload(m.f_ea, s);
  t.parent = A.upload(m.f_parent, s);
  t.vec_off = A.upload(m.f_vec_off, s);
  t.piv_off = A.upload(m.f_piv_off, s);
  t.col_nz = A.upload(m.f_col_nz, s);
  t.col_nz_off = A.upload(m.f_col_nz_off, s);
  upload_work(m, s);
  VIV_CUDA(cudaStreamSynchronize(s));
}

}  // namespace viv
