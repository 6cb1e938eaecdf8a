// Host-side topology of the SLDM discretisation (Sec. II-B): RWG edges with
// T+/T-, object ranges, barycentric refinement, BC coefficients (CSC),
// touching-pair lists for singularity extraction and the sparsity of the
// Gram matrix I_x.  Integer/combinatorial work only; the geometry and every
// integral are computed on the device (fill.cu).
#include <algorithm>
#include <array>
#include <cmath>
#include <unordered_map>

#include "internal.h"

namespace sldm {

namespace {

struct DirInfo {
  int32_t t, i;
};

inline uint64_t key2(int64_t a, int64_t b) { return (uint64_t(a) << 32) | uint64_t(b); }

// Builds undirected edges of an oriented closed triangle list.  Returns false
// (with msg) if it is not an oriented 2-manifold or not closed.
bool build_edges(const std::vector<int64_t>& tv, int64_t nt, const std::vector<int32_t>& tobj,
                 std::vector<int64_t>& uv, std::vector<int32_t>& tp, std::vector<int32_t>& tm,
                 std::vector<int32_t>& tedge, std::vector<int8_t>& tsign,
                 std::unordered_map<uint64_t, DirInfo>& dir, std::string& msg) {
  dir.clear();
  dir.reserve(size_t(nt) * 3 * 2);
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      int64_t a = tv[t * 3 + (i + 1) % 3], b = tv[t * 3 + (i + 2) % 3];
      auto r = dir.emplace(key2(a, b), DirInfo{int32_t(t), i});
      if (!r.second) {
        msg = "mesh is not an oriented 2-manifold (directed edge used twice)";
        return false;
      }
    }
  struct K {
    int32_t obj;
    int64_t u, v;
  };
  std::vector<K> keys;
  keys.reserve(dir.size() / 2);
  for (auto& kv : dir) {
    int64_t a = int64_t(kv.first >> 32), b = int64_t(kv.first & 0xffffffffu);
    if (a < b) {
      auto it = dir.find(key2(b, a));
      if (it == dir.end()) {
        msg = "mesh is not closed (edge with one triangle)";
        return false;
      }
      if (tobj[kv.second.t] != tobj[it->second.t]) {
        msg = "an edge joins two objects (objects must be disjoint)";
        return false;
      }
      keys.push_back({tobj[kv.second.t], a, b});
    }
  }
  if (keys.size() * 2 != dir.size()) {
    msg = "mesh is not closed";
    return false;
  }
  std::sort(keys.begin(), keys.end(), [](const K& x, const K& y) {
    if (x.obj != y.obj) return x.obj < y.obj;
    if (x.u != y.u) return x.u < y.u;
    return x.v < y.v;
  });
  size_t ne = keys.size();
  uv.assign(ne * 2, 0);
  tp.assign(ne, 0);
  tm.assign(ne, 0);
  tedge.assign(size_t(nt) * 3, -1);
  tsign.assign(size_t(nt) * 3, 0);
  for (size_t n = 0; n < ne; ++n) {
    uv[2 * n] = keys[n].u;
    uv[2 * n + 1] = keys[n].v;
    DirInfo p = dir[key2(keys[n].u, keys[n].v)];
    DirInfo q = dir[key2(keys[n].v, keys[n].u)];
    tp[n] = p.t;
    tm[n] = q.t;
    tedge[size_t(p.t) * 3 + p.i] = int32_t(n);
    tsign[size_t(p.t) * 3 + p.i] = 1;
    tedge[size_t(q.t) * 3 + q.i] = int32_t(n);
    tsign[size_t(q.t) * 3 + q.i] = -1;
  }
  return true;
}

// The same edges, numbering and T+/T- as build_edges, found by sorting the
// directed edges instead of hashing them (no map is kept): used for the
// barycentric refinement, whose 18 nt directed edges dominate the topology.
bool build_edges_sorted(const std::vector<int64_t>& tv, int64_t nt, const std::vector<int32_t>& tobj,
                        std::vector<int64_t>& uv, std::vector<int32_t>& tp, std::vector<int32_t>& tm,
                        std::vector<int32_t>& tedge, std::vector<int8_t>& tsign, std::string& msg) {
  struct D {
    uint64_t key;  // (min, max) vertex pair
    int32_t t;
    int8_t i, fwd;  // local edge index; 1 when the triangle runs min -> max
  };
  std::vector<D> d(size_t(nt) * 3);
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) {
      const int64_t a = tv[t * 3 + (i + 1) % 3], b = tv[t * 3 + (i + 2) % 3];
      d[size_t(t) * 3 + i] = D{a < b ? key2(a, b) : key2(b, a), int32_t(t), int8_t(i), int8_t(a < b)};
    }
  std::sort(d.begin(), d.end(), [](const D& x, const D& y) {
    if (x.key != y.key) return x.key < y.key;
    return x.fwd > y.fwd;  // the forward (T+) entry first
  });
  const size_t nd = d.size();
  // a directed edge used twice: two entries of one pair in the same direction
  for (size_t k = 0; k + 1 < nd; ++k)
    if (d[k].key == d[k + 1].key && d[k].fwd == d[k + 1].fwd) {
      msg = "mesh is not an oriented 2-manifold (directed edge used twice)";
      return false;
    }
  // closed: every pair appears once in each direction
  struct E {
    int32_t obj;
    int64_t u, v;
    size_t k;  // index of the forward entry in d
  };
  std::vector<E> edges;
  edges.reserve(nd / 2);
  for (size_t k = 0; k < nd;) {
    if (k + 1 >= nd || d[k + 1].key != d[k].key) {
      msg = "mesh is not closed (edge with one triangle)";
      return false;
    }
    if (tobj[d[k].t] != tobj[d[k + 1].t]) {
      msg = "an edge joins two objects (objects must be disjoint)";
      return false;
    }
    edges.push_back({tobj[d[k].t], int64_t(d[k].key >> 32), int64_t(d[k].key & 0xffffffffu), k});
    k += 2;
  }
  std::sort(edges.begin(), edges.end(), [](const E& x, const E& y) {
    if (x.obj != y.obj) return x.obj < y.obj;
    if (x.u != y.u) return x.u < y.u;
    return x.v < y.v;
  });
  const size_t ne = edges.size();
  uv.assign(ne * 2, 0);
  tp.assign(ne, 0);
  tm.assign(ne, 0);
  tedge.assign(size_t(nt) * 3, -1);
  tsign.assign(size_t(nt) * 3, 0);
  for (size_t n = 0; n < ne; ++n) {
    const D& p = d[edges[n].k];      // u -> v: T+
    const D& q = d[edges[n].k + 1];  // v -> u: T-
    uv[2 * n] = edges[n].u;
    uv[2 * n + 1] = edges[n].v;
    tp[n] = p.t;
    tm[n] = q.t;
    tedge[size_t(p.t) * 3 + p.i] = int32_t(n);
    tsign[size_t(p.t) * 3 + p.i] = 1;
    tedge[size_t(q.t) * 3 + q.i] = int32_t(n);
    tsign[size_t(q.t) * 3 + q.i] = -1;
  }
  return true;
}

}  // namespace

void build_host_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* obj,
                     HostMesh& hm) {
  SLDM_REQUIRE(xyz && tri && nv > 0 && nt > 0, SLDM_EINVAL, "mesh_create: empty mesh or null arrays");
  SLDM_REQUIRE(nt < (int64_t(1) << 28) && nv < (int64_t(1) << 30), SLDM_EINVAL, "mesh_create: mesh too large");
  hm.nv = nv;
  hm.nt = nt;
  hm.xyz.assign(xyz, xyz + nv * 3);
  hm.tri.assign(tri, tri + nt * 3);
  hm.obj.assign(size_t(nt), 0);
  if (obj) hm.obj.assign(obj, obj + nt);
  for (int64_t t = 0; t < nt; ++t) {
    if (t > 0) SLDM_REQUIRE(hm.obj[t] >= hm.obj[t - 1], SLDM_EINVAL, "obj_id must be non-decreasing");
    SLDM_REQUIRE(hm.obj[t] >= 0, SLDM_EINVAL, "obj_id must be >= 0");
    for (int i = 0; i < 3; ++i)
      SLDM_REQUIRE(hm.tri[t * 3 + i] >= 0 && hm.tri[t * 3 + i] < nv, SLDM_EINVAL, "triangle vertex index out of range");
    const double* a = &xyz[3 * hm.tri[t * 3]];
    const double* b = &xyz[3 * hm.tri[t * 3 + 1]];
    const double* c = &xyz[3 * hm.tri[t * 3 + 2]];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double area2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double scale = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    SLDM_REQUIRE(area2 > 1e-12 * scale, SLDM_EINVAL, "degenerate triangle " + std::to_string(t));
  }
  // objects: contiguous ids 0..nobj-1 (empty ids are not allowed)
  hm.nobj = int64_t(hm.obj.back()) + 1;
  hm.tri_begin.assign(size_t(hm.nobj) + 1, 0);
  {
    int64_t t = 0;
    for (int64_t o = 0; o < hm.nobj; ++o) {
      hm.tri_begin[o] = int32_t(t);
      while (t < nt && hm.obj[t] == o) ++t;
      SLDM_REQUIRE(t > hm.tri_begin[o] + 3, SLDM_EINVAL, "object " + std::to_string(o) + " has too few triangles");
    }
    hm.tri_begin[hm.nobj] = int32_t(nt);
  }
  // vertices belong to one object only
  {
    std::vector<int32_t> vobj(static_cast<size_t>(nv), -1);
    for (int64_t t = 0; t < nt; ++t)
      for (int i = 0; i < 3; ++i) {
        int32_t v = hm.tri[t * 3 + i];
        SLDM_REQUIRE(vobj[v] < 0 || vobj[v] == hm.obj[t], SLDM_EINVAL, "a vertex is shared by two objects");
        vobj[v] = hm.obj[t];
      }
  }
  std::vector<int64_t> tv(hm.tri.begin(), hm.tri.end());
  std::unordered_map<uint64_t, DirInfo> dir;
  std::string msg;
  SLDM_REQUIRE(build_edges(tv, nt, hm.obj, hm.uv, hm.tplus, hm.tminus, hm.tri_edge, hm.tri_sign, dir, msg),
               SLDM_EINVAL, msg);
  hm.ne = int64_t(hm.tplus.size());
  // outward normals: a closed oriented surface encloses the signed volume
  // sum over its triangles of a . (b x c) / 6, positive when every normal points
  // out (vertices taken relative to the object's first vertex against cancellation)
  for (int64_t o = 0; o < hm.nobj; ++o) {
    const double* r = &xyz[3 * hm.tri[3 * int64_t(hm.tri_begin[o])]];
    double vol = 0;
    for (int64_t t = hm.tri_begin[o]; t < hm.tri_begin[o + 1]; ++t) {
      double p[3][3];
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) p[i][d] = xyz[3 * hm.tri[3 * t + i] + d] - r[d];
      vol += p[0][0] * (p[1][1] * p[2][2] - p[1][2] * p[2][1]) + p[0][1] * (p[1][2] * p[2][0] - p[1][0] * p[2][2]) +
             p[0][2] * (p[1][0] * p[2][1] - p[1][1] * p[2][0]);
    }
    SLDM_REQUIRE(vol > 0, SLDM_EINVAL,
                 "object " + std::to_string(o) + " is oriented inward (its normals enclose a negative volume)");
  }
  {
    double acc = 0;
    for (int64_t n = 0; n < hm.ne; ++n) {
      const double* a = &xyz[3 * hm.uv[2 * n]];
      const double* b = &xyz[3 * hm.uv[2 * n + 1]];
      acc += std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
    }
    hm.ell = acc / double(hm.ne);
  }
  hm.edge_begin.assign(size_t(hm.nobj) + 1, 0);
  for (int64_t n = 0, o = 0; o <= hm.nobj; ++o) {
    while (n < hm.ne && hm.obj[hm.tplus[n]] < o) ++n;
    hm.edge_begin[o] = int32_t(n);
  }
  const int64_t nv_ = nv, ne_ = hm.ne;

  // ---------------- barycentric refinement
  // child 6t+k of triangle (a, b, c): (a, m_ab, g) (m_ab, b, g) (b, m_bc, g) (m_bc, c, g) (c, m_ca, g) (m_ca, a, g)
  std::vector<int64_t> bv(size_t(6 * nt) * 3);
  std::vector<int32_t> bobj(size_t(6 * nt));
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = hm.tri[3 * t], b = hm.tri[3 * t + 1], c = hm.tri[3 * t + 2];
    int64_t mab = nv_ + hm.tri_edge[3 * t + 2], mbc = nv_ + hm.tri_edge[3 * t + 0], mca = nv_ + hm.tri_edge[3 * t + 1];
    int64_t g = nv_ + ne_ + t;
    int64_t ch[6][3] = {{a, mab, g}, {mab, b, g}, {b, mbc, g}, {mbc, c, g}, {c, mca, g}, {mca, a, g}};
    for (int k = 0; k < 6; ++k) {
      for (int j = 0; j < 3; ++j) bv[(6 * t + k) * 3 + j] = ch[k][j];
      bobj[6 * t + k] = hm.obj[t];
    }
  }
  std::vector<int64_t> buv;
  std::vector<int32_t> btp, btm;
  SLDM_REQUIRE(build_edges_sorted(bv, 6 * nt, bobj, buv, btp, btm, hm.btri_edge, hm.btri_sign, msg), SLDM_EINVAL,
               "barycentric mesh: " + msg);
  hm.nbe = int64_t(btp.size());
  hm.bedge_begin.assign(size_t(hm.nobj) + 1, 0);
  for (int64_t k = 0, o = 0; o <= hm.nobj; ++o) {
    while (k < hm.nbe && bobj[btp[k]] < o) ++k;
    hm.bedge_begin[o] = int32_t(k);
  }

  // ---------------- BC functions (columns of C)
  auto shared_bedge = [&](int32_t c1, int32_t c2) -> int32_t {
    for (int j = 0; j < 3; ++j) {
      int32_t k = hm.btri_edge[size_t(c1) * 3 + j];
      if (btp[k] == c2 || btm[k] == c2) return k;
    }
    throw Error{SLDM_EINVAL, "internal: barycentric children not adjacent"};
  };
  auto tri_pos = [&](int32_t t, int64_t v) -> int {
    for (int i = 0; i < 3; ++i)
      if (hm.tri[3 * t + i] == v) return i;
    throw Error{SLDM_EINVAL, "internal: vertex not in triangle"};
  };
  hm.bc_ptr.assign(size_t(hm.ne) + 1, 0);
  hm.bc_row.clear();
  hm.bc_val.clear();
  std::vector<std::pair<int32_t, double>> col;
  for (int64_t n = 0; n < hm.ne; ++n) {
    col.clear();
    auto add_flux = [&](int32_t from, int32_t to, double flux) {
      int32_t k = shared_bedge(from, to);
      double s = (btp[k] == from) ? 1.0 : -1.0;
      col.push_back({k, s * flux});
    };
    int64_t u = hm.uv[2 * n], v = hm.uv[2 * n + 1];
    for (int side = 0; side < 2; ++side) {
      int64_t x = side == 0 ? u : v, y0 = side == 0 ? v : u;
      double sgn = side == 0 ? 1.0 : -1.0;
      // counter-clockwise ring of triangles around x starting with edge (x, y0)
      std::vector<int32_t> children;
      int64_t y = y0;
      for (int guard = 0;; ++guard) {
        SLDM_REQUIRE(guard < 4096, SLDM_EINVAL, "vertex ring did not close");
        auto it = dir.find(key2(x, y));
        SLDM_REQUIRE(it != dir.end(), SLDM_EINVAL, "vertex ring broken");
        int32_t t = it->second.t;
        int p = tri_pos(t, x);
        children.push_back(6 * t + 2 * p);            // (x, m(x, y_k), g)
        children.push_back(6 * t + (2 * p + 5) % 6);  // (m(x, y_k+1), x, g)
        y = hm.tri[3 * t + (p + 2) % 3];
        if (y == y0) break;
      }
      int64_t N = int64_t(children.size()) / 2;
      // flux from child i to child i+1 around x: sgn (i + 1 - N) / (2 N)
      for (int64_t i = 0; i + 1 < 2 * N; ++i) {
        int64_t num = i + 1 - N;
        if (num != 0) add_flux(children[i], children[i + 1], sgn * double(num) / double(2 * N));
      }
    }
    // the two halves of the dual edge, 1/2 each, from the cell of u to the cell of v
    int32_t tp = hm.tplus[n], tm = hm.tminus[n];
    int pu = tri_pos(tp, u), pv = tri_pos(tp, v);
    add_flux(6 * tp + 2 * pu, 6 * tp + (2 * pv + 5) % 6, 0.5);
    int pu2 = tri_pos(tm, u), pv2 = tri_pos(tm, v);
    add_flux(6 * tm + (2 * pu2 + 5) % 6, 6 * tm + 2 * pv2, 0.5);
    std::sort(col.begin(), col.end());
    for (auto& e : col) {
      hm.bc_row.push_back(e.first);
      hm.bc_val.push_back(e.second);
    }
    hm.bc_ptr[n + 1] = int32_t(hm.bc_row.size());
  }

  // ---------------- touching pairs
  std::vector<std::vector<int32_t>> vtri(static_cast<size_t>(nv));
  for (int64_t t = 0; t < nt; ++t)
    for (int i = 0; i < 3; ++i) vtri[hm.tri[3 * t + i]].push_back(int32_t(t));
  hm.touchL_a.clear();
  hm.touchL_b.clear();
  hm.touchK_a.clear();
  hm.touchK_c.clear();
  std::vector<int32_t> nb;
  for (int64_t t = 0; t < nt; ++t) {
    nb.clear();
    for (int i = 0; i < 3; ++i)
      for (int32_t s : vtri[hm.tri[3 * t + i]]) nb.push_back(s);
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    for (int32_t s : nb) {
      hm.touchL_a.push_back(int32_t(t));
      hm.touchL_b.push_back(s);
      if (s == t) continue;
      for (int k = 0; k < 6; ++k) {
        int p = k / 2;
        int pvert = (k % 2 == 0) ? p : (p + 1) % 3;          // child's primal vertex
        int medge = (p + 2) % 3;                             // child's midpoint edge
        int32_t cv = hm.tri[3 * s + pvert], ce = hm.tri_edge[3 * s + medge];
        bool touch = false;
        for (int i = 0; i < 3; ++i) touch |= (hm.tri[3 * t + i] == cv) || (hm.tri_edge[3 * t + i] == ce);
        if (touch) {
          hm.touchK_a.push_back(int32_t(t));
          hm.touchK_c.push_back(6 * s + k);
        }
      }
    }
  }

  // ---------------- I_x sparsity and contribution lists
  // row m (an RWG) -> its nonzero columns n (BC functions), each with the list of
  // contributions (triangle, child, i, j, coefficient) that the device sums
  // C transposed (CSR by barycentric edge, BC columns in increasing order): bary edge -> (n, coef)
  std::vector<int32_t> rb_ptr(size_t(hm.nbe) + 1, 0), rb_n(hm.bc_row.size());
  std::vector<double> rb_val(hm.bc_row.size());
  for (int32_t r : hm.bc_row) ++rb_ptr[size_t(r) + 1];
  for (int64_t k = 0; k < hm.nbe; ++k) rb_ptr[k + 1] += rb_ptr[k];
  {
    std::vector<int32_t> fill(rb_ptr.begin(), rb_ptr.end() - 1);
    for (int64_t n = 0; n < hm.ne; ++n)
      for (int32_t q = hm.bc_ptr[n]; q < hm.bc_ptr[n + 1]; ++q) {
        const int32_t at = fill[hm.bc_row[q]]++;
        rb_n[at] = int32_t(n);
        rb_val[at] = hm.bc_val[q];
      }
  }
  hm.ix_ptr.assign(size_t(hm.ne) + 1, 0);
  hm.ix_col.clear();
  hm.ixc_ptr.assign(1, 0);
  hm.ixc_tri.clear(); hm.ixc_child.clear(); hm.ixc_i.clear(); hm.ixc_j.clear(); hm.ixc_coef.clear();
  // per row m: the contributions in generation order, grouped by column with a
  // stable sort (so each column keeps the order in which they were generated)
  struct Contrib { int32_t n, t, c, i, j; double coef; };
  std::vector<Contrib> row;
  {
    size_t total = 0;  // contributions of every row, to size the outputs once
    for (int64_t m = 0; m < hm.ne; ++m)
      for (int32_t t : {hm.tplus[m], hm.tminus[m]})
        for (int k = 0; k < 18; ++k) {
          const int32_t be = hm.btri_edge[size_t(6 * t) * 3 + k];
          total += size_t(rb_ptr[be + 1] - rb_ptr[be]);
        }
    for (auto* v : {&hm.ixc_tri, &hm.ixc_child, &hm.ixc_i, &hm.ixc_j}) v->reserve(total);
    hm.ixc_coef.reserve(total);
  }
  for (int64_t m = 0; m < hm.ne; ++m) {
    row.clear();
    for (int32_t t : {hm.tplus[m], hm.tminus[m]}) {
      int i = -1;
      for (int q = 0; q < 3; ++q)
        if (hm.tri_edge[3 * t + q] == m) i = q;
      for (int k = 0; k < 6; ++k) {
        int32_t c = 6 * t + k;
        for (int j = 0; j < 3; ++j) {
          int32_t be = hm.btri_edge[size_t(c) * 3 + j];
          for (int32_t q = rb_ptr[be]; q < rb_ptr[be + 1]; ++q) row.push_back({rb_n[q], t, c, i, j, rb_val[q]});
        }
      }
    }
    std::stable_sort(row.begin(), row.end(), [](const Contrib& x, const Contrib& y) { return x.n < y.n; });
    for (size_t q = 0; q < row.size(); ++q) {
      const Contrib& cb = row[q];
      if (q == 0 || cb.n != row[q - 1].n) {
        if (q > 0) hm.ixc_ptr.push_back(int32_t(hm.ixc_tri.size()));
        hm.ix_col.push_back(cb.n);
      }
      hm.ixc_tri.push_back(cb.t);
      hm.ixc_child.push_back(cb.c);
      hm.ixc_i.push_back(cb.i);
      hm.ixc_j.push_back(cb.j);
      hm.ixc_coef.push_back(cb.coef);
    }
    if (!row.empty()) hm.ixc_ptr.push_back(int32_t(hm.ixc_tri.size()));
    hm.ix_ptr[m + 1] = int32_t(hm.ix_col.size());
  }
}

}  // namespace sldm
