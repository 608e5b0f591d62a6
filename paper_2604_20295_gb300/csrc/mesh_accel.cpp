// mesh_accel.cpp -- host-side acceleration structure for contact with closed triangle meshes.
//
// ETac finds contact with signed distance fields between the pad nodes and object meshes
// (Sec. III-A, "Overview").  A contact query must find, for a node q inside the mesh's
// bounding box, the nearest surface point c and the sign of the distance.  This file builds
// what such a query reads: a uniform grid over the bounding box whose cells either settle
// the sign for every point they hold (no surface within the cell's circumscribed ball) or
// list the triangles that can hold the nearest point of any point in the cell, plus, per
// triangle, its vertices, face normal and the pseudo-normals of its edges and vertices that
// decide the sign at the nearest feature (Baerentzen and Aanaes, "Signed distance
// computation using the angle weighted pseudonormal", IEEE TVCG 2005).
//
// Why the candidate list is complete.  Let o be a cell's centre, r its half-diagonal and
// d = min_t dist(o, t).  For a point q of the cell (|q - o| <= r) with nearest triangle t*:
// dist(q, t*) <= dist(q, t_o) <= d + r, so dist(o, t*) <= dist(q, t*) + r <= d + 2r.  Every
// triangle within d + 2r of the centre is therefore listed.  When d > r no surface point
// lies in the ball of radius r about o, which contains the cell, so the whole cell has the
// sign of its centre.
//
// All arithmetic is FP64 on the host; the arrays handed out are FP32 (vertices, normals)
// and int32 (cells, candidates), laid out for 16-byte loads.  Cells are processed by a
// pool of threads over contiguous cell ranges, so the output does not depend on the
// thread count.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "etac.h"

namespace etac {
void set_context_free_error(const std::string& msg);   // api.cu: read by etac_last_error(NULL)
}

struct etac_mesh_accel {
  etac_mesh_accel_view view;
  std::vector<int32_t> cell_start;
  std::vector<uint8_t> cell_kind;
  std::vector<int32_t> cand;
  std::vector<float> tri;
  std::vector<float> pseudo;
};

namespace {

struct V3 {
  double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline V3 unit(V3 a) {
  double L = std::sqrt(dot(a, a));
  return L > 0 ? (1.0 / L) * a : V3{0, 0, 0};
}

// nearest-feature codes, matching the pseudo-normal order of the view
enum { F_FACE = -1, F_AB = 0, F_BC = 1, F_CA = 2, F_A = 3, F_B = 4, F_C = 5 };

struct Nearest {
  V3 c;
  int feat;
};

// Nearest point of triangle (a, b, c) to p by the Voronoi regions of its vertices, edges and
// face, tested in that order (Ericson, "Real-Time Collision Detection", 2005, Sec. 5.1.5).
Nearest nearest_on_triangle(V3 p, V3 a, V3 b, V3 c) {
  V3 ab = b - a, ac = c - a, ap = p - a;
  double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0 && d2 <= 0) return {a, F_A};
  V3 bp = p - b;
  double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0 && d4 <= d3) return {b, F_B};
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0) return {a + (d1 / (d1 - d3)) * ab, F_AB};
  V3 cp = p - c;
  double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0 && d5 <= d6) return {c, F_C};
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0) return {a + (d2 / (d2 - d6)) * ac, F_CA};
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0)
    return {b + ((d4 - d3) / ((d4 - d3) + (d5 - d6))) * (c - b), F_BC};
  double s = 1.0 / (va + vb + vc);
  return {a + (vb * s) * ab + (vc * s) * ac, F_FACE};
}

struct MeshD {
  std::vector<V3> v;                 // vertices
  std::vector<int32_t> t;            // [T*3]
  std::vector<V3> fn;                // [T] unit face normals
  std::vector<V3> pn;                // [T*6] pseudo-normals: edges ab, bc, ca, vertices a, b, c
};

etac_status fail(const std::string& m, etac_status st = ETAC_ERR_INVALID_ARG) {
  etac::set_context_free_error("mesh acceleration structure: " + m);
  return st;
}

etac_status load_mesh(const etac_mesh_desc* d, MeshD* m) {
  if (!d->verts || !d->tris) return fail("NULL vertex or triangle array");
  if (d->num_verts < 4 || d->num_tris < 4) return fail("a closed mesh needs >= 4 vertices and triangles");
  const int V = d->num_verts, T = d->num_tris;
  m->v.resize(V);
  for (int i = 0; i < V; ++i) {
    m->v[i] = {d->verts[3 * i], d->verts[3 * i + 1], d->verts[3 * i + 2]};
    if (!std::isfinite(m->v[i].x) || !std::isfinite(m->v[i].y) || !std::isfinite(m->v[i].z))
      return fail("vertex " + std::to_string(i) + " is not finite");
  }
  m->t.assign(d->tris, d->tris + 3 * (size_t)T);
  for (size_t k = 0; k < m->t.size(); ++k)
    if (m->t[k] < 0 || m->t[k] >= V) return fail("triangle " + std::to_string(k / 3) + " has a vertex index out of range");
  // closed and consistently oriented: each directed edge once, and its reverse once
  std::unordered_map<uint64_t, int32_t> edge;   // directed edge -> triangle
  edge.reserve(3 * (size_t)T * 2);
  auto key = [](int32_t u, int32_t w) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)w; };
  for (int t = 0; t < T; ++t)
    for (int e = 0; e < 3; ++e) {
      int32_t u = m->t[3 * t + e], w = m->t[3 * t + (e + 1) % 3];
      if (u == w) return fail("triangle " + std::to_string(t) + " repeats a vertex");
      if (!edge.emplace(key(u, w), t).second)
        return fail("directed edge (" + std::to_string(u) + ", " + std::to_string(w) +
                    ") occurs twice: the mesh is not consistently wound or not manifold");
    }
  m->fn.resize(T);
  for (int t = 0; t < T; ++t) {
    V3 a = m->v[m->t[3 * t]], b = m->v[m->t[3 * t + 1]], c = m->v[m->t[3 * t + 2]];
    V3 n = cross(b - a, c - a);
    double L = std::sqrt(dot(n, n));
    double scale = std::max({std::sqrt(dot(b - a, b - a)), std::sqrt(dot(c - a, c - a)), 1e-30});
    if (!(L > 1e-12 * scale * scale)) return fail("triangle " + std::to_string(t) + " has zero area");
    m->fn[t] = (1.0 / L) * n;
  }
  // pseudo-normals
  std::vector<V3> vsum(V, V3{0, 0, 0});
  for (int t = 0; t < T; ++t)
    for (int e = 0; e < 3; ++e) {
      V3 p = m->v[m->t[3 * t + e]], q = m->v[m->t[3 * t + (e + 1) % 3]],
         r = m->v[m->t[3 * t + (e + 2) % 3]];
      double ang = std::acos(std::max(-1.0, std::min(1.0, dot(unit(q - p), unit(r - p)))));
      vsum[m->t[3 * t + e]] = vsum[m->t[3 * t + e]] + ang * m->fn[t];
    }
  m->pn.resize(6 * (size_t)T);
  for (int t = 0; t < T; ++t)
    for (int e = 0; e < 3; ++e) {
      int32_t u = m->t[3 * t + e], w = m->t[3 * t + (e + 1) % 3];
      auto it = edge.find(key(w, u));
      if (it == edge.end())
        return fail("edge (" + std::to_string(u) + ", " + std::to_string(w) +
                    ") has no opposite triangle: the mesh is not closed");
      m->pn[6 * t + e] = unit(m->fn[t] + m->fn[it->second]);
      m->pn[6 * t + 3 + e] = unit(vsum[u]);
    }
  return ETAC_OK;
}

}  // namespace

extern "C" {

etac_status etac_mesh_accel_build(etac_mesh_accel** out, const etac_mesh_desc* desc) {
  if (!out || !desc) return fail("NULL argument");
  *out = nullptr;
  const int grid = desc->grid == 0 ? 32 : desc->grid;
  if (grid < 1 || grid > 512) return fail("grid must be in [1, 512] (0 = 32)");
  try {
    MeshD m;
    etac_status st = load_mesh(desc, &m);
    if (st != ETAC_OK) return st;
    const int T = desc->num_tris;
    V3 lo = m.v[0], hi = m.v[0];
    for (const V3& p : m.v) {
      lo = {std::min(lo.x, p.x), std::min(lo.y, p.y), std::min(lo.z, p.z)};
      hi = {std::max(hi.x, p.x), std::max(hi.y, p.y), std::max(hi.z, p.z)};
    }
    // the grid is defined by its FP32 origin and cell edge, the values a query reads
    lo = {(double)(float)lo.x, (double)(float)lo.y, (double)(float)lo.z};
    const double ext[3] = {hi.x - lo.x, hi.y - lo.y, hi.z - lo.z};
    const double cell = (double)(float)(std::max({ext[0], ext[1], ext[2]}) / grid);
    if (!(cell > 0)) return fail("the mesh has an empty bounding box");
    // one extra cell along each axis covers the box's far faces after FP32 rounding
    int dims[3];
    for (int a = 0; a < 3; ++a) dims[a] = (int)std::floor(ext[a] / cell) + 1;
    const int64_t C = (int64_t)dims[0] * dims[1] * dims[2];
    if (C > (int64_t(1) << 24)) return fail("grid has more than 2^24 cells");
    const double r = 0.5 * cell * std::sqrt(3.0);
    const double slack = 1e-5 * cell + 1e-6;

    etac_mesh_accel* acc = new etac_mesh_accel();
    acc->cell_kind.assign((size_t)C, ETAC_CELL_OUTSIDE);
    std::vector<int32_t> count((size_t)C, 0);

    unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    nth = (unsigned)std::min<int64_t>(nth, C);
    std::vector<std::vector<int32_t>> part(nth);
    std::vector<int> part_err(nth, 0);
    auto work = [&](unsigned w) {
      try {
        int64_t c0 = C * w / nth, c1 = C * (w + 1) / nth;
        std::vector<double> dist((size_t)T);
        for (int64_t ci = c0; ci < c1; ++ci) {
          int i = (int)(ci % dims[0]), j = (int)((ci / dims[0]) % dims[1]),
              k = (int)(ci / ((int64_t)dims[0] * dims[1]));
          V3 o = {lo.x + (i + 0.5) * cell, lo.y + (j + 0.5) * cell, lo.z + (k + 0.5) * cell};
          double best = INFINITY;
          int bt = 0;
          Nearest bn{{0, 0, 0}, F_FACE};
          for (int t = 0; t < T; ++t) {
            Nearest nr = nearest_on_triangle(o, m.v[m.t[3 * t]], m.v[m.t[3 * t + 1]],
                                             m.v[m.t[3 * t + 2]]);
            V3 dv = o - nr.c;
            dist[t] = std::sqrt(dot(dv, dv));
            if (dist[t] < best) { best = dist[t]; bt = t; bn = nr; }
          }
          V3 nF = bn.feat == F_FACE ? m.fn[bt] : m.pn[6 * (size_t)bt + bn.feat];
          bool inside = dot(o - bn.c, nF) < 0;
          uint8_t kind = best > r + slack ? (inside ? ETAC_CELL_INSIDE : ETAC_CELL_OUTSIDE)
                                          : ETAC_CELL_SURFACE;
          acc->cell_kind[ci] = kind;
          if (kind == ETAC_CELL_OUTSIDE) continue;
          double lim = best + 2 * r + slack;
          int32_t n = 0;
          for (int t = 0; t < T; ++t)
            if (dist[t] <= lim) { part[w].push_back(t); ++n; }
          count[ci] = n;
        }
      } catch (...) {
        part_err[w] = 1;
      }
    };
    std::vector<std::thread> pool;
    for (unsigned w = 1; w < nth; ++w) pool.emplace_back(work, w);
    work(0);
    for (auto& th : pool) th.join();
    for (int e : part_err)
      if (e) { delete acc; return fail("host memory exhausted", ETAC_ERR_OOM); }

    acc->cell_start.resize((size_t)C + 1);
    int64_t total = 0;
    for (int64_t ci = 0; ci < C; ++ci) {
      acc->cell_start[ci] = (int32_t)std::min<int64_t>(total, INT32_MAX);
      total += count[ci];
    }
    if (total > (int64_t(1) << 28)) {
      delete acc;
      return fail("more than 2^28 candidate entries: use a coarser grid");
    }
    acc->cell_start[C] = (int32_t)total;
    acc->cand.reserve((size_t)total);
    for (auto& p : part) acc->cand.insert(acc->cand.end(), p.begin(), p.end());

    acc->tri.assign(16 * (size_t)T, 0.f);
    acc->pseudo.assign(24 * (size_t)T, 0.f);
    for (int t = 0; t < T; ++t) {
      for (int e = 0; e < 3; ++e) {
        const V3& p = m.v[m.t[3 * t + e]];
        float* d = &acc->tri[16 * (size_t)t + 4 * e];
        d[0] = (float)p.x; d[1] = (float)p.y; d[2] = (float)p.z;
      }
      float* nf = &acc->tri[16 * (size_t)t + 12];
      nf[0] = (float)m.fn[t].x; nf[1] = (float)m.fn[t].y; nf[2] = (float)m.fn[t].z;
      for (int f = 0; f < 6; ++f) {
        float* d = &acc->pseudo[24 * (size_t)t + 4 * f];
        const V3& q = m.pn[6 * (size_t)t + f];
        d[0] = (float)q.x; d[1] = (float)q.y; d[2] = (float)q.z;
      }
    }
    etac_mesh_accel_view& v = acc->view;
    std::memset(&v, 0, sizeof v);
    v.origin[0] = (float)lo.x; v.origin[1] = (float)lo.y; v.origin[2] = (float)lo.z;
    v.cell = (float)cell;
    for (int a = 0; a < 3; ++a) v.dims[a] = dims[a];
    v.num_tris = T;
    v.num_cand = total;
    v.cell_start = acc->cell_start.data();
    v.cell_kind = acc->cell_kind.data();
    v.cand = acc->cand.data();
    v.tri = acc->tri.data();
    v.pseudo = acc->pseudo.data();
    *out = acc;
    return ETAC_OK;
  } catch (const std::bad_alloc&) {
    return fail("host memory exhausted", ETAC_ERR_OOM);
  }
}

etac_status etac_mesh_accel_get_view(const etac_mesh_accel* accel, etac_mesh_accel_view* view) {
  if (!accel || !view) return fail("NULL argument");
  *view = accel->view;
  return ETAC_OK;
}

void etac_mesh_accel_destroy(etac_mesh_accel* accel) { delete accel; }

}  // extern "C"
