// mesh_common.cuh -- signed distance to a closed triangle mesh on the GPU, for the object-mesh
// contact of ETac Sec. III-A ("Overview"): the standalone query (mesh_query.cu) and the contact
// step's mesh objects (etac_common.cuh) share these routines.
//
// A mesh arrives as the host-built acceleration structure of mesh_accel.cpp: a uniform grid of
// cells classified OUTSIDE / INSIDE / SURFACE from exact host distances, the candidate
// triangles of every INSIDE and SURFACE cell (they hold the nearest surface point of every
// point of the cell; ascending index), and per triangle its vertices, face normal and the
// pseudo-normals of its edges and vertices.
//
// Two evaluations:
//   mesh_f32: FP32, the nearest point by Voronoi regions (Ericson, "Real-Time Collision
//     Detection", 2005, Sec. 5.1.5) and the sign from the pseudo-normal of the feature that
//     holds it (Baerentzen and Aanaes, IEEE TVCG 2005); also whether a second candidate is
//     within rounding of the nearest with another nearest point (the choice of u_hat is then
//     not settled in FP32);
//   mesh_f64: the same distance in FP64 from the definition (orthogonal projection if it lies
//     in the triangle, barycentric weights >= -1e-12, else the nearest point of the three
//     edge segments, ties to the earlier triangle and edge), for the thin band of nodes whose
//     FP32 sign or choice is not settled.  It reports the feature (face, edge interior,
//     vertex) and the edge direction, which the reverse mode's Hessian needs.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace etac {

enum { MESH_CELL_OUTSIDE = 0, MESH_CELL_INSIDE = 1, MESH_CELL_SURFACE = 2 };

// device view of one mesh's acceleration structure
struct MeshDev {
  float ox, oy, oz, cell;      // object-frame corner of cell (0, 0, 0) and cell edge (mm)
  int nx, ny, nz;              // cells per axis
  float extent;                // largest |x| of the mesh's bounding box (object frame)
  const int32_t* cell_start;   // [C+1]
  const uint8_t* cell_kind;    // [C]
  const int32_t* cand;         // candidate triangles of each cell, ascending
  const float4* tri;           // [T*4]: a, b, c, unit face normal
  const float4* pseudo;        // [T*6]: pseudo-normals of edges ab, bc, ca, vertices a, b, c
};

// The cell of object-frame point p: its index and kind, or -1 when p lies outside the grid
// (or is not finite): outside the mesh.
__device__ __forceinline__ int mesh_cell(const MeshDev& m, float3 p, int* kind) {
  const float rx = (p.x - m.ox) / m.cell, ry = (p.y - m.oy) / m.cell, rz = (p.z - m.oz) / m.cell;
  // comparisons in float first: NaN coordinates fail them and count as outside
  if (!(rx >= 0.f && ry >= 0.f && rz >= 0.f && rx < (float)m.nx && ry < (float)m.ny &&
        rz < (float)m.nz))
    return -1;
  const int ix = min((int)rx, m.nx - 1), iy = min((int)ry, m.ny - 1), iz = min((int)rz, m.nz - 1);
  const int c = (iz * m.ny + iy) * m.nx + ix;
  *kind = m.cell_kind[c];
  return c;
}

// Nearest point of triangle (a, b, c) to p in FP32 by Voronoi regions; feat: -1 face, 0..2
// edges ab, bc, ca, 3..5 vertices a, b, c (the pseudo-normal order).  Returns |p - q|^2.
__device__ __forceinline__ float nearest_on_triangle(float3 p, float3 a, float3 b, float3 c,
                                                     float3* cp, int* feat) {
  const float3 ab = make_float3(b.x - a.x, b.y - a.y, b.z - a.z);
  const float3 ac = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
  const float3 ap = make_float3(p.x - a.x, p.y - a.y, p.z - a.z);
  const float d1 = ab.x * ap.x + ab.y * ap.y + ab.z * ap.z;
  const float d2 = ac.x * ap.x + ac.y * ap.y + ac.z * ap.z;
  float3 q;
  int f;
  if (d1 <= 0.f && d2 <= 0.f) {
    q = a; f = 3;
  } else {
    const float3 bp = make_float3(p.x - b.x, p.y - b.y, p.z - b.z);
    const float d3 = ab.x * bp.x + ab.y * bp.y + ab.z * bp.z;
    const float d4 = ac.x * bp.x + ac.y * bp.y + ac.z * bp.z;
    const float vc = d1 * d4 - d3 * d2;
    if (d3 >= 0.f && d4 <= d3) {
      q = b; f = 4;
    } else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
      const float v = d1 / (d1 - d3);
      q = make_float3(a.x + v * ab.x, a.y + v * ab.y, a.z + v * ab.z); f = 0;
    } else {
      const float3 cq = make_float3(p.x - c.x, p.y - c.y, p.z - c.z);
      const float d5 = ab.x * cq.x + ab.y * cq.y + ab.z * cq.z;
      const float d6 = ac.x * cq.x + ac.y * cq.y + ac.z * cq.z;
      const float vb = d5 * d2 - d1 * d6;
      const float va = d3 * d6 - d5 * d4;
      if (d6 >= 0.f && d5 <= d6) {
        q = c; f = 5;
      } else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        const float w = d2 / (d2 - d6);
        q = make_float3(a.x + w * ac.x, a.y + w * ac.y, a.z + w * ac.z); f = 2;
      } else if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        const float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        q = make_float3(b.x + w * (c.x - b.x), b.y + w * (c.y - b.y), b.z + w * (c.z - b.z)); f = 1;
      } else {
        const float s = 1.f / (va + vb + vc);
        const float v = vb * s, w = vc * s;
        q = make_float3(a.x + v * ab.x + w * ac.x, a.y + v * ab.y + w * ac.y,
                        a.z + v * ab.z + w * ac.z);
        f = -1;
      }
    }
  }
  *cp = q;
  *feat = f;
  const float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
  return dx * dx + dy * dy + dz * dz;
}

// FP32 result at one point
struct MeshF32 {
  float phi;     // signed distance (+INFINITY outside the grid or in an OUTSIDE cell)
  float3 c;      // nearest surface point (object frame) when phi is finite
  bool tie;      // another candidate is within rounding of the nearest, at another point
};

// relative rounding allowance of the FP32 squared distances (a few hundred ulps)
constexpr float MESH_TIE_REL = 2e-5f;

static __device__ __noinline__ MeshF32 mesh_f32(const MeshDev& m, float3 p) {
  MeshF32 r;
  r.phi = INFINITY;
  r.c = p;
  r.tie = false;
  int kind = MESH_CELL_OUTSIDE;
  const int cell = mesh_cell(m, p, &kind);
  if (cell < 0 || kind == MESH_CELL_OUTSIDE) return r;
  const int s0 = m.cell_start[cell], s1 = m.cell_start[cell + 1];
  float best = INFINITY, second = INFINITY;
  float3 bc = p, sc = p;
  int bt = -1, bf = -1;
  for (int s = s0; s < s1; ++s) {
    const int t = m.cand[s];
    const float4 va = m.tri[4 * t], vb = m.tri[4 * t + 1], vc = m.tri[4 * t + 2];
    float3 cp;
    int f;
    const float d2 = nearest_on_triangle(p, make_float3(va.x, va.y, va.z),
                                         make_float3(vb.x, vb.y, vb.z),
                                         make_float3(vc.x, vc.y, vc.z), &cp, &f);
    if (d2 < best) {
      second = best;
      sc = bc;
      best = d2;
      bc = cp;
      bt = t;
      bf = f;
    } else if (d2 < second) {
      second = d2;
      sc = cp;
    }
  }
  if (bt < 0) return r;
  const float dx = p.x - bc.x, dy = p.y - bc.y, dz = p.z - bc.z;
  float sgn;
  if (kind == MESH_CELL_INSIDE) {
    sgn = -1.f;
  } else {
    const float4 nf = bf < 0 ? m.tri[4 * bt + 3] : m.pseudo[6 * bt + bf];
    sgn = (dx * nf.x + dy * nf.y + dz * nf.z) < 0.f ? -1.f : 1.f;
  }
  r.phi = sgn * sqrtf(best);
  r.c = bc;
  // a runner-up within rounding of the nearest with a nearest point of its own (not the
  // shared edge or vertex of two adjacent triangles)
  const float ex = bc.x - sc.x, ey = bc.y - sc.y, ez = bc.z - sc.z;
  r.tie = second - best <= MESH_TIE_REL * (second + m.cell * m.cell) &&
          ex * ex + ey * ey + ez * ez > 1e-10f * (best + m.cell * m.cell);
  return r;
}

// FP64 result at one point
struct MeshF64 {
  double phi;      // signed distance (+INFINITY outside)
  double c[3];     // nearest surface point
  int feat;        // 0 face, 1 edge interior, 2 vertex
  double e[3];     // unit direction of the edge (feat 1)
};

static __device__ __noinline__ MeshF64 mesh_f64(const MeshDev& m, const double q[3]) {
  MeshF64 r;
  r.phi = INFINITY;
  r.c[0] = q[0]; r.c[1] = q[1]; r.c[2] = q[2];
  r.feat = 0;
  r.e[0] = r.e[1] = r.e[2] = 0.0;
  int kind = MESH_CELL_OUTSIDE;
  const int cell = mesh_cell(m, make_float3((float)q[0], (float)q[1], (float)q[2]), &kind);
  if (cell < 0 || kind == MESH_CELL_OUTSIDE) return r;
  const int s0 = m.cell_start[cell], s1 = m.cell_start[cell + 1];
  double best = INFINITY;
  int bt = -1, bfeat = 0, bnorm = -1;   // bnorm: pseudo-normal slot, -1 the face normal
  for (int s = s0; s < s1; ++s) {
    const int t = m.cand[s];
    const float4 v4[3] = {m.tri[4 * t], m.tri[4 * t + 1], m.tri[4 * t + 2]};
    const double v[3][3] = {{v4[0].x, v4[0].y, v4[0].z}, {v4[1].x, v4[1].y, v4[1].z},
                            {v4[2].x, v4[2].y, v4[2].z}};
    double cp[3], ed[3] = {0.0, 0.0, 0.0}, d2;
    int feat, norm;
    // orthogonal projection onto the plane and its barycentric weights (signed sub-areas)
    const double u0[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    const double u1[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    const double nrm[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2],
                           u0[0] * u1[1] - u0[1] * u1[0]};
    const double nn = nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2];
    bool face = false;
    if (nn > 0.0) {
      const double h = ((q[0] - v[0][0]) * nrm[0] + (q[1] - v[0][1]) * nrm[1] +
                        (q[2] - v[0][2]) * nrm[2]) / nn;
      const double pr[3] = {q[0] - h * nrm[0], q[1] - h * nrm[1], q[2] - h * nrm[2]};
      double w[3];
      for (int k = 0; k < 3; ++k) {
        const double* x = v[(k + 1) % 3];
        const double* y = v[(k + 2) % 3];
        const double xa[3] = {x[0] - pr[0], x[1] - pr[1], x[2] - pr[2]};
        const double ya[3] = {y[0] - pr[0], y[1] - pr[1], y[2] - pr[2]};
        const double cr[3] = {xa[1] * ya[2] - xa[2] * ya[1], xa[2] * ya[0] - xa[0] * ya[2],
                              xa[0] * ya[1] - xa[1] * ya[0]};
        w[k] = (cr[0] * nrm[0] + cr[1] * nrm[1] + cr[2] * nrm[2]) / nn;
      }
      if (w[0] >= -1e-12 && w[1] >= -1e-12 && w[2] >= -1e-12) {
        face = true;
        cp[0] = pr[0]; cp[1] = pr[1]; cp[2] = pr[2];
        d2 = h * h * nn;
        feat = 0;
        norm = -1;
      }
    }
    if (!face) {
      d2 = INFINITY;
      feat = 1;
      norm = 0;
      for (int k = 0; k < 3; ++k) {   // edges ab, bc, ca
        const double* x = v[k];
        const double* y = v[(k + 1) % 3];
        const double se[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        const double L2 = se[0] * se[0] + se[1] * se[1] + se[2] * se[2];
        double tt = L2 > 0.0 ? ((q[0] - x[0]) * se[0] + (q[1] - x[1]) * se[1] +
                                (q[2] - x[2]) * se[2]) / L2 : 0.0;
        tt = tt < 0.0 ? 0.0 : (tt > 1.0 ? 1.0 : tt);
        const double pc[3] = {x[0] + tt * se[0], x[1] + tt * se[1], x[2] + tt * se[2]};
        const double dd = (q[0] - pc[0]) * (q[0] - pc[0]) + (q[1] - pc[1]) * (q[1] - pc[1]) +
                          (q[2] - pc[2]) * (q[2] - pc[2]);
        if (dd < d2) {
          d2 = dd;
          cp[0] = pc[0]; cp[1] = pc[1]; cp[2] = pc[2];
          if (tt > 0.0 && tt < 1.0) {
            feat = 1;
            norm = k;   // edge pseudo-normal
            const double L = sqrt(L2);
            ed[0] = se[0] / L; ed[1] = se[1] / L; ed[2] = se[2] / L;
          } else {
            feat = 2;
            norm = 3 + (tt <= 0.0 ? k : (k + 1) % 3);   // vertex pseudo-normal
          }
        }
      }
    }
    if (d2 < best) {
      best = d2;
      bt = t;
      bfeat = feat;
      bnorm = norm;
      r.c[0] = cp[0]; r.c[1] = cp[1]; r.c[2] = cp[2];
      r.e[0] = ed[0]; r.e[1] = ed[1]; r.e[2] = ed[2];
    }
  }
  if (bt < 0) return r;
  const double dx = q[0] - r.c[0], dy = q[1] - r.c[1], dz = q[2] - r.c[2];
  double sgn;
  if (kind == MESH_CELL_INSIDE) {
    sgn = -1.0;
  } else {
    const float4 nf = bnorm < 0 ? m.tri[4 * bt + 3] : m.pseudo[6 * bt + bnorm];
    sgn = (dx * nf.x + dy * nf.y + dz * nf.z) < 0.0 ? -1.0 : 1.0;
  }
  r.phi = sgn * sqrt(best);
  r.feat = bfeat;
  return r;
}

}  // namespace etac
