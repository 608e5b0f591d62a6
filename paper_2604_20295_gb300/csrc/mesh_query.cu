// mesh_query.cu -- GPU signed-distance query against a closed triangle mesh (the object-mesh
// contact of ETac Sec. III-A, "Overview").
//
// The mesh arrives as the host-built acceleration structure of mesh_accel.cpp: a uniform
// grid over the bounding box whose cells are OUTSIDE (every point outside), INSIDE (every
// point inside) or SURFACE, the triangles that can hold the nearest surface point of any
// point of an INSIDE or SURFACE cell, and per triangle its vertices, face normal and the
// pseudo-normals of its edges and vertices.  etac_mesh_gpu_create copies those arrays to
// the device once; they are a few MB per mesh and stay resident in L2 across queries.
//
// One thread per point.  A point outside the grid or in an OUTSIDE cell is outside and
// costs two loads.  Otherwise the thread walks its cell's candidate list (ascending triangle
// index, so the first of equally near triangles wins, as in the oracle), finds each
// triangle's nearest point by its Voronoi regions (Ericson, "Real-Time Collision Detection",
// 2005, Sec. 5.1.5) in FP32, and keeps the nearest.  The sign is -1 in an INSIDE cell and
// otherwise the sign of (q - c) . n_F with n_F the pseudo-normal of the feature that holds
// the nearest point c (Baerentzen and Aanaes, IEEE TVCG 2005).  Points of a pad are
// spatially coherent, so the lanes of a warp mostly share a cell and walk the same list.
//
// Bound: FP32 issue.  Per point in a listed cell: about 40 FLOP per candidate (a 16 B x 3
// load each, from L2) plus 16 B of output; per outside point 12 B in and 16 B out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "etac.h"
#include "mesh_common.cuh"

namespace etac {
void set_context_free_error(const std::string& msg);   // api.cu: read by etac_last_error(NULL)
}

struct etac_mesh_gpu {
  float origin[3];
  float cell;
  int dims[3];
  int num_tris;
  int64_t num_cand;
  int32_t* cell_start;   // device [C+1]
  uint8_t* cell_kind;    // device [C]
  int32_t* cand;         // device [num_cand]
  float4* tri;           // device [T*4]
  float4* pseudo;        // device [T*6]
};

namespace {

struct MeshArgs {
  float ox, oy, oz, cell;
  int nx, ny, nz;
  const int32_t* __restrict__ cell_start;
  const uint8_t* __restrict__ cell_kind;
  const int32_t* __restrict__ cand;
  const float4* __restrict__ tri;
  const float4* __restrict__ pseudo;
};

using etac::nearest_on_triangle;   // mesh_common.cuh: Voronoi-region nearest point

__global__ void __launch_bounds__(256) mesh_sdf_kernel(MeshArgs m, int64_t n,
                                                       const float* __restrict__ q,
                                                       float* __restrict__ phi,
                                                       float* __restrict__ grad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float3 p = make_float3(q[3 * i], q[3 * i + 1], q[3 * i + 2]);
    const float rx = (p.x - m.ox) / m.cell, ry = (p.y - m.oy) / m.cell, rz = (p.z - m.oz) / m.cell;
    float out_phi = INFINITY;
    float3 g = make_float3(0.f, 0.f, 0.f);
    // comparisons in float first: NaN coordinates fail them and count as outside
    if (rx >= 0.f && ry >= 0.f && rz >= 0.f && rx < (float)m.nx && ry < (float)m.ny &&
        rz < (float)m.nz) {
      const int ix = min((int)rx, m.nx - 1), iy = min((int)ry, m.ny - 1), iz = min((int)rz, m.nz - 1);
      const int c = (iz * m.ny + iy) * m.nx + ix;
      const int kind = m.cell_kind[c];
      if (kind != ETAC_CELL_OUTSIDE) {
        const int s0 = m.cell_start[c], s1 = m.cell_start[c + 1];
        float best = INFINITY;
        float3 bc = p;
        int bt = -1, bf = -1;
        for (int s = s0; s < s1; ++s) {
          const int t = m.cand[s];
          const float4 va = m.tri[4 * t], vb = m.tri[4 * t + 1], vc = m.tri[4 * t + 2];
          float3 cp;
          int f;
          const float d2 = nearest_on_triangle(p, make_float3(va.x, va.y, va.z),
                                               make_float3(vb.x, vb.y, vb.z),
                                               make_float3(vc.x, vc.y, vc.z), &cp, &f);
          if (d2 < best) { best = d2; bc = cp; bt = t; bf = f; }
        }
        if (bt >= 0) {
          const float dx = p.x - bc.x, dy = p.y - bc.y, dz = p.z - bc.z;
          float sgn;
          if (kind == ETAC_CELL_INSIDE) {
            sgn = -1.f;
          } else {
            const float4 nf = bf < 0 ? m.tri[4 * bt + 3] : m.pseudo[6 * bt + bf];
            sgn = (dx * nf.x + dy * nf.y + dz * nf.z) < 0.f ? -1.f : 1.f;
          }
          const float d = sqrtf(best);
          out_phi = sgn * d;
          if (d > 0.f) {
            const float s = sgn / d;
            g = make_float3(s * dx, s * dy, s * dz);
          }
        }
      }
    }
    phi[i] = out_phi;
    if (grad) {
      grad[3 * i] = g.x;
      grad[3 * i + 1] = g.y;
      grad[3 * i + 2] = g.z;
    }
  }
}

etac_status fail(const std::string& m, etac_status st = ETAC_ERR_INVALID_ARG) {
  etac::set_context_free_error(m);
  return st;
}

void free_mesh(etac_mesh_gpu* g) {
  if (!g) return;
  cudaFree(g->cell_start);
  cudaFree(g->cell_kind);
  cudaFree(g->cand);
  cudaFree(g->tri);
  cudaFree(g->pseudo);
  delete g;
}

}  // namespace

namespace etac {
// device view of a mesh for the contact step (etac_set_meshes)
void mesh_dev_view(const etac_mesh_gpu* g, MeshDev* d) {
  d->ox = g->origin[0];
  d->oy = g->origin[1];
  d->oz = g->origin[2];
  d->cell = g->cell;
  d->nx = g->dims[0];
  d->ny = g->dims[1];
  d->nz = g->dims[2];
  float ext = 0.f;
  for (int a = 0; a < 3; ++a)
    ext = std::max(ext, std::max(std::fabs(g->origin[a]),
                                 std::fabs(g->origin[a] + g->cell * (float)g->dims[a])));
  d->extent = ext * 1.7320508f;   // the bounding box corner's distance bounds |x| (sqrt 3)
  d->cell_start = g->cell_start;
  d->cell_kind = g->cell_kind;
  d->cand = g->cand;
  d->tri = g->tri;
  d->pseudo = g->pseudo;
}
}  // namespace etac

extern "C" {

etac_status etac_mesh_gpu_create(etac_mesh_gpu** out, const etac_mesh_accel* accel, void* stream) {
  if (!out || !accel) return fail("etac_mesh_gpu_create: NULL argument");
  *out = nullptr;
  etac_mesh_accel_view v;
  etac_status st = etac_mesh_accel_get_view(accel, &v);
  if (st != ETAC_OK) return st;
  const int64_t C = (int64_t)v.dims[0] * v.dims[1] * v.dims[2];
  const size_t T = (size_t)v.num_tris;
  cudaStream_t s = (cudaStream_t)stream;
  etac_mesh_gpu* g = new etac_mesh_gpu();
  for (int a = 0; a < 3; ++a) { g->origin[a] = v.origin[a]; g->dims[a] = v.dims[a]; }
  g->cell = v.cell;
  g->num_tris = v.num_tris;
  g->num_cand = v.num_cand;
  const size_t nc = (size_t)(v.num_cand > 0 ? v.num_cand : 1);
  if (cudaMalloc(&g->cell_start, sizeof(int32_t) * (C + 1)) != cudaSuccess ||
      cudaMalloc(&g->cell_kind, (size_t)C) != cudaSuccess ||
      cudaMalloc(&g->cand, sizeof(int32_t) * nc) != cudaSuccess ||
      cudaMalloc(&g->tri, sizeof(float4) * 4 * T) != cudaSuccess ||
      cudaMalloc(&g->pseudo, sizeof(float4) * 6 * T) != cudaSuccess) {
    cudaGetLastError();
    free_mesh(g);
    return fail("etac_mesh_gpu_create: device allocation failed", ETAC_ERR_OOM);
  }
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* d, const void* h, size_t b) {
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, s);
  };
  cp(g->cell_start, v.cell_start, sizeof(int32_t) * (C + 1));
  cp(g->cell_kind, v.cell_kind, (size_t)C);
  cp(g->cand, v.cand, sizeof(int32_t) * (size_t)v.num_cand);
  cp(g->tri, v.tri, sizeof(float4) * 4 * T);
  cp(g->pseudo, v.pseudo, sizeof(float4) * 6 * T);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host arrays belong to accel
  if (e != cudaSuccess) {
    free_mesh(g);
    return fail(std::string("etac_mesh_gpu_create: ") + cudaGetErrorString(e), ETAC_ERR_CUDA);
  }
  *out = g;
  return ETAC_OK;
}

etac_status etac_mesh_sdf_query(const etac_mesh_gpu* mesh, int64_t n, const float* q, float* phi,
                                float* grad, void* stream) {
  if (!mesh) return fail("etac_mesh_sdf_query: NULL mesh");
  if (n < 0) return fail("etac_mesh_sdf_query: negative point count");
  if (n == 0) return ETAC_OK;
  if (!q || !phi) return fail("etac_mesh_sdf_query: NULL point or output array");
  if (((uintptr_t)q | (uintptr_t)phi | (uintptr_t)grad) & 3u)
    return fail("etac_mesh_sdf_query: arrays must be 4-byte aligned");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail("etac_mesh_sdf_query: no CUDA device", ETAC_ERR_CUDA);
  }
  MeshArgs a;
  a.ox = mesh->origin[0]; a.oy = mesh->origin[1]; a.oz = mesh->origin[2];
  a.cell = mesh->cell;
  a.nx = mesh->dims[0]; a.ny = mesh->dims[1]; a.nz = mesh->dims[2];
  a.cell_start = mesh->cell_start;
  a.cell_kind = mesh->cell_kind;
  a.cand = mesh->cand;
  a.tri = mesh->tri;
  a.pseudo = mesh->pseudo;
  const int64_t blocks = (n + 255) / 256;
  const int grid = (int)std::min<int64_t>(blocks, (int64_t)sms * 8);
  mesh_sdf_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(a, n, q, phi, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(std::string("etac_mesh_sdf_query: ") + cudaGetErrorString(e), ETAC_ERR_CUDA);
  return ETAC_OK;
}

void etac_mesh_gpu_destroy(etac_mesh_gpu* mesh) {
  if (!mesh) return;
  cudaDeviceSynchronize();
  free_mesh(mesh);
}

}  // extern "C"
