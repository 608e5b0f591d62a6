// etac_common.cuh -- device building blocks shared by the ETac kernels: double-float
// arithmetic, rigid transforms, primitive signed distances and per-node contact.
//
// Contact (ETac Sec. III-A, "Overview"): a node is active when it lies strictly inside a
// rigid object (signed distance phi < 0, minimum over the environment's objects, ties to
// the lowest object index); its local displacement moves it onto the object surface along
// the outward normal, u_hat = -phi * grad(phi), expressed in the pad frame.
//
// Precision: the contact decision and the penetration of nodes near or inside an object are
// evaluated in double-float ("df32": an unevaluated sum hi + lo of two floats, built from the
// error-free transformations of Dekker 1971 and Knuth's TwoSum) so that contact sets agree
// with an exact evaluation except within ~1e-10 mm of a surface, without FP64 on the GPU.
// A cheap FP32 screen with a proven error margin sends every node that is certainly outside
// all objects down the fast path.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mesh_common.cuh"

namespace etac {

constexpr int H = 64;     // hidden width
constexpr int NIN = 9;    // per-node network input [p, n, u_hat]
constexpr int MAX_K = 8;  // objects per environment

// flat parameter layout: alpha, then (W, b) of E1, E2, G1, D1, D2
constexpr int OFF_ALPHA = 0;
constexpr int OFF_W1 = 1;
constexpr int OFF_B1 = OFF_W1 + H * NIN;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_WG = OFF_B2 + H;
constexpr int OFF_BG = OFF_WG + H * H;
constexpr int OFF_WD = OFF_BG + H;
constexpr int OFF_BD = OFF_WD + H * 2 * H;
constexpr int OFF_W4 = OFF_BD + H;
constexpr int OFF_B4 = OFF_W4 + 3 * H;
constexpr int NPARAM = OFF_B4 + 3;

enum { OBJ_NONE = 0, OBJ_SPHERE = 1, OBJ_BOX = 2, OBJ_CYLINDER = 3, OBJ_CAPSULE = 4, OBJ_MESH = 5 };
enum { MODE_FULL = 0, MODE_LINEAR_ONLY = 1, MODE_RESIDUAL_ONLY = 2, MODE_PENETRATION_ONLY = 3 };
// which terms of Eq. 4 a mode evaluates: the propagation L (Eq. 1) and the residual R
__host__ __device__ __forceinline__ bool uses_propagation(int mode) {
  return mode == MODE_FULL || mode == MODE_LINEAR_ONLY;
}
__host__ __device__ __forceinline__ bool uses_residual(int mode) {
  return mode == MODE_FULL || mode == MODE_RESIDUAL_ONLY;
}
enum { STATUS_OK = 0, STATUS_TIMEOUT = 5, STATUS_NONFINITE = 6, STATUS_BOUNDS = 8 };

__device__ __forceinline__ void latch_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Index checks of the ETAC_BOUNDS build (build variant "bounds"): ETAC_IN(status, i, n) is true
// when 0 <= i < n; otherwise it latches ETAC_ERR_BOUNDS in the device status word and is false,
// and the access it guards is skipped (no trap, no fault).  In the regular build it is the
// constant true and costs nothing.
__device__ __forceinline__ bool bounds_ok(int* status, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  latch_status(status, STATUS_BOUNDS);
  return false;
}
#ifdef ETAC_BOUNDS
#define ETAC_IN(status, i, n) ::etac::bounds_ok((status), (long long)(i), (long long)(n))
#else
#define ETAC_IN(status, i, n) true
#endif

// ------------------------------------------------------------------ tiled FP32 product
constexpr int TLD = H + 4;   // padded row stride of staged 64 x 64 tiles (16-byte aligned)

// acc[i][j] += sum_k A[k][4 ti + i] * B[k][4 tj + j], both operands k-major with stride TLD
__device__ __forceinline__ void tile_acc(const float* A, const float* B, int ti, int tj,
                                         float (&acc)[4][4]) {
#pragma unroll 8
  for (int k = 0; k < 64; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(A + k * TLD + 4 * ti);
    const float4 b = *reinterpret_cast<const float4*>(B + k * TLD + 4 * tj);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

// ------------------------------------------------------------------ double-float (df32)
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(float a) { return {a, 0.f}; }

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Dekker's FastTwoSum, valid when |a| >= |b| (or a == 0)
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

// exact product through a fused multiply-add
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}

// Dekker's double-length addition: the absolute error is below ~2^-47 (|a| + |b|), i.e.
// ~1e-12 mm for coordinates of 100 mm, far inside the 1e-6 mm contact band; cancellation in
// the result (phi = |q| - r near the surface) costs relative, not absolute, accuracy.
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// long division with two correction terms (Dekker 1971)
__device__ __forceinline__ df df_div(df a, df b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = df_sub(a, df_mul_f(b, q1));
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = df_sub(r, df_mul_f(b, q2));
  float q3 = __fdiv_rn(r.hi, b.hi);
  return df_add(quick_two_sum(q1, q2), df_from(q3));
}

// square root: FP32 root plus one Newton correction of the residual (Karp & Markstein 1997)
__device__ __forceinline__ df df_sqrt(df a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  float x = __fsqrt_rn(a.hi);
  df r = df_sub(a, two_prod(x, x));
  float c = __fdiv_rn(r.hi, __fmul_rn(2.f, x));
  return quick_two_sum(x, c);
}

__device__ __forceinline__ bool df_lt(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool df_isneg(df a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }
__device__ __forceinline__ df df_abs(df a) { return df_isneg(a) ? df_neg(a) : a; }
__device__ __forceinline__ float df_f(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ df df_sq(df a) { return df_mul(a, a); }

// ------------------------------------------------------------------ rotations

// Rotation matrix of a (not necessarily unit) quaternion (x, y, z, w) in the homogeneous form
// R = M(q) / |q|^2, which equals the matrix of q / |q| and needs no square root.
template <typename T>
__device__ __forceinline__ void quat_to_mat(const T* q, T R[3][3]) {
  T x = q[0], y = q[1], z = q[2], w = q[3];
  T n2 = x * x + y * y + z * z + w * w;
  T s = T(1) / n2, s2 = T(2) * s;
  R[0][0] = (w * w + x * x - y * y - z * z) * s;
  R[0][1] = (x * y - w * z) * s2;
  R[0][2] = (x * z + w * y) * s2;
  R[1][0] = (x * y + w * z) * s2;
  R[1][1] = (w * w - x * x + y * y - z * z) * s;
  R[1][2] = (y * z - w * x) * s2;
  R[2][0] = (x * z - w * y) * s2;
  R[2][1] = (y * z + w * x) * s2;
  R[2][2] = (w * w - x * x - y * y + z * z) * s;
}

__device__ __forceinline__ void quat_to_mat_df(const float* q, df R[3][3]) {
  float x = q[0], y = q[1], z = q[2], w = q[3];
  df xx = two_prod(x, x), yy = two_prod(y, y), zz = two_prod(z, z), ww = two_prod(w, w);
  df xy = two_prod(x, y), xz = two_prod(x, z), yz = two_prod(y, z);
  df wx = two_prod(w, x), wy = two_prod(w, y), wz = two_prod(w, z);
  df n2 = df_add(df_add(xx, yy), df_add(zz, ww));
  df s = df_div(df_from(1.f), n2);
  df s2 = {2.f * s.hi, 2.f * s.lo};
  R[0][0] = df_mul(df_sub(df_add(ww, xx), df_add(yy, zz)), s);
  R[0][1] = df_mul(df_sub(xy, wz), s2);
  R[0][2] = df_mul(df_add(xz, wy), s2);
  R[1][0] = df_mul(df_add(xy, wz), s2);
  R[1][1] = df_mul(df_sub(df_add(ww, yy), df_add(xx, zz)), s);
  R[1][2] = df_mul(df_sub(yz, wx), s2);
  R[2][0] = df_mul(df_sub(xz, wy), s2);
  R[2][1] = df_mul(df_add(yz, wx), s2);
  R[2][2] = df_mul(df_sub(df_add(ww, zz), df_add(xx, yy)), s);
}

// ------------------------------------------------------------------ pad <-> object setup

// Relative rigid transform from a pad frame to one object's frame, q = R p + t, in FP32 and
// in df32, plus the screening margin of the FP32 evaluation.
struct PadObj {
  float R[9];
  float t[3];
  df Rd[9];
  df td[3];
  float dims[3];
  float tau;   // |phi_fp32 - phi| < tau for every node of this pad
  int type;    // OBJ_*; OBJ_NONE when the slot is empty
  const MeshDev* mesh;   // OBJ_MESH: the mesh (dims[0] holds its index)
};

// The mesh an OBJ_MESH object names (dims[0] = its index among the context's meshes), or
// null when the index is not one of them.
__device__ __forceinline__ const MeshDev* object_mesh(const float* dims, const MeshDev* meshes,
                                                      int num_meshes) {
  const float f = dims[0];
  const int i = (int)f;
  return (meshes && f >= 0.f && f < (float)num_meshes && (float)i == f) ? meshes + i : nullptr;
}

__device__ __forceinline__ bool finite7(const float* a) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 7; ++i) ok &= isfinite(a[i]);
  return ok && (a[3] != 0.f || a[4] != 0.f || a[5] != 0.f || a[6] != 0.f);
}

// pmax: the largest Euclidean |p| over the pad's nodes (bounds the FP32 rounding of R p)
__device__ inline void setup_pad_obj(const float* obj_pose, int type, const float* dims,
                                     const float* pad_pose, float pmax, PadObj* o,
                                     const MeshDev* mesh = nullptr) {
  df Rk[3][3], Rp[3][3];
  quat_to_mat_df(obj_pose + 3, Rk);
  quat_to_mat_df(pad_pose + 3, Rp);
  df d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = two_sum(pad_pose[a], -obj_pose[a]);   // exact
  float tt = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      df acc = df_mul(Rk[0][a], Rp[0][b]);
      acc = df_add(acc, df_mul(Rk[1][a], Rp[1][b]));
      acc = df_add(acc, df_mul(Rk[2][a], Rp[2][b]));
      o->Rd[3 * a + b] = acc;
      o->R[3 * a + b] = df_f(acc);
    }
    df acc = df_mul(Rk[0][a], d[0]);
    acc = df_add(acc, df_mul(Rk[1][a], d[1]));
    acc = df_add(acc, df_mul(Rk[2][a], d[2]));
    o->td[a] = acc;
    o->t[a] = df_f(acc);
    tt = fmaf(o->t[a], o->t[a], tt);
  }
  // |t| (Euclidean), raised by 2^-20 relative to cover the rounding of its own evaluation
  const float tmax = sqrtf(tt) * (1.f + 0x1p-20f);
  o->type = type;
  o->mesh = mesh;
  o->dims[0] = dims[0];
  o->dims[1] = dims[1];
  o->dims[2] = dims[2];
  // FP32 error of phi: R rounded to FP32 (u |p|), the three FMAs of q = R p + t
  // (3u (sqrt(3) |p| + |t|) per component), the SDF's squares, root and differences
  // (~2.5u |q| + u (|q| + size)) and |q| <= |p| + |t| give |phi32 - phi| < 16u (|t| + |p| + size)
  // with u = 2^-24 and |t|, |p| Euclidean norms; tau = 3e-6 (~50u) of those magnitudes is a 3x
  // margin (plus 1e-5 mm).  size bounds the SDF's own magnitudes: the largest dimension.
  float size = fmaxf(fmaxf(fabsf(dims[0]), fabsf(dims[1])), fabsf(dims[2]));
  o->tau = 1e-5f + 3e-6f * (tmax + pmax + size);
  if (type == OBJ_MESH) {
    // the mesh query's FP32 nearest-point arithmetic (Voronoi tests, projections, a root)
    // runs on coordinates up to |t| + |p| and mesh extents; 2e-5 (~340 u) of those
    // magnitudes bounds it with room to spare, and nodes inside this margin (a few um) take
    // the FP64 decision
    o->tau = 1e-4f + 2e-5f * (tmax + pmax + (mesh ? mesh->extent : 0.f));
  }
}

// ------------------------------------------------------------------ signed distances

// FP32 signed distance, used only for screening (exact formula, FP32 rounding).
__device__ __forceinline__ float sdf_f32(int type, const float* dims, float3 q) {
  if (type == OBJ_SPHERE) return sqrtf(q.x * q.x + q.y * q.y + q.z * q.z) - dims[0];
  if (type == OBJ_BOX) {
    float dx = fabsf(q.x) - dims[0], dy = fabsf(q.y) - dims[1], dz = fabsf(q.z) - dims[2];
    float ox = fmaxf(dx, 0.f), oy = fmaxf(dy, 0.f), oz = fmaxf(dz, 0.f);
    return sqrtf(ox * ox + oy * oy + oz * oz) + fminf(fmaxf(dx, fmaxf(dy, dz)), 0.f);
  }
  if (type == OBJ_CYLINDER) {
    float dr = sqrtf(q.x * q.x + q.y * q.y) - dims[0], dz = fabsf(q.z) - dims[1];
    float or_ = fmaxf(dr, 0.f), oz = fmaxf(dz, 0.f);
    return sqrtf(or_ * or_ + oz * oz) + fminf(fmaxf(dr, dz), 0.f);
  }
  if (type == OBJ_CAPSULE) {
    float cz = fminf(fmaxf(q.z, -dims[1]), dims[1]);
    float vz = q.z - cz;
    return sqrtf(q.x * q.x + q.y * q.y + vz * vz) - dims[0];
  }
  return INFINITY;
}

// FP32 signed distance of object slot o at object-frame point q (screening and culling).
// MESH = false compiles the mesh query out (kernels launched for contexts without meshes:
// the query's out-of-line call would cost the streaming loops registers).
template <bool MESH = true>
__device__ __forceinline__ float sdf_obj_f32(const PadObj& o, float3 q) {
  if (MESH && o.type == OBJ_MESH) return o.mesh ? mesh_f32(*o.mesh, q).phi : INFINITY;
  return sdf_f32(o.type, o.dims, q);
}

// Signed distance in df32 where the node may be inside.  Returns true and sets phi < 0 when
// q is strictly inside; g receives the outward unit normal (object frame, FP32), hk the
// Hessian kind for the reverse mode (0 none, 1 spherical about hc, 2 radial about the z
// axis, 3 a mesh edge of direction e, 4 a mesh vertex), deg whether the normal is undefined
// at q.
struct SdfIn {
  df phi;
  float g[3];
  float qf[3];
  float e[3];
  int hk;
  bool deg;
};

// A mesh object's exact decision: FP64 from the df32 point (hi + lo is exact in double).
// Inside, the outward normal is the direction from the node to its nearest surface point.
__device__ inline bool mesh_inside(const MeshDev& m, const df q[3], SdfIn* s) {
  const double qd[3] = {(double)q[0].hi + (double)q[0].lo, (double)q[1].hi + (double)q[1].lo,
                        (double)q[2].hi + (double)q[2].lo};
  const MeshF64 r = mesh_f64(m, qd);
  if (!(r.phi < 0.0)) return false;
  const double d = -r.phi;
  const float hi = (float)r.phi;
  s->phi = {hi, (float)(r.phi - (double)hi)};
  s->g[0] = (float)((r.c[0] - qd[0]) / d);
  s->g[1] = (float)((r.c[1] - qd[1]) / d);
  s->g[2] = (float)((r.c[2] - qd[2]) / d);
  s->hk = r.feat == 1 ? 3 : (r.feat == 2 ? 4 : 0);
  s->e[0] = (float)r.e[0];
  s->e[1] = (float)r.e[1];
  s->e[2] = (float)r.e[2];
  return true;
}

template <bool MESH = true>
__device__ inline bool sdf_inside_df(int type, const float* dims, const df q[3], SdfIn* s,
                                     const MeshDev* mesh = nullptr) {
  s->deg = false;
  s->hk = 0;
  s->qf[0] = df_f(q[0]);
  s->qf[1] = df_f(q[1]);
  s->qf[2] = df_f(q[2]);
  s->g[0] = s->g[1] = s->g[2] = 0.f;
  s->e[0] = s->e[1] = s->e[2] = 0.f;
  if (MESH && type == OBJ_MESH) return mesh && mesh_inside(*mesh, q, s);
  if (type == OBJ_SPHERE) {
    df L = df_sqrt(df_add(df_add(df_sq(q[0]), df_sq(q[1])), df_sq(q[2])));
    s->phi = df_sub(L, df_from(dims[0]));
    if (!df_isneg(s->phi)) return false;
    float Lf = df_f(L);
    if (Lf > 0.f) {
      s->g[0] = s->qf[0] / Lf;
      s->g[1] = s->qf[1] / Lf;
      s->g[2] = s->qf[2] / Lf;
      s->hk = 1;
    } else {
      s->deg = true;
    }
    return true;
  }
  if (type == OBJ_BOX) {
    df best = df_sub(df_abs(q[0]), df_from(dims[0]));
    if (!df_isneg(best)) return false;
    int am = 0;
#pragma unroll
    for (int a = 1; a < 3; ++a) {
      df d = df_sub(df_abs(q[a]), df_from(dims[a]));
      if (!df_isneg(d)) return false;
      if (df_lt(best, d)) {   // strict: ties keep the lowest axis
        best = d;
        am = a;
      }
    }
    s->phi = best;
    // selects, not an indexed store: keeps *s in registers
    const bool neg = am == 0 ? df_isneg(q[0]) : (am == 1 ? df_isneg(q[1]) : df_isneg(q[2]));
    const float sg = neg ? -1.f : 1.f;
    s->g[0] = am == 0 ? sg : 0.f;
    s->g[1] = am == 1 ? sg : 0.f;
    s->g[2] = am == 2 ? sg : 0.f;
    return true;
  }
  if (type == OBJ_CYLINDER) {
    df rho = df_sqrt(df_add(df_sq(q[0]), df_sq(q[1])));
    df dr = df_sub(rho, df_from(dims[0]));
    df dz = df_sub(df_abs(q[2]), df_from(dims[1]));
    if (!df_isneg(dr) || !df_isneg(dz)) return false;
    if (!df_lt(dr, dz)) {      // dr >= dz: radial wall is nearest (ties: radial)
      s->phi = dr;
      float rf = df_f(rho);
      if (rf > 0.f) {
        s->g[0] = s->qf[0] / rf;
        s->g[1] = s->qf[1] / rf;
        s->hk = 2;
      } else {
        s->deg = true;
      }
    } else {
      s->phi = dz;
      s->g[2] = df_isneg(q[2]) ? -1.f : 1.f;
    }
    return true;
  }
  if (type == OBJ_CAPSULE) {
    df h = df_from(dims[1]);
    df cz = q[2];
    if (df_lt(q[2], df_neg(h))) cz = df_neg(h);
    else if (df_lt(h, q[2])) cz = h;
    df vz = df_sub(q[2], cz);
    df L = df_sqrt(df_add(df_add(df_sq(q[0]), df_sq(q[1])), df_sq(vz)));
    s->phi = df_sub(L, df_from(dims[0]));
    if (!df_isneg(s->phi)) return false;
    float Lf = df_f(L), vzf = df_f(vz);
    if (Lf > 0.f) {
      s->g[0] = s->qf[0] / Lf;
      s->g[1] = s->qf[1] / Lf;
      s->g[2] = vzf / Lf;
      s->hk = 1;
    } else {
      s->deg = true;
    }
    return true;
  }
  return false;
}

// Result of contact detection at one node.
struct NodeContact {
  float phi;     // signed distance (exact sign; value accurate to df32 when active)
  float u[3];    // u_hat in the pad frame (zero when passive)
  int k;         // object index of the minimum (-1 when passive)
  bool active;
};

// FP32 screen: false when the node is certainly outside every object (|error| < tau);
// *phi32 receives the FP32 minimum signed distance.
template <bool MESH = true>
__device__ inline bool contact_screen(const PadObj* po, int K, float3 p, float* phi32) {
  float best = INFINITY;
  bool maybe = false;
  for (int k = 0; k < K; ++k) {
    const PadObj& o = po[k];
    if (o.type == OBJ_NONE) continue;
    float3 q;
    q.x = fmaf(o.R[0], p.x, fmaf(o.R[1], p.y, fmaf(o.R[2], p.z, o.t[0])));
    q.y = fmaf(o.R[3], p.x, fmaf(o.R[4], p.y, fmaf(o.R[5], p.z, o.t[1])));
    q.z = fmaf(o.R[6], p.x, fmaf(o.R[7], p.y, fmaf(o.R[8], p.z, o.t[2])));
    const float ph = sdf_obj_f32<MESH>(o, q);
    best = fminf(best, ph);
    maybe |= ph < o.tau;
  }
  *phi32 = best;
  return maybe;
}

// Exact (df32) contact decision and displacement of a node that passed the screen.  Built
// inline; the ETAC_OUTLINE_REFINE build makes it an out-of-line call in every kernel (the
// library's tests check that both builds give the same results).
#ifdef ETAC_OUTLINE_REFINE
#define ETAC_REFINE_LINKAGE static __device__ __noinline__
#else
#define ETAC_REFINE_LINKAGE __device__ inline
#endif
template <bool MESH = true>
ETAC_REFINE_LINKAGE NodeContact contact_refine(const PadObj* po, int K, float3 p, float3 nrm,
                                             float phi32, SdfIn* detail = nullptr) {
  NodeContact r;
  r.phi = phi32;
  r.u[0] = r.u[1] = r.u[2] = 0.f;
  r.k = -1;
  r.active = false;
  df best = df_from(0.f);
  SdfIn bs;
  for (int k = 0; k < K; ++k) {
    const PadObj& o = po[k];
    if (o.type == OBJ_NONE) continue;
    df q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      df acc = df_add(df_mul_f(o.Rd[3 * a + 0], p.x), df_mul_f(o.Rd[3 * a + 1], p.y));
      acc = df_add(acc, df_mul_f(o.Rd[3 * a + 2], p.z));
      q[a] = df_add(acc, o.td[a]);
    }
    SdfIn s;
    if (sdf_inside_df<MESH>(o.type, o.dims, q, &s, o.mesh)) {
      if (r.k < 0 || df_lt(s.phi, best)) {   // strict: ties keep the lowest object
        best = s.phi;
        bs = s;
        r.k = k;
      }
    }
  }
  if (r.k < 0) return r;
  r.active = true;
  r.phi = df_f(best);
  const PadObj& o = po[r.k];
  if (bs.deg) {
    // undefined normal (node on a sphere centre / capsule or cylinder axis): push the node
    // back along its own inward normal, g = -R nrm in the object frame
    bs.g[0] = -(o.R[0] * nrm.x + o.R[1] * nrm.y + o.R[2] * nrm.z);
    bs.g[1] = -(o.R[3] * nrm.x + o.R[4] * nrm.y + o.R[5] * nrm.z);
    bs.g[2] = -(o.R[6] * nrm.x + o.R[7] * nrm.y + o.R[8] * nrm.z);
  }
  const float s = -r.phi;
  // u_hat (pad frame) = R^T (-phi g)
  r.u[0] = s * (o.R[0] * bs.g[0] + o.R[3] * bs.g[1] + o.R[6] * bs.g[2]);
  r.u[1] = s * (o.R[1] * bs.g[0] + o.R[4] * bs.g[1] + o.R[7] * bs.g[2]);
  r.u[2] = s * (o.R[2] * bs.g[0] + o.R[5] * bs.g[1] + o.R[8] * bs.g[2]);
  if (detail) *detail = bs;
  return r;
}

// One FP32 pass over a node's objects that sorts it into three classes:
//   CONTACT_OUT   phi32 >= tau for every object: certainly outside, passive;
//   CONTACT_FAST  certainly inside (phi32 < -gap) and no discrete choice that u_hat depends on
//                 (the nearest object, the nearest box face, radial vs. end wall of a
//                 cylinder) is within `gap` of a tie: the choices equal the exact ones
//                 (|FP32 error| < tau <= gap / 2) and *r holds u_hat from FP32 arithmetic;
//   CONTACT_BAND  anything else: contact_refine decides exactly.
// With `detail`, a FAST node also receives its SDF feature (object-frame point, normal, Hessian
// kind) in FP32, as contact_refine gives it from df32; mesh objects then go to the band, where
// contact_refine finds their face, edge or vertex.
enum { CONTACT_OUT = 0, CONTACT_FAST = 1, CONTACT_BAND = 2 };
template <bool MESH = true>
__device__ inline int contact_classify(const PadObj* po, int K, float3 p, float3 nrm, float gap,
                                       NodeContact* r, SdfIn* detail = nullptr) {
  // pass 1: FP32 distance to every object; far-outside nodes stop here
  float best = INFINITY, second = INFINITY;
  bool maybe = false;
  int bk = -1;
  float3 bq = make_float3(0.f, 0.f, 0.f);
  for (int k = 0; k < K; ++k) {
    const PadObj& o = po[k];
    if (o.type == OBJ_NONE) continue;
    float3 q;
    q.x = fmaf(o.R[0], p.x, fmaf(o.R[1], p.y, fmaf(o.R[2], p.z, o.t[0])));
    q.y = fmaf(o.R[3], p.x, fmaf(o.R[4], p.y, fmaf(o.R[5], p.z, o.t[1])));
    q.z = fmaf(o.R[6], p.x, fmaf(o.R[7], p.y, fmaf(o.R[8], p.z, o.t[2])));
    const float ph = sdf_obj_f32<MESH>(o, q);
    maybe |= ph < o.tau;
    if (ph < best) {
      second = best;
      best = ph;
      bk = k;
      bq = q;
    } else if (ph < second) {
      second = ph;
    }
  }
  if (!maybe) return CONTACT_OUT;
  if (bk < 0 || !(best < -gap) || second - best < gap) return CONTACT_BAND;
  // pass 2: the nearest object's outward normal and the margin of its discrete choice
  const PadObj& o = po[bk];
  const float3 q = bq;
  float g0 = 0.f, g1 = 0.f, g2 = 0.f, margin = INFINITY;
  bool deg = false;
  int hk = 0;   // Hessian kind, as sdf_inside_df reports it
  if (MESH && o.type == OBJ_MESH) {
    if (detail) return CONTACT_BAND;
    // the nearest point again (pass 1 kept only the distance); a runner-up within rounding
    // at another point leaves the choice of u_hat to the exact path
    const MeshF32 r = mesh_f32(*o.mesh, q);
    const float d = -r.phi;
    if (r.tie || !(d > 0.f)) return CONTACT_BAND;
    const float id = 1.f / d;
    g0 = (r.c.x - q.x) * id;
    g1 = (r.c.y - q.y) * id;
    g2 = (r.c.z - q.z) * id;
  } else if (o.type == OBJ_SPHERE || o.type == OBJ_CAPSULE) {
    float vz = q.z;
    if (o.type == OBJ_CAPSULE) vz = q.z - fminf(fmaxf(q.z, -o.dims[1]), o.dims[1]);
    const float L = sqrtf(q.x * q.x + q.y * q.y + vz * vz);
    if (L > 0.f) {
      const float il = 1.f / L;
      g0 = q.x * il;
      g1 = q.y * il;
      g2 = vz * il;
      hk = 1;
    } else {
      deg = true;
    }
  } else if (o.type == OBJ_BOX) {
    // nearest face: the largest of d = |q| - half size, lowest axis on ties (selects, so
    // nothing is indexed at run time); inside, phi = max d
    const float dx = fabsf(q.x) - o.dims[0], dy = fabsf(q.y) - o.dims[1],
                dz = fabsf(q.z) - o.dims[2];
    int am = 0;
    float dm = dx;
    if (dy > dm) {
      am = 1;
      dm = dy;
    }
    if (dz > dm) {
      am = 2;
      dm = dz;
    }
    const float sec = am == 0 ? fmaxf(dy, dz) : (am == 1 ? fmaxf(dx, dz) : fmaxf(dx, dy));
    margin = dm - sec;
    const float qs = am == 0 ? q.x : (am == 1 ? q.y : q.z);
    const float sg = qs >= 0.f ? 1.f : -1.f;
    g0 = am == 0 ? sg : 0.f;
    g1 = am == 1 ? sg : 0.f;
    g2 = am == 2 ? sg : 0.f;
  } else {   // cylinder: radial wall or end cap, whichever is nearer (phi = max(dr, dz))
    const float rho = sqrtf(q.x * q.x + q.y * q.y);
    const float dr = rho - o.dims[0], dz = fabsf(q.z) - o.dims[1];
    margin = fabsf(dr - dz);
    if (dr >= dz) {
      if (rho > 0.f) {
        const float ir = 1.f / rho;
        g0 = q.x * ir;
        g1 = q.y * ir;
        hk = 2;
      } else {
        deg = true;
      }
    } else {
      g2 = q.z >= 0.f ? 1.f : -1.f;
    }
  }
  if (margin < gap) return CONTACT_BAND;
  if (deg) {
    g0 = -(o.R[0] * nrm.x + o.R[1] * nrm.y + o.R[2] * nrm.z);
    g1 = -(o.R[3] * nrm.x + o.R[4] * nrm.y + o.R[5] * nrm.z);
    g2 = -(o.R[6] * nrm.x + o.R[7] * nrm.y + o.R[8] * nrm.z);
  }
  r->active = true;
  r->k = bk;
  r->phi = best;
  const float s = -best;
  r->u[0] = s * (o.R[0] * g0 + o.R[3] * g1 + o.R[6] * g2);
  r->u[1] = s * (o.R[1] * g0 + o.R[4] * g1 + o.R[7] * g2);
  r->u[2] = s * (o.R[2] * g0 + o.R[5] * g1 + o.R[8] * g2);
  if (detail) {
    detail->phi = df_from(best);
    detail->g[0] = g0;
    detail->g[1] = g1;
    detail->g[2] = g2;
    detail->qf[0] = q.x;
    detail->qf[1] = q.y;
    detail->qf[2] = q.z;
    detail->e[0] = detail->e[1] = detail->e[2] = 0.f;
    detail->hk = hk;
    detail->deg = deg;
  }
  return CONTACT_FAST;
}

// Contact supplied by the caller ("mode B": an external contact pipeline gives the active set
// and u_hat, the propagation input U_a of Eq. 4, in the pad frame): no SDF is evaluated, the
// node's penetration reads zero (phi = -0 so that -phi = +0) and no object is attached.
__device__ __forceinline__ NodeContact contact_given(const uint8_t* mask_in, const float* uhat_in,
                                                     long long node) {
  NodeContact r;
  r.k = -1;
  r.phi = -0.f;
  r.active = mask_in[node] != 0;
  r.u[0] = r.active ? uhat_in[3 * node] : 0.f;
  r.u[1] = r.active ? uhat_in[3 * node + 1] : 0.f;
  r.u[2] = r.active ? uhat_in[3 * node + 2] : 0.f;
  return r;
}

// Contact at node (p, nrm) of a pad against its K object slots (po[k], empty slots skipped).
template <bool MESH = true>
__device__ inline NodeContact contact_node(const PadObj* po, int K, float3 p, float3 nrm,
                                           SdfIn* detail = nullptr) {
  float phi32;
  if (!contact_screen<MESH>(po, K, p, &phi32)) {
    NodeContact r;
    r.phi = phi32;
    r.u[0] = r.u[1] = r.u[2] = 0.f;
    r.k = -1;
    r.active = false;
    return r;
  }
  return contact_refine<MESH>(po, K, p, nrm, phi32, detail);
}

// ------------------------------------------------------------------ FP64 variant
// Used only by the finite-difference gradient check: same decisions in plain double.

struct PadObj64 {
  double R[9];
  double t[3];
  double dims[3];
  int type;
};

__device__ inline void setup_pad_obj64(const double* obj_pose, int type, const double* dims,
                                       const double* pad_pose, PadObj64* o) {
  double Rk[3][3], Rp[3][3];
  quat_to_mat<double>(obj_pose + 3, Rk);
  quat_to_mat<double>(pad_pose + 3, Rp);
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b)
      o->R[3 * a + b] = Rk[0][a] * Rp[0][b] + Rk[1][a] * Rp[1][b] + Rk[2][a] * Rp[2][b];
    o->t[a] = Rk[0][a] * (pad_pose[0] - obj_pose[0]) + Rk[1][a] * (pad_pose[1] - obj_pose[1]) +
              Rk[2][a] * (pad_pose[2] - obj_pose[2]);
    o->dims[a] = dims[a];
  }
  o->type = type;
}

// returns true when strictly inside; phi and outward normal g (object frame)
__device__ inline bool sdf_inside64(int type, const double* dims, const double q[3], double* phi,
                                    double g[3], bool* deg) {
  *deg = false;
  g[0] = g[1] = g[2] = 0.0;
  if (type == OBJ_SPHERE) {
    double L = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    *phi = L - dims[0];
    if (!(*phi < 0.0)) return false;
    if (L > 0) { g[0] = q[0] / L; g[1] = q[1] / L; g[2] = q[2] / L; } else { *deg = true; }
    return true;
  }
  if (type == OBJ_BOX) {
    double best = -INFINITY;
    int am = 0;
    for (int a = 0; a < 3; ++a) {
      double d = fabs(q[a]) - dims[a];
      if (!(d < 0.0)) return false;
      if (d > best) { best = d; am = a; }
    }
    *phi = best;
    g[am] = q[am] >= 0 ? 1.0 : -1.0;
    return true;
  }
  if (type == OBJ_CYLINDER) {
    double rho = sqrt(q[0] * q[0] + q[1] * q[1]);
    double dr = rho - dims[0], dz = fabs(q[2]) - dims[1];
    if (!(dr < 0.0) || !(dz < 0.0)) return false;
    if (dr >= dz) {
      *phi = dr;
      if (rho > 0) { g[0] = q[0] / rho; g[1] = q[1] / rho; } else { *deg = true; }
    } else {
      *phi = dz;
      g[2] = q[2] >= 0 ? 1.0 : -1.0;
    }
    return true;
  }
  if (type == OBJ_CAPSULE) {
    double h = dims[1];
    double cz = q[2] < -h ? -h : (q[2] > h ? h : q[2]);
    double v[3] = {q[0], q[1], q[2] - cz};
    double L = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    *phi = L - dims[0];
    if (!(*phi < 0.0)) return false;
    if (L > 0) { g[0] = v[0] / L; g[1] = v[1] / L; g[2] = v[2] / L; } else { *deg = true; }
    return true;
  }
  return false;
}

__device__ inline bool contact_node64(const PadObj64* po, int K, const double p[3],
                                      const double nrm[3], double u[3]) {
  u[0] = u[1] = u[2] = 0.0;
  int bk = -1;
  double best = 0.0, bg[3] = {0, 0, 0};
  bool bdeg = false;
  for (int k = 0; k < K; ++k) {
    const PadObj64& o = po[k];
    if (o.type == OBJ_NONE) continue;
    double q[3];
    for (int a = 0; a < 3; ++a)
      q[a] = o.R[3 * a] * p[0] + o.R[3 * a + 1] * p[1] + o.R[3 * a + 2] * p[2] + o.t[a];
    double ph, g[3];
    bool deg;
    if (sdf_inside64(o.type, o.dims, q, &ph, g, &deg) && (bk < 0 || ph < best)) {
      bk = k; best = ph; bdeg = deg;
      bg[0] = g[0]; bg[1] = g[1]; bg[2] = g[2];
    }
  }
  if (bk < 0) return false;
  const PadObj64& o = po[bk];
  if (bdeg)
    for (int a = 0; a < 3; ++a)
      bg[a] = -(o.R[3 * a] * nrm[0] + o.R[3 * a + 1] * nrm[1] + o.R[3 * a + 2] * nrm[2]);
  for (int a = 0; a < 3; ++a)
    u[a] = -best * (o.R[a] * bg[0] + o.R[3 + a] * bg[1] + o.R[6 + a] * bg[2]);
  return true;
}

}  // namespace etac
