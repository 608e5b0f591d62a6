// bwd_common.cuh -- pieces shared by the two reverse-mode implementations (per-pad kernel of
// the plain algorithm, staged pipeline of the batched algorithms): the reverse of one active
// node's contact displacement u_hat = -phi n through its primitive's SDF (ETac Sec. III-A) to
// the penetration and the object pose.
#pragma once
#include "etac_common.cuh"

namespace etac {

// Reverse of u_hat = -phi n for one active node (p, nrm) of a pad: du = dL/du_hat in the pad
// frame.  Returns the object slot, dL/d(penetration) = n . du (n the outward normal, pad
// frame), and the object's pose gradient: translation t and the world-frame rotation
// increment w applied on the left about the object origin.  Rp is the pad's rotation, pp its
// pose, op_env the env's object poses (K x 7).
struct NodePoseGrad {
  int k;
  float pen;
  float t[3], w[3];
};

// The node's contact and SDF feature from df32 arithmetic, out of line (the fast path below
// covers most nodes).
template <bool MESH>
__device__ __noinline__ NodeContact pose_contact_exact(const PadObj* spo, int K, float3 p,
                                                       float3 nr, SdfIn* sd) {
  return contact_node<MESH>(spo, K, p, nr, sd);
}

// MESH: mesh objects may occur (their queries are compiled in).  gap > 0 (twice the largest
// FP32 error bound of the pad's objects, as the forward classifies with): nodes that
// contact_classify decides in FP32 take their feature from it, the others from df32; gap <= 0:
// df32 for every node.  Either way the discrete choices (object, face, wall) are the exact ones.
template <bool MESH = true>
__device__ inline NodePoseGrad node_pose_grad(const PadObj* spo, int K, float3 p, float3 nr,
                                              float3 du, const float (&Rp)[3][3],
                                              const float* pp, const float* op_env,
                                              float gap = 0.f) {
  NodePoseGrad out;
  SdfIn sd;
  NodeContact c;
  int cls = CONTACT_BAND;
  if (gap > 0.f) cls = contact_classify<MESH>(spo, K, p, nr, gap, &c, &sd);
  if (cls != CONTACT_FAST) {
    SdfIn se;   // only this copy's address leaves the function: sd stays in registers
    c = pose_contact_exact<MESH>(spo, K, p, nr, &se);
    sd = se;
  }
  out.k = c.k;
  if (c.k < 0) {   // not in contact (the callers pass active nodes only)
    out.pen = 0.f;
    for (int q = 0; q < 3; ++q) out.t[q] = out.w[q] = 0.f;
    return out;
  }
  const PadObj& po = spo[c.k];
  // outward normal in the pad frame: R_rel^T g
  const float npx = po.R[0] * sd.g[0] + po.R[3] * sd.g[1] + po.R[6] * sd.g[2];
  const float npy = po.R[1] * sd.g[0] + po.R[4] * sd.g[1] + po.R[7] * sd.g[2];
  const float npz = po.R[2] * sd.g[0] + po.R[5] * sd.g[1] + po.R[8] * sd.g[2];
  out.pen = npx * du.x + npy * du.y + npz * du.z;
  // v = R_pad du (world); vo = R_k^T v (object frame)
  const float* op = op_env + 7 * c.k;
  float Rk[3][3];
  quat_to_mat<float>(op + 3, Rk);
  float v[3], vo[3], gw[3];
  for (int q = 0; q < 3; ++q) v[q] = Rp[q][0] * du.x + Rp[q][1] * du.y + Rp[q][2] * du.z;
  for (int q = 0; q < 3; ++q) vo[q] = Rk[0][q] * v[0] + Rk[1][q] * v[1] + Rk[2][q] * v[2];
  for (int q = 0; q < 3; ++q) gw[q] = Rk[q][0] * sd.g[0] + Rk[q][1] * sd.g[1] + Rk[q][2] * sd.g[2];
  // A v = g (g . vo) + phi H vo, object frame
  const float phi = c.phi;
  const float gv = sd.g[0] * vo[0] + sd.g[1] * vo[1] + sd.g[2] * vo[2];
  float Av[3] = {sd.g[0] * gv, sd.g[1] * gv, sd.g[2] * gv};
  if (MESH && sd.hk >= 3) {
    // mesh edge (hk 3, direction e) or vertex (hk 4): phi = -(distance to the feature), whose
    // Hessian times phi is the projector I - g g^T (- e e^T on an edge)
    const float ev = sd.hk == 3 ? sd.e[0] * vo[0] + sd.e[1] * vo[1] + sd.e[2] * vo[2] : 0.f;
    for (int q = 0; q < 3; ++q) Av[q] += vo[q] - sd.g[q] * gv - sd.e[q] * ev;
  } else if (!sd.deg && sd.hk != 0) {
    float Hv[3];
    if (sd.hk == 1) {
      // spherical: (P - g g^T) vo / L, P = I except on a capsule's side (z row dropped)
      float L;
      bool side = false;
      if (po.type == OBJ_CAPSULE) {
        const float h = po.dims[1];
        const float qz = sd.qf[2];
        side = qz > -h && qz < h;
        const float cz = qz < -h ? -h : (qz > h ? h : qz);
        const float vz = qz - cz;
        L = sqrtf(sd.qf[0] * sd.qf[0] + sd.qf[1] * sd.qf[1] + vz * vz);
      } else {
        L = sqrtf(sd.qf[0] * sd.qf[0] + sd.qf[1] * sd.qf[1] + sd.qf[2] * sd.qf[2]);
      }
      Hv[0] = (vo[0] - sd.g[0] * gv) / L;
      Hv[1] = (vo[1] - sd.g[1] * gv) / L;
      Hv[2] = ((side ? 0.f : vo[2]) - sd.g[2] * gv) / L;
    } else {
      // radial about the z axis: (I_xy - g g^T) vo / rho
      const float rho = sqrtf(sd.qf[0] * sd.qf[0] + sd.qf[1] * sd.qf[1]);
      Hv[0] = (vo[0] - sd.g[0] * gv) / rho;
      Hv[1] = (vo[1] - sd.g[1] * gv) / rho;
      Hv[2] = 0.f;
    }
    for (int q = 0; q < 3; ++q) Av[q] = fmaf(phi, Hv[q], Av[q]);
  }
  float sw[3];
  for (int q = 0; q < 3; ++q) sw[q] = Rk[q][0] * Av[0] + Rk[q][1] * Av[1] + Rk[q][2] * Av[2];
  // r = x - t_k, x = R_pad p + t_pad (world)
  float r[3];
  for (int q = 0; q < 3; ++q)
    r[q] = Rp[q][0] * p.x + Rp[q][1] * p.y + Rp[q][2] * p.z + pp[q] - op[q];
  const float c1[3] = {r[1] * sw[2] - r[2] * sw[1], r[2] * sw[0] - r[0] * sw[2],
                       r[0] * sw[1] - r[1] * sw[0]};
  const float c2[3] = {gw[1] * v[2] - gw[2] * v[1], gw[2] * v[0] - gw[0] * v[2],
                       gw[0] * v[1] - gw[1] * v[0]};
  for (int q = 0; q < 3; ++q) {
    out.t[q] = sw[q];
    out.w[q] = c1[q] - phi * c2[q];
  }
  return out;
}

}  // namespace etac
