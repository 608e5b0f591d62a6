// backward.cu -- hand-written reverse mode (FP32) of the ETac step (ETac Sec. III-A, Eq. 1,
// Eq. 4; the paper's calibration, Eq. 5, differentiates the same quantities).
//
// For an upstream gradient G = dL/dU this computes dL/d(parameters), dL/d(u_hat) and
// dL/d(penetration) of the active nodes, and dL/d(object pose) (translation and a world-frame
// rotation increment applied on the left about the object origin), holding the contact set
// fixed (ReLU'(0) = 0, max-pool gradient to the lowest-index maximiser).
//
// One CTA per pad, pads assigned statically (CTA b takes work items b, b + G, ...), so every
// parameter-gradient partial is accumulated in a fixed order and the result is bitwise
// repeatable; no floating-point atomics.  Per pad:
//   0. recompute the forward: contact (same device functions as the forward, hence the same
//      contact set), encoder of the active nodes, max-pool argmax (active nodes vs. the first
//      passive node of each channel's table order, ties to the lower node index), global MLP;
//   1. decoder reverse over 64-node chunks of passive nodes: dA3 = ReLU'(h0 + beta) (D2^T G),
//      with the outer products dD1_f += dA3^T F0, dD2 += G^T Z3 as in-CTA GEMMs into per-CTA
//      accumulators, and S = sum dA3 for the global half;
//   2. global MLP reverse: dg = D1_g^T S, dG1, db_G1, dg0, routed to each channel's argmax;
//   3. encoder reverse of passive nodes (dF = D1_f^T dA3 + routed) and of the active argmax
//      nodes (routed only): dE2, dE1 (the u_hat columns from active nodes, giving dL/du_hat);
//   4. propagation reverse (warp per active node j): du_hat_j += sum_i Omega_ij G_i and
//      dalpha += -sum_i d_ij Omega_ij (G_i . u_hat_j) over passive i;
//   5. pose and penetration: u_hat = -phi n (object outward normal n), differentiated through
//      the primitive's SDF gradient and Hessian.
#include "bwd_common.cuh"
#include "etac_common.cuh"
#include "etac_kernels.h"

namespace etac {

namespace {

constexpr int BB = 256;
constexpr int BBW = BB / 32;
constexpr int CH = 64;        // nodes per chunk
constexpr int LD = TLD;

// shared-memory layout
struct BwdSmem {
  size_t acc, wdf, w2, w2t, sp, sq, sm, sd, sdt, xr, gr, vec, bits, route, rnode, best, cnt, po,
      total;
  __host__ __device__ BwdSmem(int nmax, int K) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    acc = take(sizeof(float) * NPARAM);
    wdf = take(sizeof(float) * H * LD);     // D1[:, 0:64] as [c][k]
    w2 = take(sizeof(float) * H * LD);      // E2 as [c][k]
    w2t = take(sizeof(float) * H * LD);     // E2 transposed, [k][c]
    sp = take(sizeof(float) * CH * LD);     // staging tiles (see the phases)
    sq = take(sizeof(float) * CH * LD);
    sm = take(sizeof(float) * CH * LD);
    sd = take(sizeof(float) * CH * LD);
    sdt = take(sizeof(float) * CH * LD);
    xr = take(sizeof(float) * CH * 12);     // per-row inputs X (9), valid flag, node
    gr = take(sizeof(float4) * CH);         // per-row G
    vec = take(sizeof(float) * 16 * H);     // g0, ag, g, beta, S, dg0, dag, tmp, alpha partials
    bits = take(sizeof(uint32_t) * (size_t)((nmax + 31) / 32));
    route = take(sizeof(int) * H);          // argmax node per channel
    rnode = take(sizeof(int) * (H + 4));    // distinct active argmax nodes
    best = take(sizeof(float2) * 16 * H);   // per (row block, channel) best (value, node)
    cnt = take(sizeof(int) * 16);
    po = take(sizeof(PadObj) * (size_t)K);
    total = o;
  }
};

enum { V_G0 = 0, V_AG = 1, V_G = 2, V_BETA = 3, V_S = 4, V_DG0 = 5, V_DAG = 6, V_TMP = 9,
       V_ALPHA = 10, V_BV = 11, V_BI = 12 };

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

__device__ __forceinline__ int find_slot(const int* idx, int m, int i) {
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (idx[mid] < i) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(BB, 1) backward_kernel(BackwardArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BwdSmem L(a.nmax, a.K);
  float* sAcc = reinterpret_cast<float*>(smem + L.acc);      // per-CTA parameter gradient
  float* sWdf = reinterpret_cast<float*>(smem + L.wdf);
  float* sW2 = reinterpret_cast<float*>(smem + L.w2);
  float* sW2T = reinterpret_cast<float*>(smem + L.w2t);
  float* sP = reinterpret_cast<float*>(smem + L.sp);
  float* sQ = reinterpret_cast<float*>(smem + L.sq);
  float* sM = reinterpret_cast<float*>(smem + L.sm);
  float* sD = reinterpret_cast<float*>(smem + L.sd);
  float* sDT = reinterpret_cast<float*>(smem + L.sdt);
  float* sX = reinterpret_cast<float*>(smem + L.xr);
  float4* sGr = reinterpret_cast<float4*>(smem + L.gr);
  float* sV = reinterpret_cast<float*>(smem + L.vec);
  uint32_t* sBits = reinterpret_cast<uint32_t*>(smem + L.bits);
  int* sRoute = reinterpret_cast<int*>(smem + L.route);
  int* sRNode = reinterpret_cast<int*>(smem + L.rnode);
  float2* sBest = reinterpret_cast<float2*>(smem + L.best);
  int* sCnt = reinterpret_cast<int*>(smem + L.cnt);
  PadObj* spo = reinterpret_cast<PadObj*>(smem + L.po);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* W = a.params;
  const float alpha = W[OFF_ALPHA];
  for (int i = tid; i < NPARAM; i += BB) sAcc[i] = 0.f;
  for (int i = tid; i < H * H; i += BB) {
    const int c = i >> 6, k = i & (H - 1);
    sWdf[c * LD + k] = W[OFF_WD + c * 2 * H + k];
    sW2[c * LD + k] = W[OFF_W2 + c * H + k];
    sW2T[k * LD + c] = W[OFF_W2 + c * H + k];
  }
  // staging threads: row tr, 16 columns from tq; GEMM threads: 4 x 4 tile (ti, tj)
  const int tr = tid >> 2, tq = (tid & 3) * 16;
  const int ti = tid >> 4, tj = tid & 15;
  const bool use_l = uses_propagation(a.mode), use_r = uses_residual(a.mode);
  float accWdf[4][4], accW2[4][4];   // per-CTA gradient tiles of D1[:, 0:64] and E2
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accWdf[i][j] = accW2[i][j] = 0.f;

  for (int item = blockIdx.x; item < a.num_items; item += gridDim.x) {
    __syncthreads();
    const int pad = a.item_pad[item];
    const int env = pad / a.P;
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const int nwords = (n + 31) >> 5;
    const long long base = a.pad_off[pad];
    const float* tpos = a.type_pos + 3 * (size_t)o;
    const float* tnrm = a.type_nrm + 3 * (size_t)o;
    int* wIdx = a.ws_idx + base;         // active node list of this pad (node order)
    float4* wU = a.ws_u + base;          // their u_hat (w = phi)
    float4* wDU = a.ws_du + base;        // their dL/du_hat
    if (tid == 0) {
      sCnt[0] = 0;   // active count
      sCnt[1] = 0;   // invalid flag
      sCnt[2] = 0;   // distinct active argmax nodes
    }
    for (int w = tid; w < nwords; w += BB) sBits[w] = 0u;
    for (int k = tid; k < a.K * 6; k += BB) a.pose_part[(size_t)pad * a.K * 6 + k] = 0.f;
    __syncthreads();
    const bool given = a.mask_in != nullptr;   // mode B: the forward's contact was supplied
    if (tid < a.K && !given) {
      const int ob = env * a.K + tid;
      const float* op = a.obj_pose + 7 * (size_t)ob;
      const float* pp = a.pad_pose + 7 * (size_t)pad;
      const float* od = a.obj_dims + 3 * (size_t)ob;
      int type = a.obj_type[ob];
      if (type < OBJ_NONE || type > OBJ_MESH) type = OBJ_NONE;
      const MeshDev* mesh = nullptr;
      if (type == OBJ_MESH && !(mesh = object_mesh(od, a.meshes, a.num_meshes))) type = OBJ_NONE;
      const bool ok = finite7(op) && finite7(pp) && isfinite(od[0]) && isfinite(od[1]) &&
                      isfinite(od[2]);
      if (!ok && type != OBJ_NONE) {
        sCnt[1] = 1;
        type = OBJ_NONE;
      }
      setup_pad_obj(op, type, od, pp, a.type_pmax[ty], &spo[tid], mesh);
    }
    __syncthreads();
    const bool invalid = sCnt[1] != 0;

    // ---- 0a. contact (the active list keeps node order: fixed summation order)
    for (int r0 = 0; r0 < n; r0 += BB) {
      const int i = r0 + tid;
      NodeContact c;
      c.active = false;
      if (i < n && !invalid)
        c = given ? contact_given(a.mask_in, a.uhat_in, base + i)
                  : contact_node(spo, a.K, make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]),
                                 make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]));
      const unsigned bal = __ballot_sync(0xffffffffu, c.active);
      if (lane == 0) {
        sCnt[4 + warp] = __popc(bal);
        if (((r0 >> 5) + warp) < nwords) sBits[(r0 >> 5) + warp] = bal;
      }
      __syncthreads();
      int woff = 0, tot = 0;
      for (int w = 0; w < BBW; ++w) {
        woff += w < warp ? sCnt[4 + w] : 0;
        tot += sCnt[4 + w];
      }
      if (c.active) {
        const int slot = sCnt[0] + woff + __popc(bal & ((1u << lane) - 1u));
        wIdx[slot] = i;
        wU[slot] = make_float4(c.u[0], c.u[1], c.u[2], c.phi);
      }
      __syncthreads();
      if (tid == 0) sCnt[0] += tot;
      __syncthreads();
    }
    const int m = sCnt[0];
    if (m == 0) {   // the pad outputs zero: no gradient flows
      for (int i = tid; i < n; i += BB) {
        if (a.grad_uhat) {
          float* g = a.grad_uhat + 3 * (base + i);
          g[0] = g[1] = g[2] = 0.f;
        }
        if (a.grad_pen) a.grad_pen[base + i] = 0.f;
      }
      continue;
    }
    // direct term: active nodes output u_hat itself
    for (int s = tid; s < m; s += BB) {
      const int i = wIdx[s];
      const float* G = a.grad_disp + 3 * (base + i);
      wDU[s] = make_float4(G[0], G[1], G[2], 0.f);
    }

    if (use_r) {
      // ---- 0b. forward of the network: encoder of the active nodes (4 x 4 GEMM tiles),
      // channel maxima and their lowest-index argmax
      if (tid < H) {
        sV[V_BV * H + tid] = -1.f;
        reinterpret_cast<int*>(sV)[V_BI * H + tid] = 0x7fffffff;
      }
      for (int s0 = 0; s0 < m; s0 += CH) {
        {
          const int s = s0 + tr;
          const bool valid = s < m;
          const int i = valid ? wIdx[s] : 0;
          const float4 u = valid ? wU[s] : make_float4(0.f, 0.f, 0.f, 0.f);
          for (int x = 0; x < 16; ++x) {
            const int c = tq + x;
            const float a1 = a.ctab[(size_t)(o + i) * H + c] + W[OFF_W1 + c * NIN + 6] * u.x +
                             W[OFF_W1 + c * NIN + 7] * u.y + W[OFF_W1 + c * NIN + 8] * u.z;
            sP[c * LD + tr] = relu(a1);   // Z1^T [k][r]
          }
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        tile_acc(sP, sW2T, ti, tj, acc);   // a2[r][c] - b2[c], rows 4ti.., channels 4tj..
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = 4 * tj + j;
          float bv = -1.f;
          int bi = 0x7fffffff;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int s = s0 + 4 * ti + i;
            if (s < m) {
              const float f = relu(acc[i][j] + W[OFF_B2 + c]);
              const int node = wIdx[s];
              if (f > bv || (f == bv && node < bi)) {
                bv = f;
                bi = node;
              }
            }
          }
          sBest[ti * H + c] = make_float2(bv, __int_as_float(bi));
        }
        __syncthreads();
        if (tid < H) {
          float bv = sV[V_BV * H + tid];
          int bi = reinterpret_cast<int*>(sV)[V_BI * H + tid];
          for (int r = 0; r < 16; ++r) {
            const float2 e = sBest[r * H + tid];
            const int node = __float_as_int(e.y);
            if (e.x > bv || (e.x == bv && node < bi)) {
              bv = e.x;
              bi = node;
            }
          }
          sV[V_BV * H + tid] = bv;
          reinterpret_cast<int*>(sV)[V_BI * H + tid] = bi;
        }
        __syncthreads();
      }
      // passive candidate: first passive node in each channel's ranked order (ties to the
      // lower index), 32 ranks per warp-wide test, 8 channels per warp
      for (int cc = 0; cc < 8; ++cc) {
        const int c = warp * 8 + cc;
        float pv = -1.f;
        int pi = 0x7fffffff;
        for (int r0 = 0; r0 < n; r0 += 32) {
          const int r = r0 + lane;
          float2 e = make_float2(0.f, __int_as_float(0));
          bool passive = false;
          if (r < n) {
            e = a.ranked[(size_t)H * o + (size_t)c * n + r];
            const int idx = __float_as_int(e.y);
            passive = !((sBits[idx >> 5] >> (idx & 31)) & 1u);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, passive);
          if (bal) {
            const int src = __ffs(bal) - 1;
            pv = __shfl_sync(0xffffffffu, e.x, src);
            pi = __float_as_int(__shfl_sync(0xffffffffu, e.y, src));
            break;
          }
        }
        if (lane == 0) {
          float bv = sV[V_BV * H + c];
          int bi = reinterpret_cast<int*>(sV)[V_BI * H + c];
          if (pv > bv || (pv == bv && pi < bi)) {
            bv = pv;
            bi = pi;
          }
          sV[V_G0 * H + c] = bv;
          sRoute[c] = bi;
        }
      }
      __syncthreads();
      if (tid < H) {
        float acc = W[OFF_BG + tid];
        for (int k = 0; k < H; ++k) acc = fmaf(W[OFF_WG + tid * H + k], sV[V_G0 * H + k], acc);
        sV[V_AG * H + tid] = acc;
        sV[V_G * H + tid] = relu(acc);
      }
      __syncthreads();
      if (tid < H) {
        float acc = 0.f;
        for (int k = 0; k < H; ++k) acc = fmaf(W[OFF_WD + tid * 2 * H + H + k], sV[V_G * H + k], acc);
        sV[V_BETA * H + tid] = acc;
        sV[V_S * H + tid] = 0.f;
      }
      __syncthreads();

      // ---- 1. decoder reverse over chunks of passive nodes
      for (int i0 = 0; i0 < n; i0 += CH) {
        {
          const int i = i0 + tr;
          const bool valid = i < n && !((sBits[i >> 5] >> (i & 31)) & 1u);
          float G0 = 0.f, G1 = 0.f, G2 = 0.f;
          if (valid) {
            const float* G = a.grad_disp + 3 * (base + i);
            G0 = G[0];
            G1 = G[1];
            G2 = G[2];
          }
          if (tq == 0) sGr[tr] = make_float4(G0, G1, G2, 0.f);
          for (int x = 0; x < 16; ++x) {
            const int c = tq + x;
            float da3 = 0.f, z3 = 0.f, f0 = 0.f;
            if (valid) {
              const float h = a.h0tab[(size_t)(o + i) * H + c] + sV[V_BETA * H + c];
              const float dz3 = W[OFF_W4 + c] * G0 + W[OFF_W4 + H + c] * G1 + W[OFF_W4 + 2 * H + c] * G2;
              da3 = h > 0.f ? dz3 : 0.f;
              z3 = relu(h);
              f0 = a.f0tab[(size_t)(o + i) * H + c];
            }
            sD[tr * LD + c] = da3;   // dA3 [r][c]
            sM[tr * LD + c] = z3;    // Z3 [r][c]
            sQ[tr * LD + c] = f0;    // F0 [r][k]
          }
        }
        __syncthreads();
        tile_acc(sD, sQ, ti, tj, accWdf);   // dD1_f[c][k] += sum_r dA3[r][c] F0[r][k]
        if (tid < H) {
          float sd = 0.f;
          for (int r = 0; r < CH; ++r) sd += sD[r * LD + tid];
          sAcc[OFF_BD + tid] += sd;
          sV[V_S * H + tid] += sd;
        }
        if (tid < 3 * H) {
          const int q = tid / H, c = tid % H;
          float s2 = 0.f;
          for (int r = 0; r < CH; ++r) {
            const float4 g = sGr[r];
            s2 = fmaf(q == 0 ? g.x : (q == 1 ? g.y : g.z), sM[r * LD + c], s2);
          }
          sAcc[OFF_W4 + q * H + c] += s2;
        }
        if (tid < 3) {
          float sb = 0.f;
          for (int r = 0; r < CH; ++r) {
            const float4 g = sGr[r];
            sb += tid == 0 ? g.x : (tid == 1 ? g.y : g.z);
          }
          sAcc[OFF_B4 + tid] += sb;
        }
        __syncthreads();
      }

      // ---- 2. global MLP reverse
      if (tid < H) {
        float dg = 0.f;
        for (int c = 0; c < H; ++c) dg = fmaf(W[OFF_WD + c * 2 * H + H + tid], sV[V_S * H + c], dg);
        sV[V_DAG * H + tid] = sV[V_AG * H + tid] > 0.f ? dg : 0.f;
      }
      __syncthreads();
      {
        const float sr = sV[V_S * H + tr], dr = sV[V_DAG * H + tr];
#pragma unroll
        for (int x = 0; x < 16; ++x) {
          const int k = tq + x;
          sAcc[OFF_WD + tr * 2 * H + H + k] += sr * sV[V_G * H + k];
          sAcc[OFF_WG + tr * H + k] += dr * sV[V_G0 * H + k];
        }
      }
      if (tid < H) {
        sAcc[OFF_BG + tid] += sV[V_DAG * H + tid];
        float dg0 = 0.f;
        for (int c = 0; c < H; ++c) dg0 = fmaf(W[OFF_WG + c * H + tid], sV[V_DAG * H + c], dg0);
        sV[V_DG0 * H + tid] = dg0;
      }
      __syncthreads();
      if (tid == 0) {
        int cnt = 0;
        for (int c = 0; c < H; ++c) {
          const int i = sRoute[c];
          if (i < 0 || i >= n || !((sBits[i >> 5] >> (i & 31)) & 1u)) continue;
          bool seen = false;
          for (int q = 0; q < cnt; ++q) seen |= sRNode[q] == i;
          if (!seen) sRNode[cnt++] = i;
        }
        sCnt[2] = cnt;
      }
      __syncthreads();

      // ---- 3. encoder reverse: passive chunks, then one chunk of active argmax nodes
      const int nchunks = (n + CH - 1) / CH;
      for (int ck = 0; ck <= nchunks; ++ck) {
        const bool act_chunk = ck == nchunks;
        if (act_chunk && sCnt[2] == 0) break;
        {
          int i = 0;
          bool valid;
          float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
          if (!act_chunk) {
            i = ck * CH + tr;
            valid = i < n && !((sBits[i >> 5] >> (i & 31)) & 1u);
          } else {
            valid = tr < sCnt[2];
            i = valid ? sRNode[tr] : 0;
            if (valid) u = wU[find_slot(wIdx, m, i)];
          }
          if (tq == 0) {
            float* xr = sX + tr * 12;
            for (int q = 0; q < 3; ++q) {
              xr[q] = valid ? tpos[3 * i + q] : 0.f;
              xr[3 + q] = valid ? tnrm[3 * i + q] : 0.f;
            }
            xr[6] = u.x;
            xr[7] = u.y;
            xr[8] = u.z;
            xr[9] = valid ? 1.f : 0.f;
            xr[10] = __int_as_float(i);
          }
          float G0 = 0.f, G1 = 0.f, G2 = 0.f;
          if (valid && !act_chunk) {
            const float* G = a.grad_disp + 3 * (base + i);
            G0 = G[0];
            G1 = G[1];
            G2 = G[2];
          }
          for (int x = 0; x < 16; ++x) {
            const int c = tq + x;
            float da3 = 0.f, z1 = 0.f, f0 = 0.f;
            if (valid) {
              if (!act_chunk) {
                const float h = a.h0tab[(size_t)(o + i) * H + c] + sV[V_BETA * H + c];
                const float dz3 = W[OFF_W4 + c] * G0 + W[OFF_W4 + H + c] * G1 + W[OFF_W4 + 2 * H + c] * G2;
                da3 = h > 0.f ? dz3 : 0.f;
                f0 = a.f0tab[(size_t)(o + i) * H + c];   // passive: f0 > 0 <=> a2 > 0
              }
              const float a1 = a.ctab[(size_t)(o + i) * H + c] + W[OFF_W1 + c * NIN + 6] * u.x +
                               W[OFF_W1 + c * NIN + 7] * u.y + W[OFF_W1 + c * NIN + 8] * u.z;
              z1 = relu(a1);
            }
            sP[c * LD + tr] = da3;   // dA3^T [c][r]
            sQ[tr * LD + c] = z1;    // Z1 [r][k]
            sM[tr * LD + c] = f0;    // mask source [r][k]
          }
        }
        __syncthreads();
        if (act_chunk) {
          // active rows: a2 = E2 z1 + b2 recomputed (routed gradient only, few rows)
          for (int x = 0; x < 16; ++x) {
            const int k = tq + x;
            float a2 = W[OFF_B2 + k];
            for (int c = 0; c < H; ++c) a2 = fmaf(sW2[k * LD + c], sQ[tr * LD + c], a2);
            sM[tr * LD + k] = relu(a2);
          }
          __syncthreads();
        }
        {
          // dF = dA3 D1_f (+ routed dg0); dA2 = dF * [a2 > 0] in both layouts
          float acc[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
          tile_acc(sP, sWdf, ti, tj, acc);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = 4 * ti + i;
            const int node = __float_as_int(sX[r * 12 + 10]);
            const bool valid = sX[r * 12 + 9] != 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int k = 4 * tj + j;
              float df = acc[i][j];
              if (sRoute[k] == node) df += sV[V_DG0 * H + k];
              const float da2 = (valid && sM[r * LD + k] > 0.f) ? df : 0.f;
              sD[r * LD + k] = da2;
              sDT[k * LD + r] = da2;
            }
          }
        }
        __syncthreads();
        {
          tile_acc(sD, sQ, ti, tj, accW2);   // dE2[c][k] += sum_r dA2[r][c] Z1[r][k]
          if (tid < H) {
            float sd = 0.f;
            for (int r = 0; r < CH; ++r) sd += sD[r * LD + tid];
            sAcc[OFF_B2 + tid] += sd;
          }
          // dZ1 = dA2 E2 ; dA1 = dZ1 * [z1 > 0] (into sP as [r][k]; dA3^T is no longer needed)
          float acc[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
          tile_acc(sDT, sW2, ti, tj, acc);
          __syncthreads();
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int r = 4 * ti + i, k = 4 * tj + j;
              sP[r * LD + k] = sQ[r * LD + k] > 0.f ? acc[i][j] : 0.f;
            }
        }
        __syncthreads();
        {
          // dE1 += dA1^T X ; db1 ; for active rows dL/du_hat += E1[:, 6:9]^T dA1
          for (int e = tid; e < H * 10; e += BB) {
            const int c = e / 10, col = e % 10;
            if (!act_chunk && col >= 6 && col < 9) continue;   // passive u_hat is zero
            float s = 0.f;
            for (int r = 0; r < CH; ++r) {
              const float xv = col < 9 ? sX[r * 12 + col] : 1.f;
              s = fmaf(sP[r * LD + c], xv, s);
            }
            if (col < 9) sAcc[OFF_W1 + c * NIN + col] += s;
            else sAcc[OFF_B1 + c] += s;
          }
          if (act_chunk && tid < sCnt[2] * 3) {
            const int r = tid / 3, q = tid % 3;
            float s = 0.f;
            for (int c = 0; c < H; ++c) s = fmaf(W[OFF_W1 + c * NIN + 6 + q], sP[r * LD + c], s);
            const int i = __float_as_int(sX[r * 12 + 10]);
            float* du = reinterpret_cast<float*>(&wDU[find_slot(wIdx, m, i)]);
            du[q] += s;   // rows are distinct nodes: no two threads share (slot, q)
          }
        }
        __syncthreads();
      }
    }

    // ---- 4. propagation reverse: warp per active node
    if (use_l) {
      float walpha = 0.f;
      for (int s = warp; s < m; s += BBW) {
        const int j = wIdx[s];
        const float4 uj = wU[s];
        const float pjx = tpos[3 * j], pjy = tpos[3 * j + 1], pjz = tpos[3 * j + 2];
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, da = 0.f;
        for (int i = lane; i < n; i += 32) {
          if ((sBits[i >> 5] >> (i & 31)) & 1u) continue;
          const float dx = pjx - tpos[3 * i], dy = pjy - tpos[3 * i + 1], dz = pjz - tpos[3 * i + 2];
          const float d = sqrtf(dx * dx + dy * dy + dz * dz);
          const float w = expf(-alpha * d);
          const float* G = a.grad_disp + 3 * (base + i);
          d0 = fmaf(w, G[0], d0);
          d1 = fmaf(w, G[1], d1);
          d2 = fmaf(w, G[2], d2);
          da = fmaf(-d * w, G[0] * uj.x + G[1] * uj.y + G[2] * uj.z, da);
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
          d0 += __shfl_xor_sync(0xffffffffu, d0, sh);
          d1 += __shfl_xor_sync(0xffffffffu, d1, sh);
          d2 += __shfl_xor_sync(0xffffffffu, d2, sh);
          da += __shfl_xor_sync(0xffffffffu, da, sh);
        }
        if (lane == 0) {
          float4 du = wDU[s];
          du.x += d0;
          du.y += d1;
          du.z += d2;
          wDU[s] = du;
        }
        walpha += da;
      }
      if (lane == 0) sV[V_ALPHA * H + warp] = walpha;
      __syncthreads();
      if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < BBW; ++w) t += sV[V_ALPHA * H + w];
        sAcc[OFF_ALPHA] += t;
      }
    }
    __syncthreads();

    // ---- 5. outputs per node, penetration and pose through the SDF
    for (int i = tid; i < n; i += BB) {
      if ((sBits[i >> 5] >> (i & 31)) & 1u) continue;
      if (a.grad_uhat) {
        float* g = a.grad_uhat + 3 * (base + i);
        g[0] = g[1] = g[2] = 0.f;
      }
      if (a.grad_pen) a.grad_pen[base + i] = 0.f;
    }
    float pose[MAX_K][6];
#pragma unroll
    for (int k = 0; k < MAX_K; ++k)
#pragma unroll
      for (int q = 0; q < 6; ++q) pose[k][q] = 0.f;
    const float* pp = given ? nullptr : a.pad_pose + 7 * (size_t)pad;
    float Rp[3][3] = {};
    if (!given) quat_to_mat<float>(pp + 3, Rp);
    for (int s = tid; s < m; s += BB) {
      const int i = wIdx[s];
      const float4 du = wDU[s];
      const float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
      const float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
      NodePoseGrad pg;
      pg.k = -1;   // mode B: no SDF, so no penetration or pose gradient
      pg.pen = 0.f;
      if (!given)
        pg = node_pose_grad(spo, a.K, p, nr, make_float3(du.x, du.y, du.z), Rp, pp,
                            a.obj_pose + 7 * (size_t)env * a.K);
      if (a.grad_uhat) {
        float* g = a.grad_uhat + 3 * (base + i);
        g[0] = du.x;
        g[1] = du.y;
        g[2] = du.z;
      }
      if (a.grad_pen) a.grad_pen[base + i] = pg.pen;
#pragma unroll
      for (int k = 0; k < MAX_K; ++k) {
        if (k != pg.k) continue;
        for (int q = 0; q < 3; ++q) {
          pose[k][q] += pg.t[q];
          pose[k][3 + q] += pg.w[q];
        }
      }
    }
    // fixed-order block reduction of the pose partials (warp shuffles, then warps in order)
    for (int k = 0; k < a.K; ++k) {
      for (int q = 0; q < 6; ++q) {
        float v = pose[k][q];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
        if (lane == 0) sV[V_TMP * H + warp] = v;
        __syncthreads();
        if (tid == 0) {
          float t = 0.f;
          for (int w = 0; w < BBW; ++w) t += sV[V_TMP * H + w];
          a.pose_part[((size_t)pad * a.K + k) * 6 + q] = t;
        }
        __syncthreads();
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * ti + i, k = 4 * tj + j;
      sAcc[OFF_WD + c * 2 * H + k] += accWdf[i][j];
      sAcc[OFF_W2 + c * H + k] += accW2[i][j];
    }
  __syncthreads();
  for (int i = tid; i < NPARAM; i += BB) a.param_part[(size_t)blockIdx.x * NPARAM + i] = sAcc[i];
}

// grad_params[q] = sum over CTAs b (in order) of the partials
__global__ void reduce_params_kernel(const float* part, int nparts, float* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPARAM) return;
  float s = 0.f;
  for (int b = 0; b < nparts; ++b) s += part[(size_t)b * NPARAM + q];
  out[q] = s;
}

// grad_obj_pose[e][k][q] = sum over the env's pads (in order) of the pad partials
__global__ void reduce_pose_kernel(const float* part, int E, int P, int K, float* out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)E * K * 6) return;
  const int e = (int)(t / (K * 6)), r = (int)(t % (K * 6));
  float s = 0.f;
  for (int p = 0; p < P; ++p) s += part[((size_t)(e * P + p)) * K * 6 + r];
  out[t] = s;
}

// dL/dq from dL/domega for R(q/|q|) with a left increment: dq = (1/2) (omega ⊗ q) for unit q,
// i.e. omega = 2 vec(dq ⊗ conj(q)) / |q|^2, so dL/dq_v = 2 (q_w g - q_v x g) / |q|^2 and
// dL/dq_w = -2 (g . q_v) / |q|^2 (the radial direction, which does not rotate, gets zero).
__global__ void pose_grad_to_quat_kernel(const float* poses, const float* tw, float* out,
                                         long long count) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= count) return;
  const float* q = poses + 7 * t + 3;
  const float* g = tw + 6 * t + 3;
  const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const float s = n2 > 0.f ? 2.f / n2 : 0.f;
  const float cx = q[1] * g[2] - q[2] * g[1], cy = q[2] * g[0] - q[0] * g[2],
              cz = q[0] * g[1] - q[1] * g[0];
  float* o = out + 7 * t;
  o[0] = tw[6 * t + 0];
  o[1] = tw[6 * t + 1];
  o[2] = tw[6 * t + 2];
  o[3] = s * (q[3] * g[0] - cx);
  o[4] = s * (q[3] * g[1] - cy);
  o[5] = s * (q[3] * g[2] - cz);
  o[6] = -s * (g[0] * q[0] + g[1] * q[1] + g[2] * q[2]);
}

}  // namespace

cudaError_t launch_pose_grad_to_quat(const float* poses, const float* tw, float* out,
                                     long long count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  pose_grad_to_quat_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(poses, tw, out, count);
  return cudaGetLastError();
}

size_t backward_smem_bytes(int nmax, int K) { return BwdSmem(nmax, K).total; }

cudaError_t launch_reduce_pose(const float* part, int E, int P, int K, float* out, cudaStream_t s) {
  const long long tot = (long long)E * K * 6;
  if (tot <= 0) return cudaSuccess;
  reduce_pose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(part, E, P, K, out);
  return cudaGetLastError();
}

cudaError_t launch_backward(const BackwardArgs& a, int grid, cudaStream_t s) {
  const size_t smem = backward_smem_bytes(a.nmax, a.K);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(backward_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  backward_kernel<<<grid, BB, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.grad_params) {
    reduce_params_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(a.param_part, grid, a.grad_params);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.grad_obj_pose) {
    const long long tot = (long long)a.E * a.K * 6;
    reduce_pose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a.pose_part, a.E, a.P, a.K,
                                                                      a.grad_obj_pose);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace etac
