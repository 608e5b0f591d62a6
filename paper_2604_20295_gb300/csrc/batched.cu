// batched.cu -- the batched FP32 ETac step: one persistent launch over every pad of the batch.
//
// Work items are pad instances ordered heaviest first (largest node count); persistent CTAs
// take them from a device ticket counter, so pads of uneven size balance across the SMs.
// Per pad (ETac Sec. III-A):
//   1. contact on every node (df32 decisions), active set compacted in node order with warp
//      ballots; active nodes keep u_hat (Eq. 4 only covers passive ones);
//   2. residual network, factored through the per-type tables: only active nodes run the
//      encoder (their first layer is c_i + W1[:, 6:9] u_hat_i); passive nodes' encoder
//      outputs f0_i are table entries, so the channel max-pool over them is the first
//      passive node in the table's per-channel order; global MLP; decoder global half
//      beta = D1[:, 64:128] g;
//   3. every passive node: Omega U_a (Eq. 1, Omega from the per-type table) plus
//      Phi_p = D2 ReLU(h0_i + beta) + b (Eq. 4).
// The algebra equals the literal network exactly; only rounding order differs.
#include <cuda_bf16.h>

#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {

constexpr int BT = 256;
constexpr int BW = BT / 32;

struct BatchedSmem {
  // byte offsets of every shared array for a given nmax / K
  size_t w2, b2, w1u, w4, b4, g, beta, red, w2frag, actu, actidx, mask, warp, po, total;
  __host__ __device__ BatchedSmem(int nmax, int K) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    w2 = take(sizeof(float) * H * H);
    b2 = take(sizeof(float) * H);
    w1u = take(sizeof(float) * H * 4);
    w4 = take(sizeof(float) * 3 * H);
    b4 = take(sizeof(float) * 4);
    g = take(sizeof(float) * H);
    beta = take(sizeof(float) * H);
    red = take(sizeof(float) * BW * H);
    w2frag = take(sizeof(uint2) * 8 * 4 * 32);
    actu = take(sizeof(float4) * (size_t)nmax);
    actidx = take(sizeof(int16_t) * (size_t)nmax);
    mask = take(sizeof(uint8_t) * (size_t)nmax);
    warp = take(sizeof(int) * (BW + 4));
    po = take(sizeof(PadObj) * (size_t)K);
    total = o;
  }
};

// kBF16 = false: the whole FP32 step.  kBF16 = true: the front half of the BF16 tensor-core
// step -- contact, encoder, pooling and global MLP -- writing the GEMM's B operand (u_hat in
// BF16, zero on passive nodes), the contact mask and each pad's decoder record.
template <bool kBF16>
__global__ void __launch_bounds__(BT, 2) batched_forward_kernel(BatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const BatchedSmem L(a.nmax, a.K);
  float* sW2 = reinterpret_cast<float*>(smem + L.w2);
  float* sB2 = reinterpret_cast<float*>(smem + L.b2);
  float* sW1u = reinterpret_cast<float*>(smem + L.w1u);   // [H][4]: weights on u_hat
  float* sW4 = reinterpret_cast<float*>(smem + L.w4);
  float* sB4 = reinterpret_cast<float*>(smem + L.b4);
  float* sG = reinterpret_cast<float*>(smem + L.g);
  float* sBeta = reinterpret_cast<float*>(smem + L.beta);
  float* sRed = reinterpret_cast<float*>(smem + L.red);
  float4* sActU = reinterpret_cast<float4*>(smem + L.actu);
  int16_t* sActIdx = reinterpret_cast<int16_t*>(smem + L.actidx);
  uint8_t* sMask = reinterpret_cast<uint8_t*>(smem + L.mask);
  int* sWarp = reinterpret_cast<int*>(smem + L.warp);
  PadObj* spo = reinterpret_cast<PadObj*>(smem + L.po);
  uint2* sW2f = reinterpret_cast<uint2*>(smem + L.w2frag);  // BF16 B fragments of E2

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* W = a.params;
  for (int i = tid; i < H * H; i += BT) sW2[i] = W[OFF_W2 + i];
  for (int i = tid; i < H; i += BT) {
    sB2[i] = W[OFF_B2 + i];
    sW1u[4 * i + 0] = W[OFF_W1 + i * NIN + 6];
    sW1u[4 * i + 1] = W[OFF_W1 + i * NIN + 7];
    sW1u[4 * i + 2] = W[OFF_W1 + i * NIN + 8];
    sW1u[4 * i + 3] = 0.f;
  }
  for (int i = tid; i < 3 * H; i += BT) sW4[i] = W[OFF_W4 + i];
  if (tid < 3) sB4[tid] = W[OFF_B4 + tid];
  if constexpr (kBF16) {
    // E2 as m16n8k16 B fragments: B[k = input unit][n = output unit] = W2[n][k]; entry
    // (nt, s, l) holds lane l's two registers for output tile nt and input step s
    for (int e = tid; e < 8 * 4 * 32; e += BT) {
      const int l = e & 31, s4 = (e >> 5) & 3, nt = e >> 7;
      const int n = 8 * nt + (l >> 2), k = 16 * s4 + 2 * (l & 3);
      __nv_bfloat162 lo = __floats2bfloat162_rn(W[OFF_W2 + n * H + k], W[OFF_W2 + n * H + k + 1]);
      __nv_bfloat162 hi =
          __floats2bfloat162_rn(W[OFF_W2 + n * H + k + 8], W[OFF_W2 + n * H + k + 9]);
      sW2f[e] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
    }
  }
  const unsigned lt_mask = (1u << lane) - 1u;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = atomicAdd(a.ticket, 1);
      sWarp[BW] = 0;   // invalid-input flag
    }
    __syncthreads();
    const int item = s_item;
    if (item >= a.num_items) break;
    const int pad = a.item_pad[item];
    const int env = pad / a.P;
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const long long base = a.pad_off[pad];
    const float* tpos = a.type_pos + 3 * (size_t)o;
    const float* tnrm = a.type_nrm + 3 * (size_t)o;

    if (tid < a.K) {
      const int ob = env * a.K + tid;
      const float* op = a.obj_pose + 7 * (size_t)ob;
      const float* pp = a.pad_pose + 7 * (size_t)pad;
      const float* od = a.obj_dims + 3 * (size_t)ob;
      int type = a.obj_type[ob];
      if (type < OBJ_NONE || type > OBJ_CAPSULE) type = OBJ_NONE;
      bool ok = finite7(op) && finite7(pp) && isfinite(od[0]) && isfinite(od[1]) &&
                isfinite(od[2]);
      if (!ok && type != OBJ_NONE) {
        sWarp[BW] = 1;
        type = OBJ_NONE;
      }
      setup_pad_obj(op, type, od, pp, a.type_pmax[ty], &spo[tid]);
    }
    __syncthreads();
    __nv_bfloat16* btrow = nullptr;   // BF16 variant: rows 3k..3k+2 of the B operand
    if constexpr (kBF16)
      btrow = reinterpret_cast<__nv_bfloat16*>(a.bt) + a.bt_off[ty] + (size_t)3 * a.pad_inst[pad] * n;
    if (sWarp[BW]) {
      if (tid == 0) latch_status(a.status, STATUS_NONFINITE);
      for (int i = tid; i < n; i += BT) {
        float* d = a.disp + 3 * (base + i);
        d[0] = d[1] = d[2] = 0.f;
        if (a.mask) a.mask[base + i] = 0;
        if (a.pen) a.pen[base + i] = 0.f;
        if constexpr (kBF16) {
          const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
          btrow[i] = z;
          btrow[n + i] = z;
          btrow[2 * n + i] = z;
        }
      }
      if constexpr (kBF16)
        for (int w = tid; w < (n + 31) / 32; w += BT) a.maskbits[a.mask_woff[pad] + w] = 0u;
      if (tid == 0 && a.count) a.count[pad] = 0;
      if constexpr (kBF16)
        if (tid == 0) a.c0m[pad] = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
      continue;
    }

    // ---- 1. contact; active set in node order
    int m = 0;
    for (int r0 = 0; r0 < n; r0 += BT) {
      const int i = r0 + tid;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      if (i < n) {
        float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
        float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
        c = contact_node(spo, a.K, p, nr);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, c.active);
      if (lane == 0) sWarp[warp] = __popc(bal);
      if constexpr (kBF16) {
        const int w = (r0 >> 5) + warp;
        if (lane == 0 && w < (n + 31) / 32) a.maskbits[a.mask_woff[pad] + w] = bal;
      }
      __syncthreads();
      int woff = 0, tot = 0;
#pragma unroll
      for (int w = 0; w < BW; ++w) {
        const int v = sWarp[w];
        woff += w < warp ? v : 0;
        tot += v;
      }
      if (i < n) {
        sMask[i] = c.active ? 1 : 0;
        if (a.mask) a.mask[base + i] = c.active ? 1 : 0;
        if constexpr (kBF16) {
          btrow[i] = __float2bfloat16_rn(c.u[0]);
          btrow[n + i] = __float2bfloat16_rn(c.u[1]);
          btrow[2 * n + i] = __float2bfloat16_rn(c.u[2]);
        }
        if (a.pen) a.pen[base + i] = c.active ? -c.phi : 0.f;
        if (c.active) {
          const int slot = m + woff + __popc(bal & lt_mask);
          sActIdx[slot] = (int16_t)i;
          sActU[slot] = make_float4(c.u[0], c.u[1], c.u[2], 0.f);
          float* d = a.disp + 3 * (base + i);
          d[0] = c.u[0];
          d[1] = c.u[1];
          d[2] = c.u[2];
        }
      }
      m += tot;
      __syncthreads();
    }
    if (tid == 0 && a.count) a.count[pad] = m;
    if (m == 0) {   // no contact: the whole pad is at rest
      for (int i = tid; i < n; i += BT) {
        float* d = a.disp + 3 * (base + i);
        d[0] = d[1] = d[2] = 0.f;
      }
      if constexpr (kBF16)
        if (tid == 0) a.c0m[pad] = make_float4(0.f, 0.f, 0.f, __int_as_float(0));
      continue;
    }

    // ---- 2. residual network (factored)
    if (a.mode != MODE_LINEAR_ONLY) {
      if constexpr (kBF16) {
        // encoder on tensor cores: 16 active nodes per warp step; E1 (c_i + W1u u_hat) is
        // evaluated directly in the A-fragment layout of m16n8k16, E2 by 32 BF16 MMAs with
        // FP32 accumulators, then ReLU and a running channel maximum per thread
        const int grp = lane >> 2, tig = lane & 3;
        float fm[8][2];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) fm[nt][0] = fm[nt][1] = 0.f;
        for (int g = warp; g * 16 < m; g += BW) {
          const int s0 = 16 * g + grp, s1 = s0 + 8;
          const bool v0 = s0 < m, v1 = s1 < m;
          const int n0 = v0 ? sActIdx[s0] : 0, n1 = v1 ? sActIdx[s1] : 0;
          const float4 u0 = v0 ? sActU[s0] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 u1 = v1 ? sActU[s1] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float* c0r = a.ctab + (size_t)(o + n0) * H;
          const float* c1r = a.ctab + (size_t)(o + n1) * H;
          uint32_t af[4][4];
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              const int col = 16 * s4 + 8 * hh + 2 * tig;
              const float2 ca = __ldg(reinterpret_cast<const float2*>(c0r + col));
              const float2 cb = __ldg(reinterpret_cast<const float2*>(c1r + col));
              const float4 w0 = *reinterpret_cast<const float4*>(sW1u + 4 * col);
              const float4 w1 = *reinterpret_cast<const float4*>(sW1u + 4 * (col + 1));
              const float z00 = fmaxf(fmaf(w0.x, u0.x, fmaf(w0.y, u0.y, fmaf(w0.z, u0.z, ca.x))), 0.f);
              const float z01 = fmaxf(fmaf(w1.x, u0.x, fmaf(w1.y, u0.y, fmaf(w1.z, u0.z, ca.y))), 0.f);
              const float z10 = fmaxf(fmaf(w0.x, u1.x, fmaf(w0.y, u1.y, fmaf(w0.z, u1.z, cb.x))), 0.f);
              const float z11 = fmaxf(fmaf(w1.x, u1.x, fmaf(w1.y, u1.y, fmaf(w1.z, u1.z, cb.y))), 0.f);
              __nv_bfloat162 p0 = __floats2bfloat162_rn(z00, z01);
              __nv_bfloat162 p1 = __floats2bfloat162_rn(z10, z11);
              af[s4][2 * hh + 0] = *reinterpret_cast<uint32_t*>(&p0);
              af[s4][2 * hh + 1] = *reinterpret_cast<uint32_t*>(&p1);
            }
          }
#pragma unroll
          for (int nt = 0; nt < 8; ++nt) {
            const float bx = sB2[8 * nt + 2 * tig], by = sB2[8 * nt + 2 * tig + 1];
            float acc[4] = {bx, by, bx, by};
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
              const uint2 bb = sW2f[(nt * 4 + s4) * 32 + lane];
              sm100::mma_bf16_16816(acc, af[s4], bb.x, bb.y, acc);
            }
            const float f00 = v0 ? fmaxf(acc[0], 0.f) : 0.f, f01 = v0 ? fmaxf(acc[1], 0.f) : 0.f;
            const float f10 = v1 ? fmaxf(acc[2], 0.f) : 0.f, f11 = v1 ? fmaxf(acc[3], 0.f) : 0.f;
            fm[nt][0] = fmaxf(fm[nt][0], fmaxf(f00, f10));
            fm[nt][1] = fmaxf(fm[nt][1], fmaxf(f01, f11));
          }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            float v = fm[nt][e];
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 4));
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 8));
            v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 16));
            if (grp == 0) sRed[warp * H + 8 * nt + 2 * tig + e] = v;
          }
        __syncthreads();
      } else {
      float fm0 = 0.f, fm1 = 0.f;   // running max of channels lane and lane + 32
      for (int a0 = 0; a0 < m; a0 += BT) {
        const int aa = a0 + tid;
        const bool live = aa < m;
        float z1[H];
        if (live) {
          const int i = sActIdx[aa];
          const float4 u = sActU[aa];
          const float4* crow = reinterpret_cast<const float4*>(a.ctab + (size_t)(o + i) * H);
#pragma unroll
          for (int c4 = 0; c4 < H / 4; ++c4) {
            const float4 cv = __ldg(crow + c4);
            const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int c = 4 * c4 + q;
              const float4 w = *reinterpret_cast<const float4*>(sW1u + 4 * c);
              z1[c] = fmaxf(fmaf(w.x, u.x, fmaf(w.y, u.y, fmaf(w.z, u.z, cc[q]))), 0.f);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < H; ++c) z1[c] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < H; ++c) {
          float acc = sB2[c];
          const float4* wr = reinterpret_cast<const float4*>(sW2 + c * H);
#pragma unroll
          for (int k4 = 0; k4 < H / 4; ++k4) {
            const float4 w = wr[k4];
            acc = fmaf(w.x, z1[4 * k4 + 0], acc);
            acc = fmaf(w.y, z1[4 * k4 + 1], acc);
            acc = fmaf(w.z, z1[4 * k4 + 2], acc);
            acc = fmaf(w.w, z1[4 * k4 + 3], acc);
          }
          const float f = live ? fmaxf(acc, 0.f) : 0.f;
          // f >= 0, so unsigned order of the bit patterns is the float order
          const float mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(f)));
          if (c < 32) {
            if (lane == c) fm0 = fmaxf(fm0, mx);
          } else {
            if (lane == c - 32) fm1 = fmaxf(fm1, mx);
          }
        }
      }
      sRed[warp * H + lane] = fm0;
      sRed[warp * H + 32 + lane] = fm1;
      __syncthreads();
      }

      if (tid < H) {
        float g0 = 0.f;
#pragma unroll
        for (int w = 0; w < BW; ++w) g0 = fmaxf(g0, sRed[w * H + tid]);
        // passive maximum: first passive node in this channel's descending order of f0
        const int16_t* ord = a.order + (size_t)H * o + (size_t)tid * n;
        for (int r = 0; r < n; ++r) {
          const int idx = ord[r];
          if (!sMask[idx]) {
            g0 = fmaxf(g0, __ldg(a.f0tab + (size_t)(o + idx) * H + tid));
            break;
          }
        }
        sG[tid] = g0;
      }
      __syncthreads();
      {
        // global MLP and the decoder's global half, 4 partial sums per output on 256 threads
        const int u = tid & (H - 1), part = tid >> 6;
        float acc = 0.f;
        const float* wr = W + OFF_WG + u * H + part * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(__ldg(wr + k), sG[part * 16 + k], acc);
        sRed[part * H + u] = acc;
        __syncthreads();
        if (tid < H) {
          const float gsum = W[OFF_BG + tid] + sRed[tid] + sRed[H + tid] + sRed[2 * H + tid] +
                             sRed[3 * H + tid];
          sG[tid] = fmaxf(gsum, 0.f);
        }
        __syncthreads();
        acc = 0.f;
        const float* wd = W + OFF_WD + u * 2 * H + H + part * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(__ldg(wd + k), sG[part * 16 + k], acc);
        sRed[part * H + u] = acc;
        __syncthreads();
        if (tid < H) sBeta[tid] = sRed[tid] + sRed[H + tid] + sRed[2 * H + tid] + sRed[3 * H + tid];
        __syncthreads();
      }
    }

    if constexpr (kBF16) {
      // decoder record: ReLU(h0 + beta) = max(h0, -beta) + beta, so the GEMM epilogue needs
      // -beta (BF16) and the constant D2 beta + b_D2 of this pad
      if (a.mode != MODE_LINEAR_ONLY && tid < H)
        reinterpret_cast<__nv_bfloat16*>(a.negbeta)[(size_t)pad * H + tid] =
            __float2bfloat16_rn(-sBeta[tid]);
      if (warp < 3) {
        float acc = 0.f;
        if (a.mode != MODE_LINEAR_ONLY)
          acc = fmaf(sW4[warp * H + lane], sBeta[lane], sW4[warp * H + 32 + lane] * sBeta[32 + lane]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == 0) sRed[warp] = a.mode != MODE_LINEAR_ONLY ? acc + sB4[warp] : 0.f;
      }
      __syncthreads();
      if (tid == 0) a.c0m[pad] = make_float4(sRed[0], sRed[1], sRed[2], __int_as_float(m));
      continue;
    }

    // ---- 3. passive nodes: Eq. 4
    const float* Om = a.omega + a.omega_off[ty];
    for (int i = tid; i < n; i += BT) {
      if (sMask[i]) continue;
      float l0 = 0.f, l1 = 0.f, l2 = 0.f;
      if (a.mode != MODE_RESIDUAL_ONLY) {
        const float* col = Om + i;
#pragma unroll 4
        for (int aa = 0; aa < m; ++aa) {
          const int j = sActIdx[aa];
          const float4 u = sActU[aa];
          const float w = __ldg(col + (size_t)j * n);
          l0 = fmaf(w, u.x, l0);
          l1 = fmaf(w, u.y, l1);
          l2 = fmaf(w, u.z, l2);
        }
      }
      if (a.mode != MODE_LINEAR_ONLY) {
        float r0 = sB4[0], r1 = sB4[1], r2 = sB4[2];
        const float4* hrow = reinterpret_cast<const float4*>(a.h0tab + (size_t)(o + i) * H);
#pragma unroll
        for (int c4 = 0; c4 < H / 4; ++c4) {
          const float4 hv = __ldg(hrow + c4);
          const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * c4 + q;
            const float z = fmaxf(hh[q] + sBeta[c], 0.f);
            r0 = fmaf(sW4[c], z, r0);
            r1 = fmaf(sW4[H + c], z, r1);
            r2 = fmaf(sW4[2 * H + c], z, r2);
          }
        }
        l0 += r0;
        l1 += r1;
        l2 += r2;
      }
      float* d = a.disp + 3 * (base + i);
      d[0] = l0;
      d[1] = l1;
      d[2] = l2;
    }
  }
}

size_t batched_smem_bytes(int nmax, int K) { return BatchedSmem(nmax, K).total; }
int batched_threads() { return BT; }

template <bool kBF16>
static cudaError_t configure(size_t smem) {
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(batched_forward_kernel<kBF16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  return cudaSuccess;
}

cudaError_t batched_occupancy(int nmax, int K, int* blocks_per_sm) {
  size_t smem = batched_smem_bytes(nmax, K);
  cudaError_t e = configure<false>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm,
                                                       batched_forward_kernel<false>, BT, smem);
}

cudaError_t batched_front_occupancy(int nmax, int K, int* blocks_per_sm) {
  size_t smem = batched_smem_bytes(nmax, K);
  cudaError_t e = configure<true>(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batched_forward_kernel<true>,
                                                       BT, smem);
}

cudaError_t launch_batched_forward(const BatchedArgs& a, int grid, cudaStream_t s) {
  size_t smem = batched_smem_bytes(a.nmax, a.K);
  cudaError_t e = configure<false>(smem);
  if (e != cudaSuccess) return e;
  batched_forward_kernel<false><<<grid, BT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batched_front_bf16(const BatchedArgs& a, int grid, cudaStream_t s) {
  size_t smem = batched_smem_bytes(a.nmax, a.K);
  cudaError_t e = configure<true>(smem);
  if (e != cudaSuccess) return e;
  batched_forward_kernel<true><<<grid, BT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace etac
