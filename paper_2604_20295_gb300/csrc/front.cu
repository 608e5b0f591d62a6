// front.cu -- front half of the BF16 tensor-core ETac step (ETac Sec. III-A).
//
// front_contact_kernel (persistent, one CTA per pad from a work queue, heaviest pads first):
//   1. FP32 screen of every node; nodes certainly outside all objects are passive (their B
//      operand entries are zeroed); the rest become a compact candidate list;
//   2. the candidates' exact (df32) contact decision and u_hat -- candidates are dense in the
//      list, so warps do not diverge on the long df32 chains; active nodes keep u_hat (Eq. 4
//      covers passive nodes only), their u_hat goes to the B operand, their contact bits to a
//      per-pad bit field;
//   3. the encoder on the active nodes on tensor cores (E1 evaluated straight into the
//      m16n8k16 A-fragment layout, E2 as BF16 MMAs with FP32 accumulation), channel maxima
//      per pad written out.  Passive nodes need no encoder: their outputs are table entries.
//   Four block barriers per pad.
//   4. the max-pool over the passive nodes: the first passive node of each channel's table
//      order (ranked f0 values), 32 ranks per warp-wide test.
//   Nodes certainly inside an object, with no near-tie among the discrete choices, take u_hat
//   from FP32 arithmetic (the BF16 step's error budget); the exact df32 path decides the thin
//   band near surfaces and ties, so contact sets still equal the exact ones.
// front_global_kernel (one warp per pad): global MLP g = ReLU(G1 g0), the decoder's global half
//   beta = D1[:, 64:] g, and the record the propagation GEMM's epilogue needs: -beta in BF16
//   and D2 beta + b_D2 (ReLU(h0 + beta) = max(h0, -beta) + beta).
#include <cuda_bf16.h>

#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {

namespace {

constexpr int FT = 128;
constexpr int FW = FT / 32;
constexpr int CPW = H / FW;   // channels per warp in the passive max-pool search

struct FrontSmem {
  size_t w2f, b2, w1u, red, cand, actidx, actu, actbits, cnt, po, total;
  __host__ __device__ FrontSmem(int nmax, int K) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    w2f = take(sizeof(uint2) * 8 * 4 * 32);
    b2 = take(sizeof(float) * H);
    w1u = take(sizeof(float4) * H);
    red = take(sizeof(float) * FW * H);
    cand = take(sizeof(int16_t) * (size_t)nmax);
    actidx = take(sizeof(int16_t) * (size_t)nmax);
    actu = take(sizeof(float4) * (size_t)nmax);
    actbits = take(sizeof(uint32_t) * (size_t)((nmax + 31) / 32));
    cnt = take(sizeof(int) * 8);
    po = take(sizeof(PadObj) * (size_t)K);
    total = o;
  }
};

// appends the lanes of a warp whose flag is set to a shared list; returns each lane's slot
__device__ __forceinline__ int warp_append(bool flag, int* counter) {
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  if (!bal) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  return flag ? base + __popc(bal & ((1u << lane) - 1u)) : -1;
}

// every pad's relative transforms and screening margins, one thread per pad (object slots in
// turn); pad_bad[pad] = 1 when one of its poses or sizes is not finite
__global__ void __launch_bounds__(256) pad_obj_kernel(FrontArgs a) {
  const int pad = blockIdx.x * blockDim.x + threadIdx.x;
  if (pad >= a.num_items) return;
  const int env = pad / a.P;
  const float* pp = a.pad_pose + 7 * (size_t)pad;
  const float pmax = a.type_pmax[a.pad_type[pad]];
  int bad = 0;
  for (int k = 0; k < a.K; ++k) {
    const int ob = env * a.K + k;
    const float* op = a.obj_pose + 7 * (size_t)ob;
    const float* od = a.obj_dims + 3 * (size_t)ob;
    int type = a.obj_type[ob];
    if (type < OBJ_NONE || type > OBJ_CAPSULE) type = OBJ_NONE;
    const bool ok = finite7(op) && finite7(pp) && isfinite(od[0]) && isfinite(od[1]) &&
                    isfinite(od[2]);
    if (!ok && type != OBJ_NONE) {
      bad = 1;
      type = OBJ_NONE;
    }
    PadObj po;
    setup_pad_obj(op, type, od, pp, pmax, &po);
    a.padobj[(size_t)pad * a.K + k] = po;
  }
  a.pad_bad[pad] = bad;
}

__global__ void __launch_bounds__(FT, 4) front_contact_kernel(FrontArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const FrontSmem L(a.nmax, a.K);
  uint2* sW2f = reinterpret_cast<uint2*>(smem + L.w2f);
  float* sB2 = reinterpret_cast<float*>(smem + L.b2);
  float4* sW1u = reinterpret_cast<float4*>(smem + L.w1u);
  float* sRed = reinterpret_cast<float*>(smem + L.red);
  int16_t* sCand = reinterpret_cast<int16_t*>(smem + L.cand);
  int16_t* sActIdx = reinterpret_cast<int16_t*>(smem + L.actidx);
  float4* sActU = reinterpret_cast<float4*>(smem + L.actu);
  uint32_t* sActBits = reinterpret_cast<uint32_t*>(smem + L.actbits);
  int* sCnt = reinterpret_cast<int*>(smem + L.cnt);   // [0] candidates [1] actives [2] invalid
  PadObj* spo = reinterpret_cast<PadObj*>(smem + L.po);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* W = a.params;
  // E2 as m16n8k16 B fragments: B[k = input unit][n = output unit] = W2[n][k]; entry
  // (nt, s, l) holds lane l's two registers for output tile nt and input step s
  for (int e = tid; e < 8 * 4 * 32; e += FT) {
    const int l = e & 31, s4 = (e >> 5) & 3, nt = e >> 7;
    const int n = 8 * nt + (l >> 2), k = 16 * s4 + 2 * (l & 3);
    __nv_bfloat162 lo = __floats2bfloat162_rn(W[OFF_W2 + n * H + k], W[OFF_W2 + n * H + k + 1]);
    __nv_bfloat162 hi = __floats2bfloat162_rn(W[OFF_W2 + n * H + k + 8], W[OFF_W2 + n * H + k + 9]);
    sW2f[e] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
  }
  for (int i = tid; i < H; i += FT) {
    sB2[i] = W[OFF_B2 + i];
    sW1u[i] = make_float4(W[OFF_W1 + i * NIN + 6], W[OFF_W1 + i * NIN + 7], W[OFF_W1 + i * NIN + 8],
                          0.f);
  }

  // the next work item is fetched while the current one is processed
  __shared__ int s_next;
  if (tid == 0) s_next = atomicAdd(a.ticket, 1);
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = s_next;
      sCnt[0] = sCnt[1] = sCnt[2] = 0;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= a.num_items) break;
    if (tid == 0) s_next = atomicAdd(a.ticket, 1);
    const int pad = a.item_pad[item];
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const int nwords = (n + 31) >> 5;
    const long long base = a.pad_off[pad];
    const float* tpos = a.type_pos + 3 * (size_t)o;
    const float* tnrm = a.type_nrm + 3 * (size_t)o;
    __nv_bfloat16* btrow =
        reinterpret_cast<__nv_bfloat16*>(a.bt) + a.bt_off[ty] + (size_t)3 * a.pad_inst[pad] * n;
    {
      const int* src = reinterpret_cast<const int*>(a.padobj + (size_t)pad * a.K);
      int* dst = reinterpret_cast<int*>(spo);
      const int words = a.K * (int)(sizeof(PadObj) / 4);
      for (int e = tid; e < words; e += FT) dst[e] = src[e];
      if (tid == 0 && a.pad_bad[pad]) sCnt[2] = 1;
    }
    for (int w = tid; w < nwords; w += FT) sActBits[w] = 0u;
    __syncthreads();
    const bool invalid = sCnt[2] != 0;
    float gap = 0.f;   // twice the largest FP32 error bound over the pad's objects
    for (int k = 0; k < a.K; ++k) gap = fmaxf(gap, 2.f * spo[k].tau);

    // ---- 1. FP32 screen of every node.  Nodes certainly outside stay passive; nodes certainly
    // inside with no near-tie in their discrete choices take the FP32 u_hat (BF16 accuracy is
    // the budget here); only the thin band near a surface or a tie goes to the exact df32 path.
    for (int r0 = 0; r0 < n; r0 += FT) {
      const int i = r0 + tid;
      bool cand = false;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      c.k = -1;
      c.u[0] = c.u[1] = c.u[2] = 0.f;
      if (i < n && !invalid) {
        const float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
        float phi32;
        if (contact_screen(spo, a.K, p, &phi32)) {
          const float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
          cand = !contact_fast(spo, a.K, p, nr, gap, &c);
        }
      }
      if (i < n && !cand) {
        btrow[i] = __float2bfloat16_rn(c.u[0]);
        btrow[n + i] = __float2bfloat16_rn(c.u[1]);
        btrow[2 * n + i] = __float2bfloat16_rn(c.u[2]);
        if (a.mask) a.mask[base + i] = c.active ? 1 : 0;
        if (a.pen) a.pen[base + i] = c.active ? -c.phi : 0.f;
        if (c.active) {
          float* d = a.disp + 3 * (base + i);
          d[0] = c.u[0];
          d[1] = c.u[1];
          d[2] = c.u[2];
          atomicOr(&sActBits[i >> 5], 1u << (i & 31));
        }
      }
      const int slot = warp_append(cand, &sCnt[0]);
      if (slot >= 0) sCand[slot] = (int16_t)i;
      const int aslot = warp_append(c.active, &sCnt[1]);
      if (aslot >= 0) {
        sActIdx[aslot] = (int16_t)i;
        sActU[aslot] = make_float4(c.u[0], c.u[1], c.u[2], 0.f);
      }
    }
    __syncthreads();

    // ---- 2. exact contact of the band candidates
    const int nc = sCnt[0];
    for (int s0 = 0; s0 < nc; s0 += FT) {
      const int s = s0 + tid;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      c.k = -1;
      c.u[0] = c.u[1] = c.u[2] = 0.f;
      int i = 0;
      if (s < nc) {
        i = sCand[s];
        const float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
        const float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
        c = contact_refine(spo, a.K, p, nr, 0.f);
        btrow[i] = __float2bfloat16_rn(c.u[0]);
        btrow[n + i] = __float2bfloat16_rn(c.u[1]);
        btrow[2 * n + i] = __float2bfloat16_rn(c.u[2]);
        if (a.mask) a.mask[base + i] = c.active ? 1 : 0;
        if (a.pen) a.pen[base + i] = c.active ? -c.phi : 0.f;
        if (c.active) {
          float* d = a.disp + 3 * (base + i);
          d[0] = c.u[0];
          d[1] = c.u[1];
          d[2] = c.u[2];
          atomicOr(&sActBits[i >> 5], 1u << (i & 31));
        }
      }
      const int slot = warp_append(c.active, &sCnt[1]);
      if (slot >= 0) {
        sActIdx[slot] = (int16_t)i;
        sActU[slot] = make_float4(c.u[0], c.u[1], c.u[2], 0.f);
      }
    }
    __syncthreads();
    const int m = sCnt[1];
    for (int w = tid; w < nwords; w += FT) a.maskbits[a.mask_woff[pad] + w] = sActBits[w];
    if (tid == 0) {
      if (a.count) a.count[pad] = m;
      a.pad_m[pad] = m;
      if (invalid) latch_status(a.status, STATUS_NONFINITE);
    }
    if (m == 0) {   // no contact (or invalid pose): the whole pad is at rest
      for (int i = tid; i < n; i += FT) {
        float* d = a.disp + 3 * (base + i);
        d[0] = d[1] = d[2] = 0.f;
      }
      continue;
    }
    if (a.mode == MODE_LINEAR_ONLY) continue;

    // ---- 3. encoder of the active nodes on tensor cores, channel maxima
    {
      const int grp = lane >> 2, tig = lane & 3;
      float fm[8][2];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) fm[nt][0] = fm[nt][1] = 0.f;   // ReLU outputs are >= 0
      for (int g = warp; g * 16 < m; g += FW) {
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
            const float4 w0 = sW1u[col], w1 = sW1u[col + 1];
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
          fm[nt][0] = fmaxf(fm[nt][0], fmaxf(v0 ? acc[0] : 0.f, v1 ? acc[2] : 0.f));
          fm[nt][1] = fmaxf(fm[nt][1], fmaxf(v0 ? acc[1] : 0.f, v1 ? acc[3] : 0.f));
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
    }
    __syncthreads();
    // max-pool over the passive nodes: the first passive node in each channel's descending
    // order of f0; a warp tests 32 ranks per load for 8 channels at a time
    {
      float best[CPW];
      bool done[CPW];
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        best[c] = 0.f;
        done[c] = false;
      }
      for (int r0 = 0; r0 < n; r0 += 32) {
        const int r = r0 + lane;
        float2 e[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const int u = warp * CPW + c;
          e[c] = (!done[c] && r < n) ? __ldg(a.ranked + (size_t)H * o + (size_t)u * n + r)
                                      : make_float2(0.f, __int_as_float(0));
        }
        bool all = true;
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const int idx = __float_as_int(e[c].y);
          const bool passive = !done[c] && r < n && !((sActBits[idx >> 5] >> (idx & 31)) & 1u);
          const unsigned bal = __ballot_sync(0xffffffffu, passive);
          if (bal) {
            best[c] = __shfl_sync(0xffffffffu, e[c].x, __ffs(bal) - 1);
            done[c] = true;
          }
          all &= done[c];
        }
        if (all) break;
      }
      if (lane < CPW) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == lane) v = best[c];
        const int u = warp * CPW + lane;
#pragma unroll
        for (int w = 0; w < FW; ++w) v = fmaxf(v, sRed[w * H + u]);
        a.g0a[(size_t)pad * H + u] = v;
      }
    }
  }
}

// one warp per pad; G1 and D1's global half staged transposed so lanes read consecutive units
__global__ void __launch_bounds__(256) front_global_kernel(FrontArgs a) {
  __shared__ float sWgT[H * H];   // [k][u] = G1[u][k]
  __shared__ float sWdT[H * H];   // [k][u] = D1[u][64 + k]
  __shared__ float sBg[H];
  __shared__ float sW4[3 * H];
  __shared__ float sB4[4];
  const float* W = a.params;
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
    const int u = e >> 6, k = e & (H - 1);
    sWgT[k * H + u] = W[OFF_WG + u * H + k];
    sWdT[k * H + u] = W[OFF_WD + u * 2 * H + H + k];
  }
  for (int e = threadIdx.x; e < H; e += blockDim.x) sBg[e] = W[OFF_BG + e];
  for (int e = threadIdx.x; e < 3 * H; e += blockDim.x) sW4[e] = W[OFF_W4 + e];
  if (threadIdx.x < 3) sB4[threadIdx.x] = W[OFF_B4 + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int np = a.num_items;
  for (int pad = blockIdx.x * wpb + (threadIdx.x >> 5); pad < np; pad += gridDim.x * wpb) {
    const int m = a.pad_m[pad];
    if (m == 0 || a.mode == MODE_LINEAR_ONLY) {
      if (lane == 0) a.c0m[pad] = make_float4(0.f, 0.f, 0.f, __int_as_float(m));
      continue;
    }
    float g0[2];
    g0[0] = a.g0a[(size_t)pad * H + lane];
    g0[1] = a.g0a[(size_t)pad * H + 32 + lane];
    float g[2], beta[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = lane + 32 * h;
      float acc = sBg[u];
#pragma unroll
      for (int k = 0; k < 32; ++k) acc = fmaf(sWgT[k * H + u], __shfl_sync(0xffffffffu, g0[0], k), acc);
#pragma unroll
      for (int k = 0; k < 32; ++k)
        acc = fmaf(sWgT[(32 + k) * H + u], __shfl_sync(0xffffffffu, g0[1], k), acc);
      g[h] = fmaxf(acc, 0.f);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = lane + 32 * h;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 32; ++k) acc = fmaf(sWdT[k * H + u], __shfl_sync(0xffffffffu, g[0], k), acc);
#pragma unroll
      for (int k = 0; k < 32; ++k)
        acc = fmaf(sWdT[(32 + k) * H + u], __shfl_sync(0xffffffffu, g[1], k), acc);
      beta[h] = acc;
      reinterpret_cast<__nv_bfloat16*>(a.negbeta)[(size_t)pad * H + u] = __float2bfloat16_rn(-acc);
    }
    float c0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v = fmaf(sW4[q * H + lane], beta[0], sW4[q * H + 32 + lane] * beta[1]);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      c0[q] = v + sB4[q];
    }
    if (lane == 0) a.c0m[pad] = make_float4(c0[0], c0[1], c0[2], __int_as_float(m));
  }
}

}  // namespace

size_t front_smem_bytes(int nmax, int K) { return FrontSmem(nmax, K).total; }

cudaError_t front_occupancy(int nmax, int K, int* blocks_per_sm) {
  const size_t smem = front_smem_bytes(nmax, K);
  cudaError_t e = cudaFuncSetAttribute(front_contact_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, front_contact_kernel, FT,
                                                       smem);
}

cudaError_t launch_front_contact(const FrontArgs& a, int grid, cudaStream_t s) {
  const size_t smem = front_smem_bytes(a.nmax, a.K);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(front_contact_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  front_contact_kernel<<<grid, FT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pad_obj(const FrontArgs& a, cudaStream_t s) {
  pad_obj_kernel<<<(unsigned)((a.num_items + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_front_global(const FrontArgs& a, int grid, cudaStream_t s) {
  front_global_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace etac
