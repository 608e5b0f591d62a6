// bwd_batched.cu -- FP32 reverse mode of the batched ETac step as a staged pipeline (ETac
// Sec. III-A, Eq. 1, Eq. 4; the calibration of Eq. 5 differentiates the same quantities).
//
// Passive nodes feed the network constant inputs [p, n, 0], so their encoder activations are
// per pad type, and the reverse of the encoder for the decoder path can be summed over all
// instances of a type before it is run: once per type node instead of once per pad node.
// The stages:
//   R1 bwd_pad_kernel (warp per pad): contact (same decisions as the forward), u_hat and phi
//      of the active nodes, dL/du_hat's direct term, the passive upstream gradient G as the
//      split BF16 B operand of the propagation reverse, sum G over passive nodes, and the
//      channel maxima of f with their lowest-index argmax, either recorded by the forward
//      (FP32 batched models) or recomputed: the active nodes' encoder to FP32 accuracy on
//      tensor cores (inputs, activations and weights split into three BF16 parts), the
//      passive candidate from the ranked f0 table;
//   R2 bwd_global_kernel (64 pads per CTA, register-tiled): ag = G1 g0 + b, g = ReLU(ag),
//      beta = D1_g g;
//   R3 bwd_decoder_kernel (type x 64-instance groups): for every passive (instance k, node
//      i), dz = D2^T G_ki and dA3 = dz [h0_i + beta_k > 0]; sums S_k = sum_i dA3 (per pad,
//      complete), A3_i = sum_k dA3 (per type node, partial per group) and
//      dD2 = sum G (x) ReLU(h0 + beta);
//   R3b reduce the A3 partials in group order;
//   R4a bwd_padmlp_kernel (64 pads per CTA, register-tiled): S from the node-range partials,
//      dg = D1_g^T S, dag = dg [ag > 0], dA2 = (G1^T dag) [g0 > 0] at each channel's argmax;
//   R4 bwd_padrev_kernel (warp per pad): the E1 reverse of the distinct argmax nodes (E1, b1,
//      and for an active node dL/du_hat);
//   R4b sums over 64-pad chunks of S g^T, dag g0^T, S, dag (D1_g, G1 and their biases) and
//      of dA2 h1^T, dA2 (E2 and b2);
//   R5 bwd_typenode_kernel (64 type nodes per CTA): the decoder path's encoder reverse from
//      A3 (dD1_f, dE2, dE1, biases);
//   R6 the propagation reverse on tensor cores (prop_gemm.cu, backward modes);
//   R7 bwd_fill_kernel (streaming): outputs dL/du_hat and the passive dL/dpen;
//      bwd_pose_kernel (warp per pad, the pad's active nodes compacted into a queue so every
//      lane takes one): the active dL/dpen and the pose partials.
// Every sum runs in a fixed order (static work assignment, partials reduced in index order),
// so the result is bitwise repeatable.
#include <cuda_bf16.h>

#include "bwd_common.cuh"
#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RT = 256;            // threads per CTA of the warp-per-pad kernels
constexpr int RW = RT / 32;
constexpr int RPEND = 48;          // active rows awaiting the encoder (<= 15 + 32)
constexpr int RCAND = 64;          // undecided nodes awaiting the exact contact path

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bfr(float x) {   // x - BF16(x)
  return x - __bfloat162float(__float2bfloat16_rn(x));
}
// Three-part split of an FP32 value into BF16 parts x = x0 + x1 + x2 + r with |r| <= 2^-24 |x|
// (each part holds the next 8 significant bits of the remainder), applied to a pair.
__device__ __forceinline__ void split3(float a, float b, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const float a1 = bfr(a), b1 = bfr(b);
  p0 = bf2(a, b);
  p1 = bf2(a1, b1);
  p2 = bf2(bfr(a1), bfr(b1));
}

// ----------------------------------------------------------------------------- R1
struct R1Smem {
  size_t w1f, w2f, b2, warp0, warp_bytes, po, bits, pend, pnode, cand, fmv, fmi, total;
  __host__ __device__ R1Smem(int nmax, int K) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    w1f = take(sizeof(uint2) * 3 * 2 * 8 * 32);   // [part][k step][n tile][lane]
    w2f = take(sizeof(uint2) * 3 * 8 * 4 * 32);   // [part][n tile][k step][lane]
    b2 = take(sizeof(float) * H);
    warp0 = o;
    o = 0;
    po = take(sizeof(PadObj) * (size_t)K);
    bits = take(sizeof(uint32_t) * (size_t)((nmax + 31) / 32));
    pend = take(64 * RPEND);                      // E1 input rows: 32 BF16 each
    pnode = take(sizeof(int) * RPEND);
    cand = take(sizeof(int16_t) * RCAND);
    fmv = take(sizeof(float) * H);
    fmi = take(sizeof(int) * H);
    warp_bytes = o;
    total = warp0 + RW * warp_bytes;
  }
};

// E1 input row of an active node, 32 BF16: the three-part splits [x0, x1, x2] of x = [p, n,
// u_hat] (9 values each), then 1 (the bias column), then zeros.
__device__ __forceinline__ void pack_row32(uint4* dst, float3 p, float3 nr, const float* u) {
  const float x[9] = {p.x, p.y, p.z, nr.x, nr.y, nr.z, u[0], u[1], u[2]};
  float v[32];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float r1 = bfr(x[k]);
    v[k] = x[k];
    v[9 + k] = r1;
    v[18 + k] = bfr(r1);
  }
  v[27] = 1.f;
#pragma unroll
  for (int k = 28; k < 32; ++k) v[k] = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    dst[q] = make_uint4(bf2(v[8 * q], v[8 * q + 1]), bf2(v[8 * q + 2], v[8 * q + 3]),
                        bf2(v[8 * q + 4], v[8 * q + 5]), bf2(v[8 * q + 6], v[8 * q + 7]));
}

// W1 column read by E1 input k of the 32-wide row (-1: bias, -2: zero)
__device__ __forceinline__ int w1_col(int k) {
  if (k < 27) return k % 9;
  return k == 27 ? -1 : -2;
}

// Encoder of up to 16 active rows to FP32 accuracy on BF16 tensor cores.  Every operand is
// split into three BF16 parts (x = x0 + x1 + x2 to 2^-24): E1 multiplies the row of input
// parts by the three parts of W1 (all nine products, accumulated in FP32); E2 splits
// h1 = ReLU(E1) and W2 the same way and keeps the six products whose parts sum to at most the
// third (the three dropped ones are below 2^-24 of the result).  Then f = ReLU(E2 h1 + b2) is
// folded into the per-lane running maxima with their node (lowest index wins ties).
__device__ __forceinline__ void bwd_encode(float (&fv)[8][2], int (&fi)[8][2], uint32_t rows,
                                           const int* node, int cnt, const uint2* sW1f,
                                           const uint2* sW2f, const float* sB2, int lane) {
  const int grp = lane >> 2, tig = lane & 3;
  const bool v0 = grp < cnt, v1 = grp + 8 < cnt;
  const int n0 = v0 ? node[grp] : 0x7fffffff, n1 = v1 ? node[grp + 8] : 0x7fffffff;
  uint32_t ax[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
    sm100::ldmatrix_x4(rows + (uint32_t)((lane & 15) * 64 + (lane >> 4) * 16 + ks * 32), ax[ks][0],
                       ax[ks][1], ax[ks][2], ax[ks][3]);
  // E2's k step s4 reads h columns 16 s4 .. 16 s4 + 15, which E1's n tiles 2 s4 and 2 s4 + 1
  // produce: E1 runs one k step ahead of E2, so only that step's split parts are live.  The
  // eight E2 n tiles are independent MMA chains, interleaved; each keeps its order (k steps
  // ascending, smallest products first).
  float acc2[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc2[nt][q] = 0.f;
#pragma unroll 1
  for (int s4 = 0; s4 < 4; ++s4) {   // rolled: a quarter of the code, for the instruction cache
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int part = 0; part < 3; ++part)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const uint2 bb = sW1f[((part * 2 + ks) * 8 + 2 * s4 + t) * 32 + lane];
          sm100::mma_bf16_16816(acc[t], ax[ks], bb.x, bb.y, acc[t]);
        }
    uint32_t ah[3][4];
    split3(relu(acc[0][0]), relu(acc[0][1]), ah[0][0], ah[1][0], ah[2][0]);
    split3(relu(acc[0][2]), relu(acc[0][3]), ah[0][1], ah[1][1], ah[2][1]);
    split3(relu(acc[1][0]), relu(acc[1][1]), ah[0][2], ah[1][2], ah[2][2]);
    split3(relu(acc[1][2]), relu(acc[1][3]), ah[0][3], ah[1][3], ah[2][3]);
#pragma unroll
    for (int pr = 0; pr < 6; ++pr) {
      // products (A part, W part): (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
      const int ap = pr == 0 ? 2 : (pr == 1 || pr == 3 ? 1 : 0);
      const int wp = pr == 2 ? 2 : (pr == 1 || pr == 4 ? 1 : 0);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const uint2 bw = sW2f[((wp * 8 + nt) * 4 + s4) * 32 + lane];
        sm100::mma_bf16_16816(acc2[nt], ah[ap], bw.x, bw.y, acc2[nt]);
      }
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float b = sB2[8 * nt + 2 * tig + e];
      const float f0 = relu(acc2[nt][e] + b), f1 = relu(acc2[nt][2 + e] + b);
      if (v0 && (f0 > fv[nt][e] || (f0 == fv[nt][e] && n0 < fi[nt][e]))) {
        fv[nt][e] = f0;
        fi[nt][e] = n0;
      }
      if (v1 && (f1 > fv[nt][e] || (f1 == fv[nt][e] && n1 < fi[nt][e]))) {
        fv[nt][e] = f1;
        fi[nt][e] = n1;
      }
    }
  }
}

// MESH: the context has mesh objects (the mesh queries are compiled in)
template <bool MESH>
__global__ void __launch_bounds__(RT, 2) bwd_pad_kernel(BwdBatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const R1Smem L(a.nmax, a.K);
  uint2* sW1f = reinterpret_cast<uint2*>(smem + L.w1f);
  uint2* sW2f = reinterpret_cast<uint2*>(smem + L.w2f);
  float* sB2 = reinterpret_cast<float*>(smem + L.b2);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* W = a.params;
  // the part `part` (0..2) of the three-part BF16 split of w
  auto wpart = [](float w, int part) {
    float r = w;
    for (int q = 0; q < part; ++q) r = bfr(r);
    return __float2bfloat16_rn(r);
  };
  for (int e = tid; e < 3 * 2 * 8 * 32; e += RT) {
    const int l = e & 31, nt = (e >> 5) & 7, ks = (e >> 8) & 1, part = e >> 9;
    const int n = 8 * nt + (l >> 2), k0 = 16 * ks + 2 * (l & 3);
    auto wv = [&](int k) {
      const int col = w1_col(k);
      const float w = col == -1 ? W[OFF_B1 + n] : (col == -2 ? 0.f : W[OFF_W1 + n * NIN + col]);
      return wpart(w, part);
    };
    __nv_bfloat162 lo = __halves2bfloat162(wv(k0), wv(k0 + 1));
    __nv_bfloat162 hi = __halves2bfloat162(wv(k0 + 8), wv(k0 + 9));
    sW1f[e] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
  }
  for (int e = tid; e < 3 * 8 * 4 * 32; e += RT) {
    const int l = e & 31, s4 = (e >> 5) & 3, nt = (e >> 7) & 7, part = e >> 10;
    const int n = 8 * nt + (l >> 2), k = 16 * s4 + 2 * (l & 3);
    __nv_bfloat162 lo = __halves2bfloat162(wpart(W[OFF_W2 + n * H + k], part),
                                           wpart(W[OFF_W2 + n * H + k + 1], part));
    __nv_bfloat162 hi = __halves2bfloat162(wpart(W[OFF_W2 + n * H + k + 8], part),
                                           wpart(W[OFF_W2 + n * H + k + 9], part));
    sW2f[e] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
  }
  for (int i = tid; i < H; i += RT) sB2[i] = W[OFF_B2 + i];
  __syncthreads();

  unsigned char* wb = smem + L.warp0 + (size_t)warp * L.warp_bytes;
  PadObj* spo = reinterpret_cast<PadObj*>(wb + L.po);
  uint32_t* sBits = reinterpret_cast<uint32_t*>(wb + L.bits);
  uint4* sPend = reinterpret_cast<uint4*>(wb + L.pend);
  const uint32_t sPend_addr = (uint32_t)__cvta_generic_to_shared(sPend);
  int* sPNode = reinterpret_cast<int*>(wb + L.pnode);
  int16_t* sCand = reinterpret_cast<int16_t*>(wb + L.cand);
  float* sFv = reinterpret_cast<float*>(wb + L.fmv);
  int* sFi = reinterpret_cast<int*>(wb + L.fmi);
  const unsigned lt = (1u << lane) - 1u;
  const bool use_l = uses_propagation(a.mode);
  // the max-pool state: recorded by the forward (FP32 batched models), else recomputed here
  const bool rec = a.g0rec != nullptr;
  const bool use_r = uses_residual(a.mode) && !rec;

  int next = 0;
  if (lane == 0) next = atomicAdd(a.ticket, 1);
  for (;;) {
    __syncwarp();
    const int item = __shfl_sync(FULL, next, 0);
    if (item >= a.num_items) break;
    if (lane == 0) next = atomicAdd(a.ticket, 1);
    const int pad = a.item_pad[item];
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const int nwords = (n + 31) >> 5;
    const long long base = a.pad_off[pad];
    const float* tpos = a.type_pos + 3 * (size_t)o;
    const float* tnrm = a.type_nrm + 3 * (size_t)o;
    const float* G = a.grad_disp + 3 * base;
    const size_t brow = (size_t)a.bg_off[ty] + (size_t)3 * a.pad_inst[pad] * n;
    __nv_bfloat16* bgh = reinterpret_cast<__nv_bfloat16*>(a.bg_hi) + brow;
    __nv_bfloat16* bgl = reinterpret_cast<__nv_bfloat16*>(a.bg_lo) + brow;
    {
      const int* src = reinterpret_cast<const int*>(a.padobj + (size_t)pad * a.K);
      int* dst = reinterpret_cast<int*>(spo);
      const int words = a.K * (int)(sizeof(PadObj) / 4);
      for (int e = lane; e < words; e += 32) dst[e] = src[e];
    }
    const bool invalid = a.pad_bad[pad] != 0;
    __syncwarp();
    float gap = 0.f;
    for (int k = 0; k < a.K; ++k) gap = fmaxf(gap, 2.f * spo[k].tau);

    float fv[8][2];
    int fi[8][2];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        fv[nt][e] = -1.f;   // features are >= 0
        fi[nt][e] = 0x7fffffff;
      }
    float gs0 = 0.f, gs1 = 0.f, gs2 = 0.f;   // sum of G over this lane's passive nodes
    int npend = 0, ncand = 0, m = 0;         // warp-uniform

    // a decided node: its workspace entries, the B operand of the propagation reverse, and
    // (active) a row for the encoder
    auto decided = [&](int i, const NodeContact& c, float3 p, float3 nr, bool push) {
      const float g0 = G[3 * i], g1 = G[3 * i + 1], g2 = G[3 * i + 2];
      if (c.active) {
        a.ws_u[base + i] = make_float4(c.u[0], c.u[1], c.u[2], c.phi);
        a.ws_du[base + i] = make_float4(g0, g1, g2, 0.f);   // U_i = u_hat_i: direct term
      } else {
        gs0 += g0;
        gs1 += g1;
        gs2 += g2;
      }
      if (use_l) {
        const float q0 = c.active ? 0.f : g0, q1 = c.active ? 0.f : g1, q2 = c.active ? 0.f : g2;
        bgh[i] = __float2bfloat16_rn(q0);
        bgh[n + i] = __float2bfloat16_rn(q1);
        bgh[2 * n + i] = __float2bfloat16_rn(q2);
        bgl[i] = __float2bfloat16_rn(bfr(q0));
        bgl[n + i] = __float2bfloat16_rn(bfr(q1));
        bgl[2 * n + i] = __float2bfloat16_rn(bfr(q2));
      }
      (void)push;
    };
    auto refine_batch = [&]() {
      const int cnt = min(32, ncand);
      const bool has = lane < cnt;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      c.k = -1;
      c.u[0] = c.u[1] = c.u[2] = 0.f;
      int i = 0;
      float3 p = make_float3(0.f, 0.f, 0.f), nr = p;
      if (has) {
        i = sCand[ncand - cnt + lane];
        p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
        nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
        c = contact_refine<MESH>(spo, a.K, p, nr, 0.f);
        decided(i, c, p, nr, true);
        if (c.active) atomicOr(&sBits[i >> 5], 1u << (i & 31));
      }
      ncand -= cnt;
      const unsigned b = __ballot_sync(FULL, c.active);
      if (c.active && use_r) {
        const int q = npend + __popc(b & lt);
        sPNode[q] = i;
        pack_row32(sPend + 4 * q, p, nr, c.u);
      }
      m += __popc(b);
      if (use_r) npend += __popc(b);
      __syncwarp();
    };
    auto drain = [&](int keep) {
      while (npend > keep) {
        const int cnt = min(16, npend);
        bwd_encode(fv, fi, sPend_addr + 64u * (uint32_t)(npend - cnt), sPNode + npend - cnt, cnt,
                   sW1f, sW2f, sB2, lane);
        npend -= cnt;
      }
      __syncwarp();
    };

    // One step per iteration: a 32-node row (classification) or a batch of undecided nodes (the
    // exact path), then encoder tiles.  The encoder has this one call site, so its code exists
    // once (the instruction cache is the kernel's first stall); the order of rows, batches and
    // tiles is that of classifying every row with a batch whenever the queue nears full.
    int r0 = 0;
    bool force = false;   // warp-uniform: the candidate queue is nearly full
    for (;;) {
      if (force || (r0 >= n && ncand > 0)) {
        refine_batch();
        force = false;
      } else if (r0 < n) {
        const int i = r0 + lane;
        int cls = CONTACT_OUT;
        NodeContact c;
        c.active = false;
        c.phi = 0.f;
        c.k = -1;
        c.u[0] = c.u[1] = c.u[2] = 0.f;
        float3 p = make_float3(0.f, 0.f, 0.f), nr = p;
        if (i < n && !invalid) {
          p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
          nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
          if (a.mask_in) {   // mode B: the forward's caller-supplied contact (never in the band)
            c = contact_given(a.mask_in, a.uhat_in, base + i);
            cls = c.active ? CONTACT_FAST : CONTACT_OUT;
          } else {
            cls = contact_classify<MESH>(spo, a.K, p, nr, gap, &c);
          }
        }
        if (i < n && cls != CONTACT_BAND) decided(i, c, p, nr, false);
        const unsigned bA = __ballot_sync(FULL, cls == CONTACT_FAST);
        const unsigned bC = __ballot_sync(FULL, cls == CONTACT_BAND);
        if (lane == 0) sBits[r0 >> 5] = bA;
        if (cls == CONTACT_FAST && use_r) {
          const int q = npend + __popc(bA & lt);
          sPNode[q] = i;
          pack_row32(sPend + 4 * q, p, nr, c.u);
        }
        if (cls == CONTACT_BAND) sCand[ncand + __popc(bC & lt)] = (int16_t)i;
        m += __popc(bA);
        if (use_r) npend += __popc(bA);
        ncand += __popc(bC);
        __syncwarp();
        r0 += 32;
        force = ncand > RCAND - 32;
      }
      const bool last = r0 >= n && ncand == 0;
      drain(last ? 0 : 15);
      if (last) break;
    }

    const int gi = a.pad_gi[pad];
    for (int w = lane; w < nwords; w += 32) a.maskbits[a.mask_woff[pad] + w] = sBits[w];
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      gs0 += __shfl_xor_sync(FULL, gs0, sh);
      gs1 += __shfl_xor_sync(FULL, gs1, sh);
      gs2 += __shfl_xor_sync(FULL, gs2, sh);
    }
    float* pr = a.pr + (size_t)pad * PR_STRIDE;
    if (lane == 0) {
      a.pad_m[pad] = m;
      a.inst_m[gi] = m;
      // dL/db_D2 sums G over passive nodes of pads with contact (no decoder in LINEAR_ONLY)
      const bool dec = m > 0 && uses_residual(a.mode);
      pr[PR_GSUM + 0] = dec ? gs0 : 0.f;
      pr[PR_GSUM + 1] = dec ? gs1 : 0.f;
      pr[PR_GSUM + 2] = dec ? gs2 : 0.f;
    }
    if (m > 0 && rec && uses_residual(a.mode)) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        pr[PR_G0 + c] = a.g0rec[(size_t)pad * H + c];
        reinterpret_cast<int*>(pr)[PR_ROUTE + c] = a.g0arg[(size_t)pad * H + c];
      }
    }
    if (m == 0 || !use_r) continue;

    // channel maxima of the active nodes: reduce (value, node) over the row groups
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float v = fv[nt][e];
        int id = fi[nt][e];
#pragma unroll
        for (int sh = 4; sh < 32; sh <<= 1) {
          const float ov = __shfl_xor_sync(FULL, v, sh);
          const int oi = __shfl_xor_sync(FULL, id, sh);
          if (ov > v || (ov == v && oi < id)) {
            v = ov;
            id = oi;
          }
        }
        if (lane < 4) {
          sFv[8 * nt + 2 * lane + e] = v;
          sFi[8 * nt + 2 * lane + e] = id;
        }
      }
    __syncwarp();
    // passive candidate of each channel: the first passive node of the ranked f0 order
    // (equal values are ranked by node index); lane l walks channels l and l + 32, and the
    // channels still open go warp-wide, 32 ranks per test
    const float2* rk = a.ranked + (size_t)H * o;
    float pv[2] = {-1.f, -1.f};
    int pi[2] = {0x7fffffff, 0x7fffffff};
    bool done[2] = {false, false};
    {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2* row = rk + (size_t)(lane + 32 * h) * n;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (done[h] || j >= n) continue;
          const float2 e = __ldg(row + j);
          const int idx = __float_as_int(e.y);
          if (!((sBits[idx >> 5] >> (idx & 31)) & 1u)) {
            pv[h] = e.x;
            pi[h] = idx;
            done[h] = true;
          }
        }
        if (n <= 4) done[h] = true;
      }
    }
    unsigned long long open = (unsigned long long)__ballot_sync(FULL, !done[0]) |
                              ((unsigned long long)__ballot_sync(FULL, !done[1]) << 32);
    while (open) {   // warp-uniform: one open channel at a time, 32 ranks per test
      const int ch = __ffsll((long long)open) - 1;
      open &= open - 1;
      float bv = -1.f;
      int bi = 0x7fffffff;
      for (int q0 = 4; q0 < n; q0 += 32) {
        const int r = q0 + lane;
        float2 e = make_float2(0.f, __int_as_float(0));
        bool passive = false;
        if (r < n) {
          e = __ldg(rk + (size_t)ch * n + r);
          const int idx = __float_as_int(e.y);
          passive = !((sBits[idx >> 5] >> (idx & 31)) & 1u);
        }
        const unsigned bal = __ballot_sync(FULL, passive);
        if (bal) {
          const int src = __ffs(bal) - 1;
          bv = __shfl_sync(FULL, e.x, src);
          bi = __float_as_int(__shfl_sync(FULL, e.y, src));
          break;
        }
      }
      if (ch == lane) {
        pv[0] = bv;
        pi[0] = bi;
      }
      if (ch == lane + 32) {
        pv[1] = bv;
        pi[1] = bi;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      float v = sFv[c];
      int id = sFi[c];
      if (pv[h] > v || (pv[h] == v && pi[h] < id)) {
        v = pv[h];
        id = pi[h];
      }
      pr[PR_G0 + c] = v;
      reinterpret_cast<int*>(pr)[PR_ROUTE + c] = id;
    }
  }
}

// ----------------------------------------------------------------------------- R2
// 64 pads per CTA, two register-tiled products: ag = G0 G1^T + b_G1, g = ReLU(ag),
// beta = g D1_g^T (FP32; the decoder's bias rides in the h0 table); thread (ti, tj) holds pads
// 4 ti .. + 3 x units 4 tj .. + 3
constexpr int R2_PADS = 64;

__global__ void __launch_bounds__(256) bwd_global_kernel(BwdBatchedArgs a) {
  __shared__ __align__(16) float sW[H * TLD];   // [k][c] = G1[c][k], then D1[c][64 + k]
  __shared__ __align__(16) float sX[H * TLD];   // [k][pad]: g0, then g
  const float* W = a.params;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const int p0 = blockIdx.x * R2_PADS;
  for (int e = tid; e < H * H; e += 256) {
    const int c = e >> 6, k = e & (H - 1);
    sW[k * TLD + c] = W[OFF_WG + c * H + k];
  }
  for (int e = tid; e < R2_PADS * H; e += 256) {
    const int r = e >> 6, k = e & (H - 1), pad = p0 + r;
    sX[k * TLD + r] = pad < a.num_items ? a.pr[(size_t)pad * PR_STRIDE + PR_G0 + k] : 0.f;
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = W[OFF_BG + 4 * tj + j];
  tile_acc(sX, sW, ti, tj, acc);
  __syncthreads();   // g0 and G1 are read; g and D1's global half take their places
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pad = p0 + 4 * ti + i;
    const bool live = pad < a.num_items && a.pad_m[pad] > 0;
    float* pr = a.pr + (size_t)(live ? pad : 0) * PR_STRIDE;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * tj + j;
      const float g = relu(acc[i][j]);
      sX[c * TLD + 4 * ti + i] = g;
      if (live) {
        pr[PR_AG + c] = acc[i][j];
        pr[PR_G + c] = g;
      }
    }
  }
  for (int e = tid; e < H * H; e += 256) {
    const int c = e >> 6, k = e & (H - 1);
    sW[k * TLD + c] = W[OFF_WD + c * 2 * H + H + k];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sX, sW, ti, tj, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pad = p0 + 4 * ti + i;
    if (pad >= a.num_items || a.pad_m[pad] == 0) continue;
    float* pr = a.pr + (size_t)pad * PR_STRIDE;
#pragma unroll
    for (int j = 0; j < 4; ++j) pr[PR_BETA + 4 * tj + j] = acc[i][j];
  }
}

// ----------------------------------------------------------------------------- R3
// CTA = (pad type, 64 instances, a range of up to 256 nodes); warp w takes instances
// 8 w .. 8 w + 7; the CTA walks its nodes 16 at a time, node-outer / instance-inner, so the
// running A3 of a node is two registers per lane; lane l owns channels 2 l and 2 l + 1.  S is
// partial per node range (summed in range order by the global-MLP reverse).
constexpr int R3_INST = 64;
constexpr int R3_IPW = R3_INST / 8;
constexpr int R3_NODES = 16;

struct R3Smem {
  float2 A3[8][R3_NODES][32];            // per-warp A3 of the current node chunk
  float D2[8][3][H];                     // per-warp dD2 partials
  float H0[2][R3_NODES][H];              // h0 rows of the chunk (double buffer)
  float4 G[2][8][R3_IPW][R3_NODES];      // per-warp dL/dU of the chunk, (x, y, z, -)
};

__global__ void __launch_bounds__(256, 2) bwd_decoder_kernel(BwdBatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_r3[];
  R3Smem& sm = *reinterpret_cast<R3Smem*>(smem_r3);
  auto& sA3 = sm.A3;
  auto& sD2 = sm.D2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const R3Group grp = a.r3_groups[blockIdx.x];
  const int t = grp.type;
  const int o = a.type_off[t], n = a.type_off[t + 1] - o;
  const int ninst = a.inst_off[t + 1] - a.inst_off[t];
  const int nw = (n + 31) >> 5;
  const float* W = a.params;
  const float2 w4a = make_float2(W[OFF_W4 + 2 * lane], W[OFF_W4 + 2 * lane + 1]);
  const float2 w4b = make_float2(W[OFF_W4 + H + 2 * lane], W[OFF_W4 + H + 2 * lane + 1]);
  const float2 w4c = make_float2(W[OFF_W4 + 2 * H + 2 * lane], W[OFF_W4 + 2 * H + 2 * lane + 1]);
  // this warp's instances: beta, running S, node base and contact-word offset
  float2 beta[R3_IPW], S[R3_IPW];
  int gofs[R3_IPW], mofs[R3_IPW];   // 3 x node base, contact-word offset (both < 2^31)
  unsigned live = 0u;
#pragma unroll
  for (int x = 0; x < R3_IPW; ++x) {
    const int k = grp.k0 + R3_IPW * warp + x;
    const bool in = k < ninst;
    const int gi = a.inst_off[t] + (in ? k : 0);
    const bool lv = in && a.inst_m[gi] > 0;
    const float* pr = a.pr + (size_t)a.inst_pad[gi] * PR_STRIDE;
    beta[x] = lv ? make_float2(pr[PR_BETA + 2 * lane], pr[PR_BETA + 2 * lane + 1]) : make_float2(0.f, 0.f);
    S[x] = make_float2(0.f, 0.f);
    gofs[x] = (int)(3 * a.inst_base[gi]);
    mofs[x] = (int)(a.type_woff[t] + (long long)(in ? k : 0) * nw);
    live |= lv ? 1u << x : 0u;
  }
  // stage chunk i0 into buffer b with cp.async: h0 rows (whole CTA, 16-byte copies) and this
  // warp's dL/dU rows of its live instances (4-byte copies into (x, y, z, -) slots)
  auto stage = [&](int i0, int b) {
    const int cn = min(R3_NODES, grp.i1 - i0);
    const float* h0src = a.h0tab + (size_t)(o + i0) * H;
    for (int e = threadIdx.x; e < cn * (H / 4); e += blockDim.x)
      sm100::cp_async16((uint32_t)__cvta_generic_to_shared(&sm.H0[b][0][0]) + 16 * e, h0src + 4 * e, 16);
#pragma unroll
    for (int x = 0; x < R3_IPW; ++x) {
      if (!((live >> x) & 1u)) continue;
      const float* g = a.grad_disp + gofs[x] + 3 * i0;
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sm.G[b][warp][x][0]);
      for (int e = lane; e < 3 * cn; e += 32) {
        const int r = e / 3, q = e - 3 * r;
        sm100::cp_async4(dst + 16 * r + 4 * q, g + e, 4);
      }
    }
    sm100::cp_async_commit();
  };
  auto words = [&](int i0, uint32_t (&wd)[R3_IPW]) {   // the chunk's contact bits per instance
#pragma unroll
    for (int x = 0; x < R3_IPW; ++x)
      wd[x] = ((live >> x) & 1u) ? (a.maskbits[mofs[x] + (i0 >> 5)] >> (i0 & 31)) : 0xffffffffu;
  };
  float2 d2a = make_float2(0.f, 0.f), d2b = d2a, d2c = d2a;   // dD2 rows 0..2, my channels
  uint32_t word[R3_IPW];
  if (grp.i0 < grp.i1) {
    stage(grp.i0, 0);
    words(grp.i0, word);
  }
  int buf = 0;
  for (int i0 = grp.i0; i0 < grp.i1; i0 += R3_NODES, buf ^= 1) {
    const int cn = min(R3_NODES, grp.i1 - i0);   // nodes in this chunk
    const bool more = i0 + R3_NODES < grp.i1;
    uint32_t wnext[R3_IPW];
    if (more) {
      stage(i0 + R3_NODES, buf ^ 1);
      words(i0 + R3_NODES, wnext);
      sm100::cp_async_wait_one();
    } else {
      sm100::cp_async_wait_all();
    }
    __syncthreads();
    const float (&sH0)[R3_NODES][H] = sm.H0[buf];
    const float4 (&sG)[R3_IPW][R3_NODES] = sm.G[buf][warp];
#pragma unroll 4
    for (int r = 0; r < R3_NODES; ++r) {
      float2 A3 = make_float2(0.f, 0.f);
      if (r < cn) {
        const float2 h0 = *reinterpret_cast<const float2*>(&sH0[r][2 * lane]);
#pragma unroll
        for (int x = 0; x < R3_IPW; ++x) {
          if ((word[x] >> r) & 1u) continue;   // active node or no contact: no decoder term
          const float4 g = sG[x][r];
          float2 dz = __fmul2_rn(w4a, make_float2(g.x, g.x));
          dz = __ffma2_rn(w4b, make_float2(g.y, g.y), dz);
          dz = __ffma2_rn(w4c, make_float2(g.z, g.z), dz);
          const float2 z = __fadd2_rn(h0, beta[x]);
          const float2 da = make_float2(z.x > 0.f ? dz.x : 0.f, z.y > 0.f ? dz.y : 0.f);
          const float2 rz = make_float2(relu(z.x), relu(z.y));
          S[x] = __fadd2_rn(S[x], da);
          A3 = __fadd2_rn(A3, da);
          d2a = __ffma2_rn(make_float2(g.x, g.x), rz, d2a);
          d2b = __ffma2_rn(make_float2(g.y, g.y), rz, d2b);
          d2c = __ffma2_rn(make_float2(g.z, g.z), rz, d2c);
        }
      }
      sA3[warp][r][lane] = A3;
    }
    // A3 of these nodes over the group's 64 instances: warps in order
    __syncthreads();
    for (int e = threadIdx.x; e < R3_NODES * 32; e += blockDim.x) {
      const int r = e >> 5, l = e & 31;
      if (r >= cn) continue;
      float2 s2 = sA3[0][r][l];
#pragma unroll
      for (int w = 1; w < 8; ++w) s2 = __fadd2_rn(s2, sA3[w][r][l]);
      *reinterpret_cast<float2*>(a.a3part + grp.a3off + (size_t)(i0 + r) * H + 2 * l) = s2;
    }
    if (more) {
#pragma unroll
      for (int x = 0; x < R3_IPW; ++x) word[x] = wnext[x];
    }
  }
#pragma unroll
  for (int x = 0; x < R3_IPW; ++x) {
    const int k = grp.k0 + R3_IPW * warp + x;
    if (k >= ninst) continue;
    float* sp = a.spart + ((size_t)(a.s_toff[t] + (long long)grp.srange * ninst) + k) * H;
    *reinterpret_cast<float2*>(sp + 2 * lane) = S[x];   // zero for instances without contact
  }
  sD2[warp][0][2 * lane] = d2a.x;
  sD2[warp][0][2 * lane + 1] = d2a.y;
  sD2[warp][1][2 * lane] = d2b.x;
  sD2[warp][1][2 * lane + 1] = d2b.y;
  sD2[warp][2][2 * lane] = d2c.x;
  sD2[warp][2][2 * lane + 1] = d2c.y;
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * H; e += blockDim.x) {
    float s2 = 0.f;
    for (int w = 0; w < 8; ++w) s2 += sD2[w][e / H][e % H];
    a.d2part[(size_t)blockIdx.x * 3 * H + e] = s2;
  }
}

// A3[type node][c] = sum over the type's groups of the partials: eight threads per entry
// (thread j sums groups j, j + 8, ... in order), combined by a fixed butterfly
__global__ void __launch_bounds__(256) bwd_reduce_a3_kernel(BwdBatchedArgs a) {
  const long long e = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 3;
  const int j = threadIdx.x & 7;
  const long long total = (long long)a.total_nodes * H;
  const bool in = e < total;
  const int node = in ? (int)(e / H) : 0, c = (int)(e % H);
  int t = 0;
  while (node >= a.type_off[t + 1]) ++t;
  const int o = a.type_off[t], n = a.type_off[t + 1] - o;
  const float* src = a.a3part + a.a3_toff[t] + (size_t)(node - o) * H + c;
  float s = 0.f;
  if (in)
    for (int g = j; g < a.a3_tgroups[t]; g += 8) s += src[(size_t)g * n * H];
  s += __shfl_xor_sync(FULL, s, 1);
  s += __shfl_xor_sync(FULL, s, 2);
  s += __shfl_xor_sync(FULL, s, 4);
  if (in && j == 0) a.a3[e] = s;
}

// ----------------------------------------------------------------------------- R4a
// 64 pads per CTA, two register-tiled products: S = dL/dbeta (the decoder partials of the
// pad's node ranges, summed in range order), dg = S D1_g, dag = dg [ag > 0], and
// dA2 = (dag G1) [g0 > 0]: each channel's dA2 at its argmax node (the pooled value is that
// node's ReLU(a2)).  Records S, dag and dA2 per pad.
constexpr int R4A_PADS = 64;

__global__ void __launch_bounds__(256) bwd_padmlp_kernel(BwdBatchedArgs a) {
  __shared__ __align__(16) float sW[H * TLD];   // [u][c] = D1[u][64 + c], then G1[c][k]
  __shared__ __align__(16) float sX[H * TLD];   // [k][pad]: S, then dag
  const float* W = a.params;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const int p0 = blockIdx.x * R4A_PADS;
  for (int e = tid; e < H * H; e += 256) {
    const int u = e >> 6, c = e & (H - 1);
    sW[u * TLD + c] = W[OFF_WD + u * 2 * H + H + c];
  }
  for (int e = tid; e < R4A_PADS * H; e += 256) {
    const int r = e >> 6, k = e & (H - 1), pad = p0 + r;
    float v = 0.f;
    if (pad < a.num_items && a.pad_m[pad] > 0) {
      const int ty = a.pad_type[pad];
      const int ninst = a.inst_off[ty + 1] - a.inst_off[ty];
      const float* sp = a.spart + ((size_t)a.s_toff[ty] + a.pad_inst[pad]) * H + k;
      for (int q = 0; q < a.s_nr[ty]; ++q) v += sp[(size_t)q * ninst * H];
      a.pr[(size_t)pad * PR_STRIDE + PR_S + k] = v;
    }
    sX[k * TLD + r] = v;
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sX, sW, ti, tj, acc);   // dg[pad][c]
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pad = p0 + 4 * ti + i;
    const bool live = pad < a.num_items && a.pad_m[pad] > 0;
    float* pr = a.pr + (size_t)(live ? pad : 0) * PR_STRIDE;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * tj + j;
      const float dag = live && pr[PR_AG + c] > 0.f ? acc[i][j] : 0.f;
      sX[c * TLD + 4 * ti + i] = dag;
      if (live) pr[PR_DAG + c] = dag;
    }
  }
  for (int e = tid; e < H * H; e += 256) {
    const int c = e >> 6, k = e & (H - 1);
    sW[c * TLD + k] = W[OFF_WG + c * H + k];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sX, sW, ti, tj, acc);   // dg0[pad][k]
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pad = p0 + 4 * ti + i;
    if (pad >= a.num_items || a.pad_m[pad] == 0) continue;
    float* pr = a.pr + (size_t)pad * PR_STRIDE;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = 4 * tj + j;
      pr[PR_D + k] = pr[PR_G0 + k] > 0.f ? acc[i][j] : 0.f;
    }
  }
}

// ----------------------------------------------------------------------------- R4
// warp per pad (static assignment, 8 warps per CTA), from the dA2 that bwd_padmlp_kernel
// recorded: the E1 reverse of each distinct argmax node.  The E1 / b1 partials live in
// registers (lane l owns units l and l + 32) and are summed over the CTA's warps in warp order.
// Per pad it records dA2, each channel's slot in the pad's list of distinct argmax nodes and
// those nodes' inputs, from which R4b sums dE2 and b2 per 64-pad chunk.
constexpr int R4_WARPS = 8;
constexpr int R4_LEN = OFF_W2 - OFF_W1;   // E1, b1
constexpr int R4_WREG = 2 * (NIN + 1) * 32;   // per-warp shared floats (inputs, then partials)

__global__ void __launch_bounds__(R4_WARPS * 32, 3) bwd_padrev_kernel(BwdBatchedArgs a) {
  __shared__ int sNode[R4_WARPS][H];
  __shared__ __align__(16) float sReg[R4_WARPS][R4_WREG];
  const float* W = a.params;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* sNodeW = sNode[warp];
  float* sX = sReg[warp];   // [slot][NIN] inputs of the pad's distinct argmax nodes
  float e1[2][NIN], b1[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    b1[h] = 0.f;
#pragma unroll
    for (int q = 0; q < NIN; ++q) e1[h][q] = 0.f;
  }
  const int gw = blockIdx.x * R4_WARPS + warp, nwarps = gridDim.x * R4_WARPS;
  for (int pad = gw; pad < a.num_items; pad += nwarps) {
    if (a.pad_m[pad] == 0) continue;
    float* pr = a.pr + (size_t)pad * PR_STRIDE;
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const long long base = a.pad_off[pad];
    const uint32_t* bits = a.maskbits + a.mask_woff[pad];
    const int rt0 = reinterpret_cast<const int*>(pr)[PR_ROUTE + lane];
    const int rt1 = reinterpret_cast<const int*>(pr)[PR_ROUTE + 32 + lane];
    float d[2];   // dA2 of channel k at its argmax node (bwd_padmlp_kernel)
    d[0] = pr[PR_D + lane];
    d[1] = pr[PR_D + 32 + lane];
    // routes: the distinct argmax nodes, channels 0..31 first (lowest lane of each node),
    // then nodes of channels 32..63 that no channel below 32 routes to; slot of each channel
    int nd = 0;
    {
      const unsigned lt = (1u << lane) - 1u;
      const unsigned m0 = __match_any_sync(FULL, rt0), m1 = __match_any_sync(FULL, rt1);
      const bool lead0 = (m0 & lt) == 0u;
      int in0 = -1;   // lowest channel below 32 that routes to rt1
      for (int l = 31; l >= 0; --l) in0 = __shfl_sync(FULL, rt0, l) == rt1 ? l : in0;
      const bool lead1 = (m1 & lt) == 0u && in0 < 0;
      const unsigned b0 = __ballot_sync(FULL, lead0), b1b = __ballot_sync(FULL, lead1);
      const int my0 = __popc(b0 & lt), my1 = __popc(b0) + __popc(b1b & lt);
      if (lead0) sNodeW[my0] = rt0;
      if (lead1) sNodeW[my1] = rt1;
      nd = __popc(b0) + __popc(b1b);
      const int slot0 = __shfl_sync(FULL, my0, __ffs(m0) - 1);
      const int sl1a = __shfl_sync(FULL, slot0, in0 < 0 ? 0 : in0);
      const int sl1b = __shfl_sync(FULL, my1, __ffs(m1) - 1);
      reinterpret_cast<int*>(pr)[PR_SLOT + lane] = slot0;
      reinterpret_cast<int*>(pr)[PR_SLOT + 32 + lane] = in0 >= 0 ? sl1a : sl1b;
      __syncwarp();
    }
    // inputs [p, n, u_hat] of the distinct nodes, one node per lane
    for (int q = lane; q < nd; q += 32) {
      const int node = sNodeW[q];
      const bool act = (bits[node >> 5] >> (node & 31)) & 1u;
      const float4 u = act ? a.ws_u[base + node] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float* pp = a.type_pos + 3 * (size_t)(o + node);
      const float* nn = a.type_nrm + 3 * (size_t)(o + node);
      const float xv[NIN] = {pp[0], pp[1], pp[2], nn[0], nn[1], nn[2], u.x, u.y, u.z};
#pragma unroll
      for (int j = 0; j < NIN; ++j) {
        sX[q * NIN + j] = xv[j];
        pr[PR_X + q * NIN + j] = xv[j];
      }
    }
    __syncwarp();
    const unsigned dz0 = __ballot_sync(FULL, d[0] != 0.f), dz1 = __ballot_sync(FULL, d[1] != 0.f);
    float4 duq[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    for (int q = 0; q < nd; ++q) {
      const int node = sNodeW[q];
      // the channels routed to this node with a nonzero dA2
      unsigned long long cm = (unsigned long long)(__ballot_sync(FULL, rt0 == node) & dz0) |
                              ((unsigned long long)(__ballot_sync(FULL, rt1 == node) & dz1) << 32);
      if (cm == 0ull) continue;   // warp-uniform
      // dh1 = sum over those channels of dA2_c E2[c, :] (lanes over units k)
      float dh1[2] = {0.f, 0.f};
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const float g = __shfl_sync(FULL, c < 32 ? d[0] : d[1], c & 31);
        dh1[0] = fmaf(__ldg(W + OFF_W2 + c * H + lane), g, dh1[0]);
        dh1[1] = fmaf(__ldg(W + OFF_W2 + c * H + 32 + lane), g, dh1[1]);
      }
      float x[NIN];
#pragma unroll
      for (int j = 0; j < NIN; ++j) x[j] = sX[q * NIN + j];
      // dA1 = dh1 [a1 > 0] (a1 of this node recomputed); dE1 += dA1 x^T; db1;
      // du_hat = E1[:, 6:9]^T dA1 (kept by lane q mod 32, applied to active nodes below)
      float du0 = 0.f, du1 = 0.f, du2 = 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        float v = __ldg(W + OFF_B1 + k);
#pragma unroll
        for (int q2 = 0; q2 < NIN; ++q2) v = fmaf(__ldg(W + OFF_W1 + k * NIN + q2), x[q2], v);
        const float d1 = v > 0.f ? dh1[h] : 0.f;
#pragma unroll
        for (int q2 = 0; q2 < NIN; ++q2) e1[h][q2] = fmaf(d1, x[q2], e1[h][q2]);
        b1[h] += d1;
        du0 = fmaf(__ldg(W + OFF_W1 + k * NIN + 6), d1, du0);
        du1 = fmaf(__ldg(W + OFF_W1 + k * NIN + 7), d1, du1);
        du2 = fmaf(__ldg(W + OFF_W1 + k * NIN + 8), d1, du2);
      }
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) {
        du0 += __shfl_xor_sync(FULL, du0, sh);
        du1 += __shfl_xor_sync(FULL, du1, sh);
        du2 += __shfl_xor_sync(FULL, du2, sh);
      }
      if (lane == (q & 31)) {
        if (q < 32) duq[0] = make_float4(du0, du1, du2, 1.f);
        else duq[1] = make_float4(du0, du1, du2, 1.f);
      }
    }
    // dL/du_hat of the active argmax nodes (distinct nodes: no two lanes share an entry)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = lane + 32 * h;
      if (q < nd && duq[h].w != 0.f) {
        const int node = sNodeW[q];
        if ((bits[node >> 5] >> (node & 31)) & 1u) {
          float4 dd = a.ws_du[base + node];
          dd.x += duq[h].x;
          dd.y += duq[h].y;
          dd.z += duq[h].z;
          a.ws_du[base + node] = dd;
        }
      }
    }
    __syncwarp();
  }
  // the CTA's partial of E1 and b1: warps summed in warp order (the warp's input slots are
  // reused for its partials once its pads are done)
  float* sP = sReg[warp];   // [h][q][lane], q = NIN is b1
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int q = 0; q < NIN; ++q) sP[(h * (NIN + 1) + q) * 32 + lane] = e1[h][q];
    sP[(h * (NIN + 1) + NIN) * 32 + lane] = b1[h];
  }
  __syncthreads();
  float* out = a.r4part + (size_t)blockIdx.x * R4_LEN;
  for (int e = threadIdx.x; e < R4_LEN; e += blockDim.x) {
    const int k = e < H * NIN ? e / NIN : e - H * NIN;   // E1 row k, column e % 9; then b1
    const int q = e < H * NIN ? e % NIN : NIN;
    const int idx = ((k >> 5) * (NIN + 1) + q) * 32 + (k & 31);
    float v = 0.f;
    for (int w = 0; w < R4_WARPS; ++w) v += sReg[w][idx];
    out[e] = v;
  }
}

// ----------------------------------------------------------------------------- R4b
// sums over pads (chunks of 64 pads, in order): dD1_g = sum S g^T, db_D1 = sum S,
// dG1 = sum dag g0^T, db_G1 = sum dag, and dE2 = sum over (pad, channel c) of
// dA2_c h1(argmax node of c)^T with db2 = sum dA2; h1 is recomputed from the recorded inputs
// (thread t owns unit t mod 64 of channels 16 (t / 64) .. + 15).  Partial layout per chunk:
// params [OFF_W2, OFF_W4).
constexpr int R4B_PADS = 64;
constexpr int R4B_LEN = OFF_W4 - OFF_W2;
constexpr int R4B_GRP = 8;   // pads staged at a time for the dE2 sums

constexpr int R4B_XS = 12;   // padded input row (three 16-byte reads)

struct R4bSmem {
  float A[R4B_PADS][TLD];             // S or dag per pad
  float B[R4B_PADS][TLD];             // g or g0 per pad
  float2 D[R4B_GRP][H];               // (dA2, slot bits) per channel
  float X[R4B_GRP][H][R4B_XS];        // inputs per slot
};

__global__ void __launch_bounds__(256) bwd_padsum_kernel(BwdBatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_r4b[];
  R4bSmem& sm = *reinterpret_cast<R4bSmem*>(smem_r4b);
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const int p0 = blockIdx.x * R4B_PADS;
  float* out = a.r4bpart + (size_t)blockIdx.x * R4B_LEN;
  const float* W = a.params;
  for (int which = 0; which < 2; ++which) {
    const int oa = which == 0 ? PR_S : PR_DAG, ob = which == 0 ? PR_G : PR_G0;
    for (int e = tid; e < R4B_PADS * H; e += 256) {
      const int r = e >> 6, c = e & (H - 1);
      const int pad = p0 + r;
      const bool ok = pad < a.num_items && a.pad_m[pad] > 0;
      const float* pr = a.pr + (size_t)(ok ? pad : 0) * PR_STRIDE;
      sm.A[r][c] = ok ? pr[oa + c] : 0.f;
      sm.B[r][c] = ok ? pr[ob + c] : 0.f;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    tile_acc(&sm.A[0][0], &sm.B[0][0], ti, tj, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * ti + i, k = 4 * tj + j;
        if (which == 0) out[OFF_WD - OFF_W2 + c * 2 * H + H + k] = acc[i][j];
        else out[OFF_WG - OFF_W2 + c * H + k] = acc[i][j];
      }
    if (tid < H) {
      float s = 0.f;
      for (int r = 0; r < R4B_PADS; ++r) s += sm.A[r][tid];
      if (which == 0) out[OFF_BD - OFF_W2 + tid] = s;
      else out[OFF_BG - OFF_W2 + tid] = s;
    }
    if (which == 0 && tid < 3) {   // sum of G over passive nodes (dL/db_D2), this chunk
      float g = 0.f;
      for (int r = 0; r < R4B_PADS; ++r) {
        const int pad = p0 + r;
        if (pad < a.num_items) g += a.pr[(size_t)pad * PR_STRIDE + PR_GSUM + tid];
      }
      a.gsum_part[(size_t)blockIdx.x * 3 + tid] = g;
    }
    if (which == 0) {   // the local half of D1 belongs to R5: zeros here
      for (int e = tid; e < H * H; e += 256) out[OFF_WD - OFF_W2 + (e >> 6) * 2 * H + (e & 63)] = 0.f;
    }
    __syncthreads();
  }
  // dE2[c][k] for unit k and channels cb .. cb + 15, pads of the chunk in order
  const int k = tid & (H - 1), cb = (tid >> 6) * 16;
  float w1[NIN];
#pragma unroll
  for (int q = 0; q < NIN; ++q) w1[q] = W[OFF_W1 + k * NIN + q];
  const float bk = W[OFF_B1 + k];
  float e2[16], b2[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) e2[j] = b2[j] = 0.f;
  // the chunk's records, R4B_GRP pads at a time: loaded into registers one group ahead,
  // stored to shared memory, then summed (every channel, including those with dA2 = 0, whose
  // slot is still a valid node of the pad, so the loop has no branch)
  constexpr int ND = R4B_GRP * H / 256, NX = R4B_GRP * H * NIN / 256;
  float2 rd[ND];
  float rx[NX];
  auto load = [&](int g0) {
#pragma unroll
    for (int u = 0; u < ND; ++u) {
      const int e = tid + 256 * u, r = e >> 6, c = e & (H - 1);
      const int pad = p0 + g0 + r;
      const bool ok = pad < a.num_items && a.pad_m[pad] > 0;
      const float* pr = a.pr + (size_t)(ok ? pad : 0) * PR_STRIDE;
      rd[u] = ok ? make_float2(pr[PR_D + c], __int_as_float(reinterpret_cast<const int*>(pr)[PR_SLOT + c]))
                 : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = tid + 256 * u, r = e / (H * NIN), jj = e - r * (H * NIN);
      const int pad = p0 + g0 + r;
      const bool ok = pad < a.num_items && a.pad_m[pad] > 0;
      rx[u] = ok ? a.pr[(size_t)pad * PR_STRIDE + PR_X + jj] : 0.f;
    }
  };
  load(0);
  for (int g0 = 0; g0 < R4B_PADS; g0 += R4B_GRP) {
#pragma unroll
    for (int u = 0; u < ND; ++u) {
      const int e = tid + 256 * u;
      sm.D[e >> 6][e & (H - 1)] = rd[u];
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int e = tid + 256 * u, r = e / (H * NIN), jj = e - r * (H * NIN);
      const int sl = jj / NIN;
      sm.X[r][sl][jj - sl * NIN] = rx[u];
    }
    __syncthreads();
    if (g0 + R4B_GRP < R4B_PADS) load(g0 + R4B_GRP);
    for (int r = 0; r < R4B_GRP; ++r) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float2 ds = sm.D[r][cb + j];   // warp-uniform
        const float* xr = sm.X[r][__float_as_int(ds.y)];
        const float4 xa = *reinterpret_cast<const float4*>(xr);
        const float4 xb = *reinterpret_cast<const float4*>(xr + 4);
        const float x8 = xr[8];
        float v0 = fmaf(w1[0], xa.x, bk), v1 = w1[1] * xa.y;
        v0 = fmaf(w1[2], xa.z, v0);
        v1 = fmaf(w1[3], xa.w, v1);
        v0 = fmaf(w1[4], xb.x, v0);
        v1 = fmaf(w1[5], xb.y, v1);
        v0 = fmaf(w1[6], xb.z, v0);
        v1 = fmaf(w1[7], xb.w, v1);
        v0 = fmaf(w1[8], x8, v0);
        e2[j] = fmaf(ds.x, relu(v0 + v1), e2[j]);
        b2[j] += ds.x;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) out[(cb + j) * H + k] = e2[j];
  if (k == 0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) out[OFF_B2 - OFF_W2 + cb + j] = b2[j];
  }
}

// ----------------------------------------------------------------------------- R5
// 64 type nodes per CTA: the decoder path's encoder reverse with passive inputs [p, n, 0]:
// dD1_f += A3^T F0 ; dF = A3 D1_f ; dA2 = dF [f0 > 0] ; dE2 += dA2^T H1 ; dH1 = dA2 E2 ;
// dA1 = dH1 [c > 0] ; dE1[:, 0:6] += dA1^T [P N] ; biases.  Partial layout per CTA: params
// [OFF_W1, OFF_W4) (the global half of D1 and G1 stay zero).
constexpr int R5_LEN = OFF_W4 - OFF_W1;

__global__ void __launch_bounds__(256) bwd_typenode_kernel(BwdBatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* sA3 = reinterpret_cast<float*>(smem);        // [r][c]
  float* sA3T = sA3 + 64 * TLD;                        // [c][r]
  float* sF0 = sA3T + 64 * TLD;                        // [r][k]
  float* sH1 = sF0 + 64 * TLD;                         // [r][k]
  float* sWd = sH1 + 64 * TLD;                         // D1_f [c][k]
  float* sW2 = sWd + 64 * TLD;                         // E2 [c][k]
  float* sD = sW2 + 64 * TLD;                          // dA2 [r][c]
  float* sDT = sD + 64 * TLD;                          // dA2 [c][r]
  float* sX = sDT + 64 * TLD;                          // [r][6]
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const float* W = a.params;
  const int r0 = blockIdx.x * 64;
  float* out = a.r5part + (size_t)blockIdx.x * R5_LEN;
  for (int e = tid; e < R5_LEN; e += 256) out[e] = 0.f;
  for (int e = tid; e < 64 * H; e += 256) {
    const int r = e >> 6, c = e & (H - 1);
    const int node = r0 + r;
    const bool ok = node < a.total_nodes;
    const float v = ok ? a.a3[(size_t)node * H + c] : 0.f;
    sA3[r * TLD + c] = v;
    sA3T[c * TLD + r] = v;
    sF0[r * TLD + c] = ok ? a.f0tab[(size_t)node * H + c] : 0.f;
    sH1[r * TLD + c] = ok ? relu(a.ctab[(size_t)node * H + c]) : 0.f;
    sWd[r * TLD + c] = W[OFF_WD + r * 2 * H + c];
    sW2[r * TLD + c] = W[OFF_W2 + r * H + c];
  }
  for (int e = tid; e < 64 * 6; e += 256) {
    const int r = e / 6, q = e % 6;
    const int node = r0 + r;
    const bool ok = node < a.total_nodes;
    sX[e] = ok ? (q < 3 ? a.type_pos[3 * (size_t)node + q] : a.type_nrm[3 * (size_t)node + q - 3]) : 0.f;
  }
  __syncthreads();
  float acc[4][4];
  // dD1_f[c][k] = sum_r A3[r][c] F0[r][k]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sA3, sF0, ti, tj, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[OFF_WD - OFF_W1 + (4 * ti + i) * 2 * H + 4 * tj + j] = acc[i][j];
  // dF[r][k] = sum_c A3[r][c] D1_f[c][k] ; dA2 = dF [f0 > 0]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sA3T, sWd, ti, tj, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = 4 * ti + i, k = 4 * tj + j;
      const float d = sF0[r * TLD + k] > 0.f ? acc[i][j] : 0.f;
      sD[r * TLD + k] = d;
      sDT[k * TLD + r] = d;
    }
  __syncthreads();
  // dE2[c][k] = sum_r dA2[r][c] H1[r][k] ; db2
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  tile_acc(sD, sH1, ti, tj, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[OFF_W2 - OFF_W1 + (4 * ti + i) * H + 4 * tj + j] = acc[i][j];
  if (tid < H) {
    float s = 0.f;
    for (int r = 0; r < 64; ++r) s += sD[r * TLD + tid];
    out[OFF_B2 - OFF_W1 + tid] = s;
  }
  // dH1[r][k] = sum_c dA2[r][c] E2[c][k] ; dA1 = dH1 [c > 0] (into sA3, no longer needed)
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
      sA3[r * TLD + k] = sH1[r * TLD + k] > 0.f ? acc[i][j] : 0.f;
    }
  __syncthreads();
  // dE1[c][q] = sum_r dA1[r][c] X[r][q] (q < 6) ; db1
  for (int e = tid; e < H * 7; e += 256) {
    const int c = e / 7, q = e % 7;
    float s = 0.f;
    for (int r = 0; r < 64; ++r) s = fmaf(sA3[r * TLD + c], q < 6 ? sX[r * 6 + q] : 1.f, s);
    if (q < 6) out[c * NIN + q] = s;
    else out[OFF_B1 - OFF_W1 + c] = s;
  }
}

// ----------------------------------------------------------------------------- R7
// warp per pad: dL/du_hat and dL/dpen per node, and the pose partials (active nodes in
// node order)
// R7a: dL/du_hat (the propagated sum for active nodes, 0 for passive ones) and, for passive
// nodes, dL/dpen = 0: a streaming pass over every node, warp per pad (the active nodes'
// penetration gradients come from R7b)
__global__ void __launch_bounds__(256) bwd_fill_kernel(BwdBatchedArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int pad = blockIdx.x * wpb + warp; pad < a.num_items; pad += gridDim.x * wpb) {
    const int ty = a.pad_type[pad];
    const int n = a.type_off[ty + 1] - a.type_off[ty];
    const long long base = a.pad_off[pad];
    const int m = a.pad_m[pad];
    const uint32_t* bits = a.maskbits + a.mask_woff[pad];
#pragma unroll 4
    for (int i = lane; i < n; i += 32) {
      const bool act = m > 0 && ((bits[i >> 5] >> (i & 31)) & 1u);
      if (a.grad_uhat) {
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (act) d = a.ws_du[base + i];
        float* g = a.grad_uhat + 3 * (base + i);
        g[0] = d.x;
        g[1] = d.y;
        g[2] = d.z;
      }
      if (a.grad_pen && !act) a.grad_pen[base + i] = 0.f;
    }
  }
}

// R7b: the active nodes' dL/dpen and pose partials through the SDF gradient and Hessian, warp
// per pad.  The pad's active nodes are compacted (in node order) into a per-warp queue, so all
// 32 lanes of a pass take one active node each; lane l takes queue entries l, l + 32, ... of the
// pad and adds its terms, in that order, to its own column of the warp's pose accumulators in
// shared memory ([object][6][lane]: no bank conflicts, no registers held per object slot); the
// columns are then summed over lanes in a fixed order.
constexpr int POSE_Q = 64;   // per-warp queue of active nodes (<= 31 pending + 32 of a word)
constexpr int POSE_T = 128;  // threads per CTA (95 registers: 5 CTAs per SM)
struct PoseSmem {
  size_t po, q, acc, warp_bytes;
  __host__ __device__ explicit PoseSmem(int K) {
    po = 0;
    q = sizeof(PadObj) * (size_t)K;
    acc = (q + sizeof(int16_t) * POSE_Q + 15) & ~size_t(15);
    warp_bytes = acc + sizeof(float) * 6 * 32 * (size_t)K;
  }
  __host__ __device__ size_t total() const { return warp_bytes * (POSE_T / 32); }
};
template <bool MESH>
__global__ void __launch_bounds__(POSE_T) bwd_pose_kernel(BwdBatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const PoseSmem L(a.K);
  unsigned char* wb = smem + (size_t)warp * L.warp_bytes;
  PadObj* spo = reinterpret_cast<PadObj*>(wb + L.po);
  int16_t* sq = reinterpret_cast<int16_t*>(wb + L.q);
  float* sacc = reinterpret_cast<float*>(wb + L.acc);   // [k][6][32]
  const unsigned lt = (1u << lane) - 1u;
  for (int pad = blockIdx.x * wpb + warp; pad < a.num_items; pad += gridDim.x * wpb) {
    const int m = a.pad_m[pad];
    if (m == 0) continue;   // warp-uniform
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const int env = pad / a.P;
    const long long base = a.pad_off[pad];
    {
      const int* src = reinterpret_cast<const int*>(a.padobj + (size_t)pad * a.K);
      int* dst = reinterpret_cast<int*>(spo);
      const int words = a.K * (int)(sizeof(PadObj) / 4);
      for (int e = lane; e < words; e += 32) dst[e] = src[e];
    }
    for (int e = 0; e < 6 * a.K; ++e) sacc[32 * e + lane] = 0.f;
    __syncwarp();
    const uint32_t* bits = a.maskbits + a.mask_woff[pad];
    const bool given = a.mask_in != nullptr;   // mode B: no SDF, no pose or penetration gradient
    const float* pp = given ? nullptr : a.pad_pose + 7 * (size_t)pad;
    float Rp[3][3] = {};
    if (!given) quat_to_mat<float>(pp + 3, Rp);
    const float* op_env = a.obj_pose + 7 * (size_t)env * a.K;
    float gap = 0.f;
    for (int k = 0; k < a.K; ++k) gap = fmaxf(gap, 2.f * spo[k].tau);
    // one active node per lane (lane < cnt): its penetration gradient and pose partials
    auto run = [&](int cnt) {
      if (lane < cnt) {
        const int i = sq[lane];
        const float4 d = a.ws_du[base + i];
        const float3 du = make_float3(d.x, d.y, d.z);
        const float* tp = a.type_pos + 3 * (size_t)(o + i);
        const float* tn = a.type_nrm + 3 * (size_t)(o + i);
        const float3 p = make_float3(tp[0], tp[1], tp[2]);
        const float3 nr = make_float3(tn[0], tn[1], tn[2]);
        float pen = 0.f;
        if (!given) {
          const NodePoseGrad pg = node_pose_grad<MESH>(spo, a.K, p, nr, du, Rp, pp, op_env, gap);
          pen = pg.pen;
          if (pg.k >= 0) {
            float* ac = sacc + (size_t)pg.k * 6 * 32 + lane;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              ac[32 * q] += pg.t[q];
              ac[32 * (3 + q)] += pg.w[q];
            }
          }
        }
        if (a.grad_pen) a.grad_pen[base + i] = pen;
      }
      __syncwarp();
    };
    int npend = 0;   // warp-uniform
    const int nwords = (n + 31) >> 5;
    for (int w = 0; w < nwords; ++w) {
      const uint32_t bw = bits[w];   // every lane reads the same word
      if (bw & (1u << lane)) sq[npend + __popc(bw & lt)] = (int16_t)(32 * w + lane);
      npend += __popc(bw);
      __syncwarp();
      if (npend >= 32) {
        run(32);
        // the rest of the queue moves to the front (at most 31 entries)
        const int rest = npend - 32;
        const int16_t v = lane < rest ? sq[32 + lane] : (int16_t)0;
        __syncwarp();
        if (lane < rest) sq[lane] = v;
        npend = rest;
        __syncwarp();
      }
    }
    if (npend > 0) run(npend);
    for (int e = 0; e < 6 * a.K; ++e) {
      float v = sacc[32 * e + lane];
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(FULL, v, sh);
      if (lane == 0) a.pose_part[(size_t)pad * a.K * 6 + e] = v;
    }
    __syncwarp();
  }
  // pads without contact: zero pose partials (every warp covers its own pads)
  for (int pad = blockIdx.x * wpb + warp; pad < a.num_items; pad += gridDim.x * wpb) {
    if (a.pad_m[pad] != 0) continue;
    for (int e = lane; e < 6 * a.K; e += 32) a.pose_part[(size_t)pad * a.K * 6 + e] = 0.f;
  }
}

// ----------------------------------------------------------------------------- final sums
// grad_params[q]: the sums of every stage's partials that cover q.  Eight threads per
// parameter: thread j sums partials j, j + 8, ... of each stage in order, and a fixed
// butterfly combines the eight (one thread per parameter left a few warps per SM, each
// walking hundreds of partials in sequence)
__global__ void __launch_bounds__(256) bwd_reduce_params_kernel(BwdBatchedArgs a, float* out) {
  const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 3);
  const int j = threadIdx.x & 7;
  float s = 0.f;
  if (q < NPARAM) {
    if (q >= OFF_W1 && q < OFF_W2)
      for (int w = j; w < a.r4_parts; w += 8) s += a.r4part[(size_t)w * R4_LEN + q - OFF_W1];
    if (q >= OFF_W1 && q < OFF_W4)
      for (int b = j; b < a.r5_parts; b += 8) s += a.r5part[(size_t)b * R5_LEN + q - OFF_W1];
    if (q >= OFF_W2 && q < OFF_W4)
      for (int b = j; b < a.r4b_parts; b += 8) s += a.r4bpart[(size_t)b * R4B_LEN + q - OFF_W2];
    if (q >= OFF_W4 && q < OFF_W4 + 3 * H)
      for (int b = j; b < a.r3_parts; b += 8) s += a.d2part[(size_t)b * 3 * H + q - OFF_W4];
    if (q >= OFF_B4 && q < OFF_B4 + 3)
      for (int b = j; b < a.r4b_parts; b += 8) s += a.gsum_part[(size_t)b * 3 + q - OFF_B4];
    if (q == OFF_ALPHA)
      for (int b = j; b < a.alpha_parts; b += 8) s -= a.alpha_part[b];
  }
  s += __shfl_xor_sync(FULL, s, 1);
  s += __shfl_xor_sync(FULL, s, 2);
  s += __shfl_xor_sync(FULL, s, 4);
  if (q < NPARAM && j == 0) out[q] = s;
}

}  // namespace

size_t bwd_pad_smem_bytes(int nmax, int K) { return R1Smem(nmax, K).total; }

cudaError_t bwd_pad_occupancy(int nmax, int K, int* blocks_per_sm) {
  const size_t smem = R1Smem(nmax, K).total;
  cudaError_t e = cudaFuncSetAttribute(bwd_pad_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bwd_pad_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e != cudaSuccess) return e;
  int a = 0, b = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, bwd_pad_kernel<false>, RT, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bwd_pad_kernel<true>, RT, smem);
  *blocks_per_sm = a < b ? a : b;   // the grid suits either instantiation
  return e;
}

// one stage of the staged reverse mode (BWD_STAGE_*), launched on stream s
cudaError_t launch_backward_stage(const BwdBatchedArgs& a, const BwdBatchedLaunch& l, int stage,
                                  float* grad_params, cudaStream_t s) {
  switch (stage) {
    case BWD_STAGE_PAD: {
      const size_t smem = R1Smem(a.nmax, a.K).total;
      static size_t configured = 0;
      if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(bwd_pad_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(bwd_pad_kernel<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
      }
      if (a.has_meshes)
        bwd_pad_kernel<true><<<l.r1_grid, RT, smem, s>>>(a);
      else
        bwd_pad_kernel<false><<<l.r1_grid, RT, smem, s>>>(a);
      break;
    }
    case BWD_STAGE_GLOBAL:
      bwd_global_kernel<<<(a.num_items + R2_PADS - 1) / R2_PADS, 256, 0, s>>>(a);
      break;
    case BWD_STAGE_DECODER: {
      static bool c3 = false;
      if (!c3) {
        cudaError_t e = cudaFuncSetAttribute(bwd_decoder_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(R3Smem));
        if (e != cudaSuccess) return e;
        c3 = true;
      }
      bwd_decoder_kernel<<<a.r3_parts, 256, sizeof(R3Smem), s>>>(a);
      break;
    }
    case BWD_STAGE_A3SUM: {
      const long long tot = (long long)a.total_nodes * H * 8;
      bwd_reduce_a3_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a);
      break;
    }
    case BWD_STAGE_PADREV: {
      bwd_padmlp_kernel<<<(a.num_items + R4A_PADS - 1) / R4A_PADS, 256, 0, s>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      bwd_padrev_kernel<<<a.r4_parts, R4_WARPS * 32, 0, s>>>(a);
      break;
    }
    case BWD_STAGE_PADSUM: {
      static bool c4b = false;
      if (!c4b) {
        cudaError_t e = cudaFuncSetAttribute(bwd_padsum_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(R4bSmem));
        if (e != cudaSuccess) return e;
        c4b = true;
      }
      bwd_padsum_kernel<<<a.r4b_parts, 256, sizeof(R4bSmem), s>>>(a);
      break;
    }
    case BWD_STAGE_TYPENODE: {
      const size_t s5 = sizeof(float) * (8 * 64 * TLD + 64 * 6);
      static bool c5 = false;
      if (!c5) {
        cudaError_t e = cudaFuncSetAttribute(bwd_typenode_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s5);
        if (e != cudaSuccess) return e;
        c5 = true;
      }
      bwd_typenode_kernel<<<a.r5_parts, 256, s5, s>>>(a);
      break;
    }
    case BWD_STAGE_POSE:
    {
      bwd_fill_kernel<<<l.r7_grid, 256, 0, s>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      const size_t smem = PoseSmem(a.K).total();
      static size_t configured = 0;
      if (smem > configured) {
        e = cudaFuncSetAttribute(bwd_pose_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(bwd_pose_kernel<true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
      }
      const int grid = l.r7_grid * (256 / POSE_T);   // r7_grid counts 8-warp CTAs
      if (a.has_meshes)
        bwd_pose_kernel<true><<<grid, POSE_T, smem, s>>>(a);
      else
        bwd_pose_kernel<false><<<grid, POSE_T, smem, s>>>(a);
      break;
    }
    case BWD_STAGE_PARAMS:
      if (grad_params) bwd_reduce_params_kernel<<<(8 * NPARAM + 255) / 256, 256, 0, s>>>(a, grad_params);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace etac
