// front.cu -- front half of the BF16 tensor-core ETac step (ETac Sec. III-A).
//
// pad_obj_kernel (one thread per pad): the pad -> object relative transforms (FP32 and df32)
//   and the FP32 screening margins, so that no pad's work starts with a serial setup chain.
// front_contact_kernel (persistent, one WARP per pad from a work queue, heaviest pads first;
//   warps never wait on each other, so the latency of one pad's chain hides behind the others):
//   the warp streams over its pad's nodes, 32 per step:
//   * one FP32 pass sorts each node: certainly outside every object (passive), certainly inside
//     with no near-tie among the discrete choices (u_hat from FP32 arithmetic, the BF16 step's
//     error budget), or undecided (a thin band near a surface or a tie);
//   * undecided nodes go to a short list and take the exact df32 decision 32 at a time (called
//     out of line: it runs rarely, and inlined it crowds the loop's instruction cache), so
//     contact sets equal the exact ones;
//   * active nodes keep u_hat (Eq. 4 covers passive nodes only), their u_hat goes to the
//     propagation GEMM's B operand, their contact bit to a per-pad bit field, and they are
//     pushed on a short stack that the encoder drains 16 at a time on tensor cores (E1
//     evaluated straight into the m16n8k16 A-fragment layout, E2 as BF16 MMAs with FP32
//     accumulation); the running channel maxima live in shared memory between drains.
//     Passive nodes need no encoder: their outputs are table entries;
//   * at the end, the max-pool over the passive nodes: the first passive node of each
//     channel's table order (ranked f0 values), 32 ranks per warp-wide test.
// front_global_kernel (64 pads per CTA, two register-tiled products; one warp per pad for
//   batches under 64 pads per SM): global MLP g = ReLU(G1 g0), the decoder's global half
//   beta = D1[:, 64:] g, and the record the propagation GEMM's epilogue needs: -beta in BF16
//   and D2 beta + b_D2 (ReLU(h0 + beta) = max(h0, -beta) + beta).
#include <cuda_bf16.h>

#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {

namespace {

constexpr int FT = 256;      // threads per CTA: eight independent pad warps
constexpr int FW = FT / 32;
constexpr int PEND = 48;     // per-warp stack of active nodes awaiting the encoder (<= 15 + 32)
constexpr int CANDCAP = 64;  // per-warp list of undecided nodes awaiting the exact path
constexpr unsigned FULL = 0xffffffffu;

// shared weights, then one region per warp
struct FrontSmem {
  size_t w2f, w1f, b2, warp0, warp_bytes, po, bits, obits, pend_a, cand, fmax, fmlane, total;
  __host__ __device__ FrontSmem(int nmax, int K) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    w2f = take(sizeof(uint2) * 8 * 4 * 32);
    w1f = take(sizeof(uint2) * 2 * 8 * 32);
    b2 = take(sizeof(float) * H);
    warp0 = o;
    o = 0;
    po = take(sizeof(PadObj) * (size_t)K);
    bits = take(sizeof(uint32_t) * (size_t)((nmax + 31) / 32));
    obits = take(sizeof(uint32_t) * (size_t)((nmax + 31) / 32));
    pend_a = take(sizeof(uint4) * 2 * PEND);
    cand = take(sizeof(int16_t) * CANDCAP);
    fmax = take(sizeof(float) * H);
    fmlane = take(sizeof(float) * 16 * 32);
    warp_bytes = o;
    total = warp0 + FW * warp_bytes;
  }
};

// every pad's relative transforms and screening margins, one thread per pad (object slots in
// turn); pad_bad[pad] = 1 when one of its poses or sizes is not finite
__global__ void __launch_bounds__(256) pad_obj_kernel(FrontArgs a) {
  const int pad = blockIdx.x * blockDim.x + threadIdx.x;
  if (pad >= a.num_items) return;
  const int env = pad / a.P;
  if (a.mask_in) {   // mode B: contact supplied by the caller, no object is read
    PadObj po{};
    po.type = OBJ_NONE;
    for (int k = 0; k < a.K; ++k) a.padobj[(size_t)pad * a.K + k] = po;
    a.pad_bad[pad] = 0;
    return;
  }
  const float* pp = a.pad_pose + 7 * (size_t)pad;
  const float pmax = a.type_pmax[a.pad_type[pad]];
  int bad = 0;
  for (int k = 0; k < a.K; ++k) {
    const int ob = env * a.K + k;
    const float* op = a.obj_pose + 7 * (size_t)ob;
    const float* od = a.obj_dims + 3 * (size_t)ob;
    int type = a.obj_type[ob];
    if (type < OBJ_NONE || type > OBJ_MESH) type = OBJ_NONE;
    const MeshDev* mesh = nullptr;
    if (type == OBJ_MESH && !(mesh = object_mesh(od, a.meshes, a.num_meshes))) type = OBJ_NONE;
    const bool ok = finite7(op) && finite7(pp) && isfinite(od[0]) && isfinite(od[1]) &&
                    isfinite(od[2]);
    if (!ok && type != OBJ_NONE) {
      bad = 1;
      type = OBJ_NONE;
    }
    PadObj po;
    setup_pad_obj(op, type, od, pp, pmax, &po, mesh);
    a.padobj[(size_t)pad * a.K + k] = po;
  }
  a.pad_bad[pad] = bad;
}

// Writes a decided node's outputs: the B-operand row entries (only when the node is active
// or was active in the previous step: the other entries are zero already), mask,
// penetration and, for an active node, its displacement (= u_hat).
__device__ __forceinline__ void front_write_node(const FrontArgs& a, __nv_bfloat16* btrow, int n,
                                                 long long base, int i, const NodeContact& c,
                                                 bool was) {
  if ((c.active || was) &&
      ETAC_IN(a.status, btrow - reinterpret_cast<const __nv_bfloat16*>(a.bt) + 2 * n + i,
              a.bt_total)) {
    btrow[i] = __float2bfloat16_rn(c.u[0]);
    btrow[n + i] = __float2bfloat16_rn(c.u[1]);
    btrow[2 * n + i] = __float2bfloat16_rn(c.u[2]);
  }
  if (!ETAC_IN(a.status, base + i, a.num_nodes)) return;
  if (a.mask) a.mask[base + i] = c.active ? 1 : 0;
  if (a.pen) a.pen[base + i] = c.active ? -c.phi : 0.f;
  if (c.active) {
    float* d = a.disp + 3 * (base + i);
    d[0] = c.u[0];
    d[1] = c.u[1];
    d[2] = c.u[2];
  }
}

// E1 input row of an active node, 16 BF16 values: [p_hi, p_lo, n_hi, n_lo, u_hat, 1].  The
// position and normal are split into two BF16 parts (p = p_hi + p_lo to 16 bits), so with W1
// split the same way the first layer is evaluated to about FP32 accuracy on tensor cores;
// u_hat enters rounded to BF16.
__device__ __forceinline__ uint32_t bf2_bits(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf_rest(float x) {   // x - BF16(x), itself rounded later
  return x - __bfloat162float(__float2bfloat16_rn(x));
}
// The exact (df32) decision of an undecided node, kept out of line: it runs for a thin band of
// nodes only, and inlined its code crowds the instruction cache of the streaming loop.
template <bool MESH>
__device__ __noinline__ NodeContact front_refine(const PadObj* po, int K, float3 p, float3 nrm) {
  return contact_refine<MESH>(po, K, p, nrm, 0.f);
}

__device__ __forceinline__ void front_pack_row(uint4* dst, float3 p, float3 nr, const float* u) {
  dst[0] = make_uint4(bf2_bits(p.x, p.y), bf2_bits(p.z, bf_rest(p.x)),
                      bf2_bits(bf_rest(p.y), bf_rest(p.z)), bf2_bits(nr.x, nr.y));
  dst[1] = make_uint4(bf2_bits(nr.z, bf_rest(nr.x)), bf2_bits(bf_rest(nr.y), bf_rest(nr.z)),
                      bf2_bits(u[0], u[1]), bf2_bits(u[2], 1.f));
}

// Encoder of up to 16 active nodes on tensor cores, rows = E1 input rows (front_pack_row) at
// shared address `rows` (16 consecutive 32-byte rows; rows at or beyond cnt are ignored):
// h = ReLU(W1 x + b1) as 2 x 8 m16n8k16 MMAs (W1 hi and lo parts, bias in the constant
// column), whose accumulators are the A fragments of y = E2 h (32 MMAs); y is folded into the
// per-lane running channel maxima fm (the bias and the outer ReLU commute with the max:
// max ReLU(y + b) = ReLU(max y + b)).  Lane (grp, tig) holds rows grp and grp + 8 and channels
// 8 nt + 2 tig + {0, 1}.
__device__ __forceinline__ void front_encode(float (&fm)[8][2], uint32_t rows, int cnt,
                                             const uint2* sW1f, const uint2* sW2f, int lane) {
  const int grp = lane >> 2;
  const bool v0 = grp < cnt, v1 = grp + 8 < cnt;
  uint32_t ax[4];
  sm100::ldmatrix_x4(rows + (uint32_t)((lane & 15) * 32 + (lane >> 4) * 16), ax[0], ax[1], ax[2],
                     ax[3]);
  uint32_t af[4][4];
#pragma unroll
  for (int s4 = 0; s4 < 4; ++s4) {
    // n tiles 2 s4 and 2 s4 + 1 as two interleaved chains (W1 hi, then lo)
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint2 b = sW1f[(8 * part + 2 * s4 + t) * 32 + lane];
        sm100::mma_bf16_16816(acc[t], ax, b.x, b.y, acc[t]);
      }
    __nv_bfloat162 p0 = __floats2bfloat162_rn(fmaxf(acc[0][0], 0.f), fmaxf(acc[0][1], 0.f));
    __nv_bfloat162 p1 = __floats2bfloat162_rn(fmaxf(acc[0][2], 0.f), fmaxf(acc[0][3], 0.f));
    __nv_bfloat162 p2 = __floats2bfloat162_rn(fmaxf(acc[1][0], 0.f), fmaxf(acc[1][1], 0.f));
    __nv_bfloat162 p3 = __floats2bfloat162_rn(fmaxf(acc[1][2], 0.f), fmaxf(acc[1][3], 0.f));
    af[s4][0] = *reinterpret_cast<uint32_t*>(&p0);
    af[s4][1] = *reinterpret_cast<uint32_t*>(&p1);
    af[s4][2] = *reinterpret_cast<uint32_t*>(&p2);
    af[s4][3] = *reinterpret_cast<uint32_t*>(&p3);
  }
  // E2 in two halves of four n tiles, four interleaved chains each (k steps ascending)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint2 bb = sW2f[((4 * half + j) * 4 + s4) * 32 + lane];
        sm100::mma_bf16_16816(acc[j], af[s4], bb.x, bb.y, acc[j]);
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nt = 4 * half + j;
      fm[nt][0] = fmaxf(fm[nt][0], fmaxf(v0 ? acc[j][0] : -INFINITY, v1 ? acc[j][2] : -INFINITY));
      fm[nt][1] = fmaxf(fm[nt][1], fmaxf(v0 ? acc[j][1] : -INFINITY, v1 ? acc[j][3] : -INFINITY));
    }
  }
}

// MESH: the context has mesh objects (the FP32 mesh query is compiled in; without meshes it
// is left out, so its out-of-line call costs the streaming loop no registers)
template <bool MESH>
__global__ void __launch_bounds__(FT, 4) front_contact_kernel(FrontArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const FrontSmem L(a.nmax, a.K);
  uint2* sW2f = reinterpret_cast<uint2*>(smem + L.w2f);
  uint2* sW1f = reinterpret_cast<uint2*>(smem + L.w1f);
  float* sB2 = reinterpret_cast<float*>(smem + L.b2);
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
  // E1 as B fragments over the 16-wide input row [p_hi, p_lo, n_hi, n_lo, u, 1]: input k reads
  // W1 column kcol(k) (b1 for k = 15); entry (part, nt, l): part 0 = BF16(W), 1 = BF16(W - hi)
  for (int e = tid; e < 2 * 8 * 32; e += FT) {
    const int l = e & 31, nt = (e >> 5) & 7, part = e >> 8;
    const int n = 8 * nt + (l >> 2), k0 = 2 * (l & 3);
    auto wv = [&](int k) {
      const int col = k < 6 ? k % 3 : (k < 12 ? 3 + (k - 6) % 3 : 6 + (k - 12));
      const float w = k == 15 ? W[OFF_B1 + n] : W[OFF_W1 + n * NIN + col];
      const __nv_bfloat16 h = __float2bfloat16_rn(w);
      return part == 0 ? h : __float2bfloat16_rn(w - __bfloat162float(h));
    };
    __nv_bfloat162 lo = __halves2bfloat162(wv(k0), wv(k0 + 1));
    __nv_bfloat162 hi = __halves2bfloat162(wv(k0 + 8), wv(k0 + 9));
    sW1f[e] = make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
  }
  for (int i = tid; i < H; i += FT) sB2[i] = W[OFF_B2 + i];
  __syncthreads();   // the only block barrier: from here on every warp runs its own pads

  unsigned char* wb = smem + L.warp0 + (size_t)warp * L.warp_bytes;
  PadObj* spo = reinterpret_cast<PadObj*>(wb + L.po);
  uint32_t* sBits = reinterpret_cast<uint32_t*>(wb + L.bits);
  uint32_t* sOld = reinterpret_cast<uint32_t*>(wb + L.obits);   // previous B-operand bits
  uint4* sPendA = reinterpret_cast<uint4*>(wb + L.pend_a);
  const uint32_t sPendA_addr = (uint32_t)__cvta_generic_to_shared(sPendA);
  int16_t* sCand = reinterpret_cast<int16_t*>(wb + L.cand);
  float* sFmax = reinterpret_cast<float*>(wb + L.fmax);
  float* sFm = reinterpret_cast<float*>(wb + L.fmlane) + lane;   // lane's maxima, stride 32
  const unsigned lt = (1u << lane) - 1u;
  const bool enc = uses_residual(a.mode);

  // the next work item is fetched while the current one is processed
  int next = 0;
  if (lane == 0) next = atomicAdd(a.ticket, 1);
  for (;;) {
    __syncwarp();   // the previous pad's shared-memory reads are done
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
    __nv_bfloat16* btrow =
        reinterpret_cast<__nv_bfloat16*>(a.bt) + a.bt_off[ty] + (size_t)3 * a.pad_inst[pad] * n;
    {
      const int* src = reinterpret_cast<const int*>(a.padobj + (size_t)pad * a.K);
      int* dst = reinterpret_cast<int*>(spo);
      const int words = a.K * (int)(sizeof(PadObj) / 4);
      for (int e = lane; e < words; e += 32) dst[e] = src[e];
    }
    const bool invalid = a.pad_bad[pad] != 0;
    __syncwarp();
    float gap = 0.f;   // twice the largest FP32 error bound over the pad's objects
    for (int k = 0; k < a.K; ++k) gap = fmaxf(gap, 2.f * spo[k].tau);

    // running channel maxima live in shared memory between drains (registers go to the
    // contact pass)
#pragma unroll
    for (int q = 0; q < 16; ++q) sFm[32 * q] = -INFINITY;
    int npend = 0, ncand = 0, m = 0;   // warp-uniform

    // exact decision of the top (up to) 32 undecided nodes; the active ones join the stack
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
        c = front_refine<MESH>(spo, a.K, p, nr);
        front_write_node(a, btrow, n, base, i, c, (sOld[i >> 5] >> (i & 31)) & 1u);
        if (c.active) atomicOr(&sBits[i >> 5], 1u << (i & 31));
      }
      ncand -= cnt;
      const unsigned b = __ballot_sync(FULL, c.active);
      if (c.active && enc) {
        const int q = npend + __popc(b & lt);
        front_pack_row(sPendA + 2 * q, p, nr, c.u);
      }
      m += __popc(b);
      if (enc) npend += __popc(b);
      __syncwarp();
    };
    auto drain = [&](int keep) {   // encode full tiles until at most `keep` remain
      if (npend > keep) {
        float fm[8][2];
#pragma unroll
        for (int q = 0; q < 16; ++q) fm[q >> 1][q & 1] = sFm[32 * q];
        while (npend > keep) {
          const int cnt = min(16, npend);
          front_encode(fm, sPendA_addr + 32u * (uint32_t)(npend - cnt), cnt, sW1f, sW2f, lane);
          npend -= cnt;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) sFm[32 * q] = fm[q >> 1][q & 1];
      }
      __syncwarp();
    };

    // the previous step's B-operand bits of this pad; this step's contact bits start clear
    uint32_t* btb = a.btbits + a.mask_woff[pad];
    for (int w = lane; w < nwords; w += 32) {
      sOld[w] = btb[w];
      sBits[w] = 0u;
    }
    __syncwarp();
    // nodes in blocks of 32 (Morton order of their positions), each with a bounding sphere:
    // the SDF is 1-Lipschitz, so a block whose centroid lies farther than its radius plus
    // twice the FP32 error bound from every object holds passive nodes only (exactly), and
    // its nodes skip the transform and the SDF.  Lane l tests blocks l, l + 32, ... up front,
    // so the tests' loads overlap; the loop reads the pad's block-ordered positions,
    // normals and node indices.
    const int nb = (n + 31) >> 5;
    const int16_t* bperm = a.blk_perm + o;
    const float* bpos = a.blk_pos + 3 * (size_t)o;
    const float* bnrm = a.blk_nrm + 3 * (size_t)o;
    const float4* bsph = a.blk_sphere + a.type_boff[ty];
    uint32_t cull[4] = {0u, 0u, 0u, 0u};   // blocks 32 w + l known passive (nb <= 128)
    if (!invalid && !a.mask_in) {
#pragma unroll
      for (int w4 = 0; w4 < 4; ++w4) {
        const int b = 32 * w4 + lane;
        bool out = false;
        if (b < nb) {
          const float4 sc = bsph[b];
          out = true;
          for (int k = 0; k < a.K; ++k) {
            const PadObj& ob = spo[k];
            if (ob.type == OBJ_NONE) continue;
            float3 q;
            q.x = fmaf(ob.R[0], sc.x, fmaf(ob.R[1], sc.y, fmaf(ob.R[2], sc.z, ob.t[0])));
            q.y = fmaf(ob.R[3], sc.x, fmaf(ob.R[4], sc.y, fmaf(ob.R[5], sc.z, ob.t[1])));
            q.z = fmaf(ob.R[6], sc.x, fmaf(ob.R[7], sc.y, fmaf(ob.R[8], sc.z, ob.t[2])));
            // a mesh reports +inf (outside, distance not computed) in cells known to be
            // outside: that proves nothing about the rest of the block
            const float ph = sdf_obj_f32<MESH>(ob, q);
            out &= ph != INFINITY && ph >= sc.w + 2.f * ob.tau;
          }
        }
        cull[w4] = __ballot_sync(FULL, out);
      }
    }
    // One step per iteration: a 32-node row (classification) or a batch of undecided nodes (the
    // exact path), then encoder tiles.  The encoder has this one call site, so its code exists
    // once (instruction fetch is the kernel's first stall); the order of rows, batches and tiles
    // is that of classifying every row with a batch whenever the queue nears full.
    auto row = [&](int r0) {
      const bool live = r0 + lane < n;
      const int i = live ? (int)bperm[r0 + lane] : 0;
      const int b = r0 >> 5;
      const uint32_t cw = b < 32 ? cull[0] : (b < 64 ? cull[1] : (b < 96 ? cull[2] : cull[3]));
      if (invalid || ((cw >> (b & 31)) & 1u)) {   // warp-uniform: the whole block is passive
        if (live) {
          NodeContact c;
          c.active = false;
          c.phi = 0.f;
          c.k = -1;
          c.u[0] = c.u[1] = c.u[2] = 0.f;
          front_write_node(a, btrow, n, base, i, c, (sOld[i >> 5] >> (i & 31)) & 1u);
        }
        return;
      }
      int cls = CONTACT_OUT;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      c.k = -1;
      c.u[0] = c.u[1] = c.u[2] = 0.f;
      float3 p = make_float3(0.f, 0.f, 0.f), nr = p;
      if (live) {
        const int s3 = 3 * (r0 + lane);
        p = make_float3(bpos[s3], bpos[s3 + 1], bpos[s3 + 2]);
        nr = make_float3(bnrm[s3], bnrm[s3 + 1], bnrm[s3 + 2]);
        if (a.mask_in) {   // mode B: the caller's contact is final (never in the band)
          c = contact_given(a.mask_in, a.uhat_in, base + i);
          cls = c.active ? CONTACT_FAST : CONTACT_OUT;
        } else {
          cls = contact_classify<MESH>(spo, a.K, p, nr, gap, &c);
        }
      }
      if (live && cls != CONTACT_BAND)
        front_write_node(a, btrow, n, base, i, c, (sOld[i >> 5] >> (i & 31)) & 1u);
      const unsigned bA = __ballot_sync(FULL, cls == CONTACT_FAST);
      const unsigned bC = __ballot_sync(FULL, cls == CONTACT_BAND);
      if (cls == CONTACT_FAST) atomicOr(&sBits[i >> 5], 1u << (i & 31));
      if (cls == CONTACT_FAST && enc) {
        const int q = npend + __popc(bA & lt);
        front_pack_row(sPendA + 2 * q, p, nr, c.u);
      }
      if (cls == CONTACT_BAND) sCand[ncand + __popc(bC & lt)] = (int16_t)i;
      m += __popc(bA);
      if (enc) npend += __popc(bA);
      ncand += __popc(bC);
      __syncwarp();
    };
    int r0 = 0;
    bool force = false;   // warp-uniform: the candidate queue is nearly full
    for (;;) {
      if (force || (r0 >= n && ncand > 0)) {
        refine_batch();
        force = false;
      } else if (r0 < n) {
        row(r0);
        r0 += 32;
        force = ncand > CANDCAP - 32;
      }
      const bool last = r0 >= n && ncand == 0;
      drain(last ? 0 : 15);
      if (last) break;
    }

    __syncwarp();
    for (int w = lane; w < nwords; w += 32) {
      if (!ETAC_IN(a.status, a.mask_woff[pad] + w, a.mask_words)) break;
      a.maskbits[a.mask_woff[pad] + w] = sBits[w];
      btb[w] = sBits[w];
    }
    if (lane == 0) {
      if (a.count && ETAC_IN(a.status, pad, a.num_items)) a.count[pad] = m;
      a.pad_m[pad] = m;
      if (invalid) latch_status(a.status, STATUS_NONFINITE);
    }
    if (m == 0) {   // no contact (or invalid pose): the whole pad is at rest
      float* d = a.disp + 3 * base;
      if (ETAC_IN(a.status, base + n - 1, a.num_nodes))
        for (int e = lane; e < 3 * n; e += 32) d[e] = 0.f;
      continue;
    }
    if (!enc) continue;

    // channel maxima of the active nodes: reduce over the tile rows (lane groups), then park
    // them in shared memory by channel
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float v = sFm[32 * (2 * nt + e)];
        v = fmaxf(v, __shfl_xor_sync(FULL, v, 4));
        v = fmaxf(v, __shfl_xor_sync(FULL, v, 8));
        v = fmaxf(v, __shfl_xor_sync(FULL, v, 16));
        if (lane < 4) sFmax[8 * nt + 2 * lane + e] = fmaxf(v + sB2[8 * nt + 2 * lane + e], 0.f);
      }
    __syncwarp();
    // max-pool over the passive nodes: the first passive node in each channel's descending
    // order of f0.  First step: lane l tests ranks 0..3 of channels l and l + 32, which settles
    // most channels.  Walks are long-tailed (the top of a channel's order can sit inside the
    // contact patch; on the hand workload 1 % of them pass rank 116), so the rest go
    // warp-wide: 2 channels per batch, 256 ranks per test (2 measured faster than 4: fewer
    // registers live across the test).
    {
      const float2* rk = a.ranked + (size_t)H * o;
      const float2* row0 = rk + (size_t)lane * n;
      const float2* row1 = rk + (size_t)(lane + 32) * n;
      float best0 = 0.f, best1 = 0.f;   // empty passive set: features are >= 0
      bool done0 = false, done1 = false;
      {
        float2 e0[4], e1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = j < n;
          e0[j] = in ? __ldg(row0 + j) : make_float2(0.f, __int_as_float(-1));
          e1[j] = in ? __ldg(row1 + j) : make_float2(0.f, __int_as_float(-1));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i0 = __float_as_int(e0[j].y), i1 = __float_as_int(e1[j].y);
          if (!done0 && i0 >= 0 && !((sBits[i0 >> 5] >> (i0 & 31)) & 1u)) {
            best0 = e0[j].x;
            done0 = true;
          }
          if (!done1 && i1 >= 0 && !((sBits[i1 >> 5] >> (i1 & 31)) & 1u)) {
            best1 = e1[j].x;
            done1 = true;
          }
        }
        if (n <= 4) done0 = done1 = true;
      }
      unsigned long long open = (unsigned long long)__ballot_sync(FULL, !done0) |
                                ((unsigned long long)__ballot_sync(FULL, !done1) << 32);
      // channels still open: the first passive node of each channel's descending order, up
      // to WB channels at a time; lane l tests ranks q0 + 8 l .. + 7 of the node-index order
      // (one 16-byte load per channel), so one test covers 256 ranks
      const int16_t* ord = a.order + (size_t)H * o;
      constexpr int WB = 2;
      while (open) {   // warp-uniform
        int ch[WB];
        bool dn[WB];
        float bv[WB];
#pragma unroll
        for (int c = 0; c < WB; ++c) {
          ch[c] = open ? __ffsll((long long)open) - 1 : -1;
          if (open) open &= open - 1;
          dn[c] = ch[c] < 0;
          bv[c] = 0.f;
        }
        for (int q0 = 0; q0 < n; q0 += 256) {
          const int r = q0 + 8 * lane;
          uint4 w[WB];
#pragma unroll
          for (int c = 0; c < WB; ++c)
            w[c] = (!dn[c] && r < n)
                       ? __ldg(reinterpret_cast<const uint4*>(ord + (size_t)ch[c] * n + r))
                       : make_uint4(0u, 0u, 0u, 0u);
          bool all = true;
#pragma unroll
          for (int c = 0; c < WB; ++c) {
            int cand = 0x7fffffff;
            if (!dn[c] && r < n) {
              const uint32_t wv[4] = {w[c].x, w[c].y, w[c].z, w[c].w};
#pragma unroll
              for (int j = 7; j >= 0; --j) {   // the lowest passive position wins
                const int idx = (int)((wv[j >> 1] >> (16 * (j & 1))) & 0xffffu);
                if (!((sBits[idx >> 5] >> (idx & 31)) & 1u)) cand = 8 * lane + j;
              }
            }
            const int first = __reduce_min_sync(FULL, cand);
            if (!dn[c] && first != 0x7fffffff) {
              bv[c] = __ldg(rk + (size_t)ch[c] * n + q0 + first).x;
              dn[c] = true;
            }
            all &= dn[c];
          }
          if (all) break;
        }
#pragma unroll
        for (int c = 0; c < WB; ++c) {
          if (ch[c] == lane) best0 = bv[c];
          if (ch[c] == lane + 32) best1 = bv[c];
        }
      }
      if (ETAC_IN(a.status, pad, a.num_items)) {
        a.g0a[(size_t)pad * H + lane] = fmaxf(best0, sFmax[lane]);
        a.g0a[(size_t)pad * H + lane + 32] = fmaxf(best1, sFmax[lane + 32]);
      }
    }
    __syncwarp();
  }
}

// one warp per pad (small batches, where 64-pad tiles would leave most SMs idle); G1 and D1's
// global half staged transposed so lanes read consecutive units
__global__ void __launch_bounds__(256) front_global_warp_kernel(FrontArgs a) {
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
    const int gi = a.pad_gi[pad];
    if (m == 0 || !uses_residual(a.mode)) {
      if (lane == 0) a.c0m[gi] = make_float4(0.f, 0.f, 0.f, __int_as_float(m));
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
      // -beta in BF16, words (channels 2w, 2w + 1) stored in MMA-fragment order: word
      // w = 8 s + 4 hh + t goes to position 8 t + 2 s + hh (see the propagation GEMM)
      __nv_bfloat16 nbv = __float2bfloat16_rn(-acc);
      const unsigned short mine = *reinterpret_cast<unsigned short*>(&nbv);
      const unsigned short odd = (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)mine, 1);
      if ((lane & 1) == 0) {
        const int w = u >> 1, s4 = w >> 3, hh = (w >> 2) & 1, t = w & 3;
        reinterpret_cast<uint32_t*>(a.negbeta)[(size_t)gi * 32 + 8 * t + 2 * s4 + hh] =
            (uint32_t)mine | ((uint32_t)odd << 16);
      }
    }
    float c0[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v = fmaf(sW4[q * H + lane], beta[0], sW4[q * H + 32 + lane] * beta[1]);
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      c0[q] = v + sB4[q];
    }
    if (lane == 0) a.c0m[gi] = make_float4(c0[0], c0[1], c0[2], __int_as_float(m));
  }
}

// 64 pads per CTA as two register-tiled products over shared memory: G = ReLU(G0 G1^T + b_G1)
// and B = G D1_g^T (rows: pads); thread (ti, tj) holds pads 4 ti .. + 3 x units 4 tj .. + 3.
// Then the per-pad epilogue records: -beta in BF16 (MMA-fragment word order) and
// (D2 beta + b_D2, m).
constexpr int FG_PADS = 64;
static_assert(FG_PADS == H, "the staging loops map pad rows like unit rows");

__global__ void __launch_bounds__(256) front_global_kernel(FrontArgs a) {
  __shared__ __align__(16) float sW[H * TLD];    // [k][u] = G1[u][k], then D1[u][64 + k]
  __shared__ __align__(16) float sX[H * TLD];    // [k][pad]: g0, then g
  __shared__ float sBg[H];
  __shared__ float sW4[3 * H];
  const float* W = a.params;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  const int p0 = blockIdx.x * FG_PADS;
  const int np = a.num_items;
  // every global load of the kernel is issued up front (G1, g0 and D1's global half, 16 of
  // each per thread), so their latencies overlap; D1 waits in registers until G1 is consumed
  constexpr int PER = H * H / 256;   // 16
  float wg[PER], xg[PER], wd[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = tid + 256 * t, u = e >> 6, k = e & (H - 1);
    const int r = e >> 6, pad = p0 + r;
    wg[t] = W[OFF_WG + u * H + k];
    xg[t] = pad < np ? a.g0a[(size_t)pad * H + k] : 0.f;
    wd[t] = W[OFF_WD + u * 2 * H + H + k];
  }
  for (int e = tid; e < H; e += 256) sBg[e] = W[OFF_BG + e];
  for (int e = tid; e < 3 * H; e += 256) sW4[e] = W[OFF_W4 + e];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = tid + 256 * t, u = e >> 6, k = e & (H - 1);
    sW[k * TLD + u] = wg[t];
    sX[k * TLD + u] = xg[t];   // u doubles as the pad row here (FG_PADS == H)
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = sBg[4 * tj + j];
  tile_acc(sX, sW, ti, tj, acc);
  __syncthreads();   // g0 and G1 are read; g and D1's global half take their places
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) sX[(4 * tj + j) * TLD + 4 * ti + i] = fmaxf(acc[i][j], 0.f);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int e = tid + 256 * t, u = e >> 6, k = e & (H - 1);
    sW[k * TLD + u] = wd[t];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;   // the D1 bias is part of the h0 table
  tile_acc(sX, sW, ti, tj, acc);
  const bool res = uses_residual(a.mode);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int pad = p0 + 4 * ti + i;
    const bool ok = pad < np;
    const int m = ok ? a.pad_m[pad] : 0;
    const int gi = ok ? a.pad_gi[pad] : 0;
    const bool live = ok && m > 0 && res;
    // -beta in BF16: words (channels 2w, 2w + 1), word w = 8 s + 4 hh + t at position
    // 8 t + 2 s + hh (the propagation GEMM's fragment order); this thread has w = 2 tj, 2 tj + 1
    if (live) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int w = 2 * tj + h, s4 = w >> 3, hh = (w >> 2) & 1, t = w & 3;
        __nv_bfloat162 v = __floats2bfloat162_rn(-acc[i][2 * h], -acc[i][2 * h + 1]);
        reinterpret_cast<uint32_t*>(a.negbeta)[(size_t)gi * 32 + 8 * t + 2 * s4 + hh] =
            *reinterpret_cast<uint32_t*>(&v);
      }
    }
    // c0 = D2 beta + b_D2: partial over this thread's 4 units, summed over the 16 threads of
    // the pad (a half warp)
    float c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) v = fmaf(sW4[q * H + 4 * tj + j], acc[i][j], v);
#pragma unroll
      for (int d = 8; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      c[q] = v + W[OFF_B4 + q];
    }
    if (ok && tj == 0)
      a.c0m[gi] = live ? make_float4(c[0], c[1], c[2], __int_as_float(m))
                       : make_float4(0.f, 0.f, 0.f, __int_as_float(m));
  }
}

}  // namespace

size_t front_smem_bytes(int nmax, int K) { return FrontSmem(nmax, K).total; }

cudaError_t front_occupancy(int nmax, int K, int* blocks_per_sm) {
  // both instantiations share the launch bounds (64 registers) and the shared memory
  const size_t smem = front_smem_bytes(nmax, K);
  cudaError_t e = cudaFuncSetAttribute(front_contact_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(front_contact_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, front_contact_kernel<false>,
                                                       FT, smem);
}

cudaError_t launch_front_contact(const FrontArgs& a, int grid, cudaStream_t s) {
  const size_t smem = front_smem_bytes(a.nmax, a.K);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(front_contact_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(front_contact_kernel<true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  if (a.num_meshes > 0)
    front_contact_kernel<true><<<grid, FT, smem, s>>>(a);
  else
    front_contact_kernel<false><<<grid, FT, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pad_obj(const FrontArgs& a, cudaStream_t s) {
  pad_obj_kernel<<<(unsigned)((a.num_items + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// tiles of 64 pads for batches of at least 64 pads per SM; one warp per pad below that
cudaError_t launch_front_global(const FrontArgs& a, int num_sms, cudaStream_t s) {
  if (a.num_items >= 64 * num_sms)
    front_global_kernel<<<(a.num_items + FG_PADS - 1) / FG_PADS, 256, 0, s>>>(a);
  else
    front_global_warp_kernel<<<std::max(1, std::min(4 * num_sms, (a.num_items + 7) / 8)), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace etac
