// prop_gemm.cu -- BF16 tensor-core propagation of the batched ETac step (tcgen05 + TMA + TMEM),
// with the residual decoder and Eq. 4 fused into the epilogue.
//
// Eq. 1 sums exp(-alpha |p_j - p_i|) u_hat_j over active nodes j; passive nodes carry
// u_hat = 0 (the same zero padding the residual network uses, Sec. III-A 2), so for all
// instances k of one pad type t the propagation is the dense contraction
//     L_t[i, (k, c)] = sum_j Omega_t[i, j] * Uhat[k, j, c],
// one GEMM with M = nodes i, K = nodes j, N = 3 x instances.  Omega_t is shared by every
// instance of the type and L2-resident; the B operand (u_hat in BF16) is written by the front
// kernel.  Accumulation is FP32 in tensor memory.
//
// Per CTA (persistent, one per SM): warp 16 issues TMA loads into a 3-stage shared-memory
// ring, warp 17 issues tcgen05.mma (M = 128, N = 192, K = 16) into one of two TMEM
// accumulators, warps 0-15 drain the other accumulator (four per TMEM lane quarter, 16
// instances each).  The epilogue evaluates, for every
// passive node i and instance k, the decoder residual
//     Phi = D2 ReLU(h0_i + beta_k) + b = D2 max(h0_i, -beta_k) + (D2 beta_k + b)
// with warp-level BF16 MMAs (m16n8k16) per instance, adds the propagated term and stores the
// displacement (Eq. 4).  h0 is held in registers in the MMA A-fragment layout, so the
// operand max(h0, -beta) is formed in registers (no shared-memory staging).  Every wait is bounded; a timeout latches ETAC_ERR_TIMEOUT and
// the CTA winds down (waiting, bounded, for its in-flight copies and MMAs before freeing TMEM).
#include <cuda_bf16.h>

#include <climits>

#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {
using namespace sm100;

namespace {

constexpr int GM = 128;                 // node rows per tile
constexpr int GK = 64;                  // nodes per K block (128 B of BF16)
constexpr int STAGES = 3;
constexpr int EPI_WARPS = 16;
constexpr int TMA_WARP = 16, MMA_WARP = 17;
constexpr int THREADS = 18 * 32;
constexpr int A_BYTES = GM * GK * 2;    // 16 KiB
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_STRIDE = 256;    // column offset of accumulator 1
constexpr int DEC = 2;                  // instances per decoder pass (independent MMA chains)

// Shapes and shared-memory layout (offsets from a 1024-byte aligned base) of a tile of GIT
// instances (N = 3 GIT accumulator columns).  Per-tile epilogue records are double-buffered
// (filled one tile ahead with cp.async): -beta (fragment order), (c0, m), node bases, contact
// words, h0 rows (16-byte chunks XOR-swizzled by row so fragment reads are conflict-free).
template <int GIT>
struct GemmShape {
  static constexpr int GI = GIT;
  static constexpr int GN = 3 * GI;
  static constexpr int B_BYTES = GN * GK * 2;
  static constexpr uint32_t IDESC = sm100::idesc_bf16_f32(GM, GN);
  static constexpr int INST_PER_WARP = GI / (EPI_WARPS / 4);
  static constexpr size_t SM_A = 0;
  static constexpr size_t SM_B = SM_A + (size_t)STAGES * A_BYTES;
  static constexpr size_t STG_NB = 0;                                  // GI x 64 BF16
  static constexpr size_t STG_C0 = STG_NB + (size_t)GI * H * 2;        // GI x float4
  static constexpr size_t STG_BASE = STG_C0 + (size_t)GI * 16;         // GI x int64
  static constexpr size_t STG_BITS = STG_BASE + (size_t)GI * 8;        // GI x 4 words
  static constexpr size_t STG_H0 = STG_BITS + (size_t)GI * 16;         // 128 rows x 128 B
  static constexpr size_t STG_BYTES = STG_H0 + (size_t)GM * 128;
  static constexpr size_t SM_R = SM_B + (size_t)STAGES * B_BYTES;      // EPI_WARPS x DEC x 32 x float4
  static constexpr size_t SM_STG = SM_R + (size_t)EPI_WARPS * DEC * 32 * 16;
  static constexpr size_t SM_BAR = SM_STG + 2 * STG_BYTES;
  static constexpr size_t SM_MISC = SM_BAR + 8 * (2 * STAGES + 6);
  static constexpr size_t SM_TOTAL = SM_MISC + 16;
  static constexpr size_t SM_ALLOC = SM_TOTAL + 1024;                  // alignment slack
  static_assert(STG_H0 % 128 == 0, "h0 staging rows must be 128-byte aligned");
  static_assert(SM_ALLOC <= 227 * 1024, "shared memory budget");
  static_assert(INST_PER_WARP % 4 == 0, "TMEM loads take four instances at a time");
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// MODE GEMM_FWD: the forward step above.  The reverse modes contract the same Omega_t-shaped
// tables with the passive nodes' dL/dU (B operand, split BF16 hi / lo, three K segments for
// FP32-level accuracy): GEMM_BWD_U adds sum_i Omega_ij G_i to dL/du_hat of every active node j;
// GEMM_BWD_ALPHA accumulates sum_j u_hat_j . sum_i d_ij Omega_ij G_i into per-CTA partials
// (dL/dalpha is minus their sum).
template <int MODE, int GIT>
__global__ void __launch_bounds__(THREADS, 1) prop_gemm_kernel(const __grid_constant__ GemmParams p) {
  constexpr int SEG = MODE == GEMM_FWD ? 1 : 3;
  using S = GemmShape<GIT>;
  constexpr int GI = S::GI;
  constexpr int B_BYTES = S::B_BYTES;
  constexpr uint32_t IDESC = S::IDESC;
  constexpr int INST_PER_WARP = S::INST_PER_WARP;
  constexpr size_t SM_A = S::SM_A, SM_B = S::SM_B, SM_R = S::SM_R, SM_STG = S::SM_STG,
                   SM_BAR = S::SM_BAR, SM_MISC = S::SM_MISC;
  constexpr size_t STG_NB = S::STG_NB, STG_C0 = S::STG_C0, STG_BASE = S::STG_BASE,
                   STG_BITS = S::STG_BITS, STG_H0 = S::STG_H0, STG_BYTES = S::STG_BYTES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SM_BAR);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + SM_MISC);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + SM_MISC + 4);
  volatile int* s_never = reinterpret_cast<volatile int*>(smem + SM_MISC + 8);      // stays 0
  // first epilogue tile (local index) at which a wait failed: INT_MAX while none has.  Every
  // epilogue warp compares it with its own tile after the tile's barrier, so a failure in a
  // later tile (written while a slow warp still reads) cannot make that warp leave early.
  int* s_epi_stop = reinterpret_cast<int*>(smem + SM_MISC + 12);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], EPI_WARPS);
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    *s_never = 0;
    *s_epi_stop = INT_MAX;
    fence_mbar_init();
  }
  if (warp == TMA_WARP && lane == 0) {
    for (int t = 0; t < GEMM_MAX_TYPES; ++t) {
      prefetch_tmap(&p.tmA[t]);
      prefetch_tmap(&p.tmB[t]);
      if (MODE != GEMM_FWD) {
        prefetch_tmap(&p.tmA2[t]);
        prefetch_tmap(&p.tmB2[t]);
      }
    }
  }
  if (warp == MMA_WARP) {
    tmem_alloc(s_tmem, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const uint64_t limit = p.timeout_ns;

  if (warp == TMA_WARP) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      bool withheld = false;
      for (int tile = blockIdx.x; tile < p.num_tiles && !*s_abort && !withheld;
           tile += gridDim.x) {
        const GemmTile T = p.tiles[tile];
        for (int kb = 0; kb < SEG * T.nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, s_abort, limit)) {
            *s_abort = 1;
            break;
          }
          if (p.test_withhold == tile + 1) {
            // failure-path test: this stage's loads are never issued and nothing more is
            // loaded; the copies issued before it are consumed (and so have landed) before the
            // MMA issuer reaches this stage and gives up on it
            withheld = true;
            break;
          }
          const int seg = kb / T.nkb, kk = kb - seg * T.nkb;
          const CUtensorMap* ta = seg == 2 ? &p.tmA2[T.type] : &p.tmA[T.type];
          const CUtensorMap* tb = seg == 1 ? &p.tmB2[T.type] : &p.tmB[T.type];
          mbar_expect_tx(&full[stage], A_BYTES + B_BYTES);
          tma_load_2d(smem + SM_A + (size_t)stage * A_BYTES, ta, kk * GK, T.m0, &full[stage]);
          tma_load_2d(smem + SM_B + (size_t)stage * B_BYTES, tb, kk * GK, 3 * T.k0, &full[stage]);
          ++issued;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (*s_abort) {
        // let the copies already issued land before shared memory goes away
        int st = stage;
        uint32_t ph = phase;
        for (int q = 0; q < STAGES && q < issued; ++q) {
          if (--st < 0) {
            st = STAGES - 1;
            ph ^= 1u;
          }
          mbar_wait(&full[st], ph, s_never, limit);
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int local = 0;
      bool any = false;
      for (int tile = blockIdx.x; tile < p.num_tiles && !*s_abort; tile += gridDim.x, ++local) {
        const GemmTile T = p.tiles[tile];
        const int b = local & 1;
        const uint32_t acc_phase = (uint32_t)(local >> 1) & 1u;
        if (!mbar_wait(&acc_empty[b], acc_phase ^ 1u, s_abort, limit)) {
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)b * ACC_STRIDE;
        bool ok = true;
        for (int kb = 0; kb < SEG * T.nkb; ++kb) {
          if (!mbar_wait(&full[stage], phase, s_abort, limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(smem + SM_A + (size_t)stage * A_BYTES);
          const uint32_t b_base = smem_u32(smem + SM_B + (size_t)stage * B_BYTES);
#pragma unroll
          for (int k = 0; k < GK / 16; ++k) {
            tc_mma_bf16(d_tmem, smem_desc_sw128(a_base + 32u * k), smem_desc_sw128(b_base + 32u * k),
                        IDESC, (kb | k) != 0 ? 1u : 0u);
          }
          any = true;
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) {
          *s_abort = 1;
          break;
        }
        tc_commit(&acc_full[b]);
      }
      if (any) {
        // every MMA issued by this thread has completed once the drain barrier flips
        tc_commit(drain);
        mbar_wait(drain, 0u, s_never, limit);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0-7)
    const int q = warp & 3, part = warp >> 2, etid = threadIdx.x;   // etid < 32 EPI_WARPS
    const int grp = lane >> 2, tig = lane & 3;
    float4* rbuf = reinterpret_cast<float4*>(smem + SM_R + (size_t)warp * DEC * 32 * 16);
    const float* W4 = p.params + OFF_W4;
    // decoder weights as constant B fragments: B[k = hidden][n = output component]
    uint32_t bw[4][2];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int k0 = 16 * s + 2 * tig;
      const bool live = grp < 3;
      bw[s][0] = live ? pack_bf16x2(W4[grp * H + k0], W4[grp * H + k0 + 1]) : 0u;
      bw[s][1] = live ? pack_bf16x2(W4[grp * H + k0 + 8], W4[grp * H + k0 + 9]) : 0u;
    }
    // issues the asynchronous copies of one tile's records into staging buffer sb
    auto stage = [&](const GemmTile& T, unsigned char* sb) {
      const int t = T.type;
      const int n_t = p.type_off[t + 1] - p.type_off[t];
      const int nw = (n_t + 31) >> 5;
      const int ninst = p.inst_off[t + 1] - p.inst_off[t];
      const int gi0 = p.inst_off[t] + T.k0;
      const uint32_t s0 = smem_u32(sb);
      for (int idx = etid; MODE == GEMM_FWD && idx < GI * 8; idx += EPI_WARPS * 32) {
        const int inst = idx >> 3, ch = idx & 7;
        const bool ok = T.k0 + inst < ninst;
        cp_async16(s0 + (uint32_t)(STG_NB + 16 * idx),
                   reinterpret_cast<const uint4*>(p.negbeta) + (size_t)(gi0 + (ok ? inst : 0)) * 8 + ch,
                   ok ? 16u : 0u);
      }
      for (int idx = etid; idx < GI; idx += EPI_WARPS * 32) {
        const bool ok = T.k0 + idx < ninst;
        const int g = gi0 + (ok ? idx : 0);
        if (MODE == GEMM_FWD) cp_async16(s0 + (uint32_t)(STG_C0 + 16 * idx), p.c0m + g, ok ? 16u : 0u);
        else cp_async4(s0 + (uint32_t)(STG_C0 + 16 * idx), p.inst_m + g, ok ? 4u : 0u);
        cp_async8(s0 + (uint32_t)(STG_BASE + 8 * idx), p.inst_base + g, ok ? 8u : 0u);
      }
      for (int idx = etid; idx < GI * 4; idx += EPI_WARPS * 32) {
        const int inst = idx >> 2, w = (T.m0 >> 5) + (idx & 3);
        const bool ok = T.k0 + inst < ninst && w < nw;
        const long long off = ok ? p.type_woff[t] + (long long)(T.k0 + inst) * nw + w : 0;
        cp_async4(s0 + (uint32_t)(STG_BITS + 4 * idx), p.maskbits + off, ok ? 4u : 0u);
      }
      for (int idx = etid; MODE == GEMM_FWD && idx < GM * 8; idx += EPI_WARPS * 32) {
        const int r = idx >> 3, ch = idx & 7, row = T.m0 + r;
        const bool ok = row < n_t;
        cp_async16(s0 + (uint32_t)(STG_H0 + 128 * r + ((ch ^ (r & 7)) << 4)),
                   reinterpret_cast<const uint4*>(p.h0bf16) + (size_t)(p.type_off[t] + (ok ? row : 0)) * 8 + ch,
                   ok ? 16u : 0u);
      }
      cp_async_commit();
    };
    if ((int)blockIdx.x < p.num_tiles) stage(p.tiles[blockIdx.x], smem + SM_STG);
    float alpha_acc = 0.f;   // GEMM_BWD_ALPHA: this thread's sum, tiles in order
    int local = 0;
    for (int tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x, ++local) {
      const GemmTile T = p.tiles[tile];
      const int b = local & 1;
      const uint32_t acc_phase = (uint32_t)(local >> 1) & 1u;
      const int t = T.type;
      const int n_t = p.type_off[t + 1] - p.type_off[t];
      unsigned char* sb = smem + SM_STG + (size_t)(local & 1) * STG_BYTES;
      // this tile's records have landed; every warp is done with the other buffer
      cp_async_wait_all();
      named_bar_sync(1, EPI_WARPS * 32);
      if (tile + (int)gridDim.x < p.num_tiles)
        stage(p.tiles[tile + gridDim.x], smem + SM_STG + (size_t)((local + 1) & 1) * STG_BYTES);
      const uint4* s_nb = reinterpret_cast<const uint4*>(sb + STG_NB);
      const float4* s_c0 = reinterpret_cast<const float4*>(sb + STG_C0);
      const long long* s_base = reinterpret_cast<const long long*>(sb + STG_BASE);
      const uint32_t* s_bits = reinterpret_cast<const uint32_t*>(sb + STG_BITS);
      // h0 of the warp's 32 rows in A-fragment layout: hf[rg][s][e] holds rows
      // 16 rg + grp (+ 8 for e = 1, 3), columns 16 s + 2 tig (+ 8 for e = 2, 3), BF16 pairs
      uint32_t hf[2][4][4];
#pragma unroll
      for (int rg = 0; rg < 2; ++rg)
#pragma unroll
        for (int e2 = 0; e2 < 2 && MODE == GEMM_FWD; ++e2) {
          const int r = 32 * q + 16 * rg + grp + 8 * e2;
          const unsigned char* hr = sb + STG_H0 + 128 * r + 4 * tig;
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) {
            hf[rg][s4][e2] = *reinterpret_cast<const uint32_t*>(hr + (((2 * s4) ^ (r & 7)) << 4));
            hf[rg][s4][2 + e2] =
                *reinterpret_cast<const uint32_t*>(hr + (((2 * s4 + 1) ^ (r & 7)) << 4));
          }
        }
      const int i = T.m0 + 32 * q + lane;   // my node row within the pad type
      const bool row_ok = i < n_t;
      if (!mbar_wait(&acc_full[b], acc_phase, s_abort, limit)) {
        *s_abort = 1;
        atomicMin(s_epi_stop, local);
      }
      // every epilogue warp takes the same decision (the flag is only written before here)
      named_bar_sync(2, EPI_WARPS * 32);
      if (*reinterpret_cast<volatile int*>(s_epi_stop) <= local) break;
      tc_fence_after();
      const uint32_t tbase = tmem + (uint32_t)b * ACC_STRIDE + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
      for (int g4 = 0; g4 < INST_PER_WARP / 4; ++g4) {
        // the propagated terms of four instances (columns 3 k .. 3 k + 11, k a multiple of 4)
        const int inst4 = INST_PER_WARP * part + 4 * g4;
        uint32_t lv4[12];
        {
          uint32_t r8[8], r4[4];
          tc_ld_32x32b_x8(tbase + 3u * inst4, r8);
          tc_ld_32x32b_x4(tbase + 3u * inst4 + 8u, r4);
          tc_wait_ld();
#pragma unroll
          for (int x = 0; x < 8; ++x) lv4[x] = r8[x];
#pragma unroll
          for (int x = 0; x < 4; ++x) lv4[8 + x] = r4[x];
        }
        if constexpr (MODE != GEMM_FWD) {
          // reverse modes: active rows of instances with contact
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            const int inst = inst4 + x;
            const int m = *reinterpret_cast<const int*>(s_c0 + inst);
            const bool act = ((s_bits[inst * 4 + q] >> lane) & 1u) != 0u;
            if (!(row_ok && act && m > 0)) continue;
            const float l0 = __uint_as_float(lv4[3 * x]), l1 = __uint_as_float(lv4[3 * x + 1]),
                        l2 = __uint_as_float(lv4[3 * x + 2]);
            const long long node = s_base[inst] + i;
            if (!ETAC_IN(p.status, node, p.num_nodes)) continue;
            if constexpr (MODE == GEMM_BWD_U) {
              float4 d = p.ws_du[node];
              d.x += l0;
              d.y += l1;
              d.z += l2;
              p.ws_du[node] = d;
            } else {
              const float4 u = p.ws_u[node];
              alpha_acc = fmaf(u.x, l0, fmaf(u.y, l1, fmaf(u.z, l2, alpha_acc)));
            }
          }
          continue;
        }
#pragma unroll
      for (int sub = 0; sub < 4 / DEC; ++sub) {
        const int inst0 = inst4 + DEC * sub;
        const uint32_t* lv = lv4 + 3 * DEC * sub;
        float4 r[DEC];
#pragma unroll
        for (int x = 0; x < DEC; ++x) r[x] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.use_r) {
          float acc[DEC][2][4];
#pragma unroll
          for (int x = 0; x < DEC; ++x)
#pragma unroll
            for (int rg = 0; rg < 2; ++rg)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[x][rg][e] = 0.f;
#pragma unroll
          for (int x = 0; x < DEC; ++x) {
            // -beta_k for this lane's columns: nb[2 s + h] = columns 16 s + 8 h + 2 tig, +1
            const uint4 n0 = s_nb[(inst0 + x) * 8 + 2 * tig], n1 = s_nb[(inst0 + x) * 8 + 2 * tig + 1];
            const uint32_t nb[8] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4)
#pragma unroll
              for (int rg = 0; rg < 2; ++rg) {
                uint32_t a[4];
                a[0] = bf16x2_max(hf[rg][s4][0], nb[2 * s4]);
                a[1] = bf16x2_max(hf[rg][s4][1], nb[2 * s4]);
                a[2] = bf16x2_max(hf[rg][s4][2], nb[2 * s4 + 1]);
                a[3] = bf16x2_max(hf[rg][s4][3], nb[2 * s4 + 1]);
                mma_bf16_16816(acc[x][rg], a, bw[s4][0], bw[s4][1], acc[x][rg]);
              }
          }
          // components 0..2 of the 16 x 8 results live in lanes tig 0 (0, 1) and 1 (2): pass
          // them to the lane that owns the node row
#pragma unroll
          for (int x = 0; x < DEC; ++x) {
            float* rb = reinterpret_cast<float*>(rbuf + x * 32);
#pragma unroll
            for (int rg = 0; rg < 2; ++rg) {
              const int r0 = rg * 16 + grp;
              if (tig == 0) {
                rb[r0 * 4 + 0] = acc[x][rg][0];
                rb[r0 * 4 + 1] = acc[x][rg][1];
                rb[(r0 + 8) * 4 + 0] = acc[x][rg][2];
                rb[(r0 + 8) * 4 + 1] = acc[x][rg][3];
              } else if (tig == 1) {
                rb[r0 * 4 + 2] = acc[x][rg][0];
                rb[(r0 + 8) * 4 + 2] = acc[x][rg][2];
              }
            }
          }
          __syncwarp();
#pragma unroll
          for (int x = 0; x < DEC; ++x) r[x] = rbuf[x * 32 + lane];
          __syncwarp();
        }
#pragma unroll
        for (int x = 0; x < DEC; ++x) {
          const int inst = inst0 + x;
          const float4 cm = s_c0[inst];
          const bool passive = ((s_bits[inst * 4 + q] >> lane) & 1u) == 0u;
          if (row_ok && passive && __float_as_int(cm.w) > 0) {
            float u0 = 0.f, u1 = 0.f, u2 = 0.f;
            if (p.use_l) {
              u0 = __uint_as_float(lv[3 * x + 0]);
              u1 = __uint_as_float(lv[3 * x + 1]);
              u2 = __uint_as_float(lv[3 * x + 2]);
            }
            if (p.use_r) {
              u0 += r[x].x + cm.x;
              u1 += r[x].y + cm.y;
              u2 += r[x].z + cm.z;
            }
            if (!ETAC_IN(p.status, s_base[inst] + i, p.num_nodes)) continue;
            float* d = p.disp + 3 * (s_base[inst] + i);
            d[0] = u0;
            d[1] = u1;
            d[2] = u2;
          }
        }
      }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
    cp_async_wait_all();   // no copy may still target shared memory when the CTA ends
    if constexpr (MODE == GEMM_BWD_ALPHA) {
      // fixed-order reduction of the epilogue threads' sums: lanes, then warps in order
      float* red = reinterpret_cast<float*>(smem + SM_R);
#pragma unroll
      for (int sh = 16; sh > 0; sh >>= 1) alpha_acc += __shfl_xor_sync(0xffffffffu, alpha_acc, sh);
      if (lane == 0) red[warp] = alpha_acc;
      named_bar_sync(1, EPI_WARPS * 32);
      if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < EPI_WARPS; ++w) t += red[w];
        p.alpha_part[blockIdx.x] = t;
      }
    }
  }

  __syncthreads();
  if (*s_abort && threadIdx.x == 0) latch_status(p.status, STATUS_TIMEOUT);
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace

size_t prop_gemm_smem_bytes() { return GemmShape<64>::SM_ALLOC; }

template <int MODE, int GIT>
cudaError_t launch_mode(const GemmParams& p, int grid, cudaStream_t s) {
  static bool configured = false;
  constexpr size_t smem = GemmShape<GIT>::SM_ALLOC;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(prop_gemm_kernel<MODE, GIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  prop_gemm_kernel<MODE, GIT><<<grid, THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_prop_gemm(const GemmParams& p, int grid, cudaStream_t s, int mode, int gi) {
  if (gi == 32) {
    if (mode == GEMM_BWD_U) return launch_mode<GEMM_BWD_U, 32>(p, grid, s);
    if (mode == GEMM_BWD_ALPHA) return launch_mode<GEMM_BWD_ALPHA, 32>(p, grid, s);
    return launch_mode<GEMM_FWD, 32>(p, grid, s);
  }
  if (gi == 80) {
    if (mode == GEMM_BWD_U) return launch_mode<GEMM_BWD_U, 80>(p, grid, s);
    if (mode == GEMM_BWD_ALPHA) return launch_mode<GEMM_BWD_ALPHA, 80>(p, grid, s);
    return launch_mode<GEMM_FWD, 80>(p, grid, s);
  }
  if (gi != 64) return cudaErrorInvalidValue;
  if (mode == GEMM_BWD_U) return launch_mode<GEMM_BWD_U, 64>(p, grid, s);
  if (mode == GEMM_BWD_ALPHA) return launch_mode<GEMM_BWD_ALPHA, 64>(p, grid, s);
  return launch_mode<GEMM_FWD, 64>(p, grid, s);
}

}  // namespace etac
