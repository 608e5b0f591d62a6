// regress_tc.cu -- real-to-sim taxel regressor (ETac appendix, "Modeling Real Sensors") on the
// tensor cores: tcgen05 MMAs with FP32 accumulators in tensor memory, weights streamed by bulk
// copies, activations held in shared memory from layer to layer.
//
// The per-node chain x_i = [p_i, n_i, U_i] -> h1 = relu(R1 x + b) (64) -> h2 = relu(R2 h1 + b)
// (128) -> h3 = relu(R3 h2 + b) (256) -> f = h3 + relu(R4 h3 + b) (256) -> a_i = A2 tanh(A1 f +
// b) + b is a sequence of dense contractions over 128-node tiles (M = 128 nodes, N = layer
// width, K = layer input), 280 kFLOP per node.  The softmax pooling g = sum_i alpha_i f_i and
// the head y = H2 relu(H1 g + b) + b run once per pad on the CUDA cores.
//
// Per CTA (persistent, one per SM) two slots, A and B, each run the chain on their own tiles;
// the MMA issuer alternates between them layer by layer, so one slot's epilogue overlaps the
// other slot's MMAs:
//   warp 16    streams the weight pieces (one block of 64 input channels of one layer, 8-32 KiB,
//              stored pre-swizzled in global memory) through a 3-stage ring of untiled bulk
//              copies;
//   warp 17    issues tcgen05.mma (M = 128, N = 64..256, K = 16) into the slot's 256 TMEM
//              columns (A: 0-255, B: 256-511);
//   warps 0-7  (slot A) and 8-15 (slot B) are the epilogues.  Warp w reads TMEM lanes
//              32 (w mod 4) .. + 31 (its 32 node rows) and one half of the layer's columns, adds
//              the bias, applies the activation, rounds to BF16 and writes the next layer's A
//              operand (128-byte swizzled K-major rows, the layout the MMA reads) into the slot's
//              64 KiB activation buffer, in place over the layer's input, whose MMAs are complete.
// The first layer takes x split into BF16 high and low parts ([x_hi, x_lo] against [R1, R1],
// K padded to 64), so the input enters at 2^-16 relative.  The residual layer re-reads h3 from
// the buffer.  The attention layer's epilogue applies tanh and forms the FP32 dot with A2; the two
// warps that hold one row's halves exchange their partial sums through two spare TMEM columns.
// Pooling is online (running maximum M, sum Z of exp(a - M), and exp-weighted feature sums,
// rescaled when M grows): each warp keeps the state of its 32 rows across every tile of the pad,
// four channels per lane, and the four row quarters merge at the end of the pad.
//
// Precision: BF16 operands (weights; activations h1, h2, h3, f), FP32 accumulation; the
// score, softmax, pooling and head are FP32.
//
// Every wait is bounded; a timeout latches ETAC_ERR_TIMEOUT, and the CTA winds down (all warps of
// an epilogue slot leave together, after the slot's barrier at the end of a tile; the MMA issuer
// and the copy warp wait, bounded, for their work in flight before tensor memory is freed).
#include <cuda_bf16.h>
#include <stdint.h>

#include <climits>

#include "etac_common.cuh"
#include "etac_kernels.h"
#include "sm100_ptx.cuh"

namespace etac {
using namespace sm100;

namespace {

constexpr int TM = 128;                 // node rows per tile
constexpr int NL = 5;                   // tensor-core layers: R1 R2 R3 R4 A1
constexpr int STAGES = 3;
constexpr int STAGE_BYTES = 32768;
constexpr int ACT_BYTES = 65536;        // 128 rows x 256 BF16
constexpr int KB_BYTES = 16384;         // one block of 64 BF16 columns, 128 rows
constexpr int PROD_WARP = 16, MMA_WARP = 17;
constexpr int THREADS = 18 * 32;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t SLOT_COLS = 256;
constexpr uint32_t XCH_COL = 254;       // score exchange (columns 254, 255; A1 uses 0-127)

// layer l: output width, input blocks of 64 channels, first weight piece
__host__ __device__ constexpr int lay_n(int l) { return l == 0 ? 64 : (l == 1 || l == 4) ? 128 : 256; }
__host__ __device__ constexpr int lay_nkb(int l) { return l <= 1 ? 1 : (l == 2 ? 2 : 4); }
__host__ __device__ constexpr int lay_piece(int l) {
  return l == 0 ? 0 : l == 1 ? 1 : l == 2 ? 2 : l == 3 ? 4 : 8;
}
constexpr int NPIECE = 12;
__host__ __device__ constexpr int piece_layer(int i) {
  return i < 1 ? 0 : i < 2 ? 1 : i < 4 ? 2 : i < 8 ? 3 : 4;
}
__host__ __device__ constexpr int piece_bytes(int i) { return lay_n(piece_layer(i)) * 128; }
__host__ __device__ constexpr int piece_off(int i) {
  int o = 0;
  for (int k = 0; k < i; ++k) o += piece_bytes(k);
  return o;
}
static_assert(piece_off(NPIECE) == REG_TC_IMAGE_BYTES, "weight image size");
static_assert(piece_bytes(2) <= STAGE_BYTES, "a weight piece fits one stage");

// shared memory, offsets from a 1024-byte aligned base
constexpr size_t SM_ACT = 0;
constexpr size_t SM_RING = SM_ACT + 2 * (size_t)ACT_BYTES;
constexpr size_t SM_BAR = SM_RING + (size_t)STAGES * STAGE_BYTES;   // full, empty, act, acc, drain
constexpr size_t SM_MISC = SM_BAR + 8 * (2 * STAGES + 5);
constexpr size_t SM_TOTAL = SM_MISC + 32;
constexpr size_t SM_ALLOC = SM_TOTAL + 1024;                       // alignment slack
static_assert(SM_ALLOC <= 227 * 1024, "shared memory budget");

// per-pad merge scratch (floats) in the slot's activation buffer, once the pad's tiles are done
constexpr int SC_M = 0, SC_Z = 4, SC_G = 8, SC_g = SC_G + 4 * 256, SC_z = SC_g + 256;

// byte offset of the 16-byte chunk holding columns 8 j .. 8 j + 7 of row r of a 64-column block
__device__ __forceinline__ uint32_t chunk_off(int r, int j) {
  return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ uint2 ld_shared_v2(uint32_t addr) {
  uint2 v;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Weight images: piece i is the [N rows x 64 input channels] block kb of layer l's W (row-major
// out x in), BF16, 128 bytes per row with the 16-byte chunks of row n at position chunk ^ (n & 7).
// Layer R1 (9 inputs) is stored as [R1, R1, 0]: columns 0-8 meet x_hi, 9-17 meet x_lo.
__global__ void regress_pack_kernel(const RegArgs a, unsigned char* img) {
  const int total = REG_TC_IMAGE_BYTES / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int i = 0;
    while (i + 1 < NPIECE && piece_off(i + 1) / 2 <= e) ++i;
    const int l = piece_layer(i), kb = i - lay_piece(l);
    const int local = e - piece_off(i) / 2;
    const int n = local >> 6, k = local & 63;
    float v;
    if (l == 0) {
      v = k < 9 ? a.W[0][n * 9 + k] : (k < 18 ? a.W[0][n * 9 + k - 9] : 0.f);
    } else {
      const int K = 64 * lay_nkb(l);
      v = a.W[l][(size_t)n * K + kb * 64 + k];
    }
    const uint32_t off = (uint32_t)piece_off(i) + chunk_off(n, k >> 3) + (uint32_t)(k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(img + off) = __float2bfloat16_rn(v);
  }
}

// Each epilogue thread keeps the biases of its column half in registers, lane-distributed:
// bias of column h * HALF + 32 x + lane of layer l in hb[hb_off(l) + x]; A2's weights of the
// half at hb_off(5).  A value reaches the lanes that need it by a warp shuffle.
__host__ __device__ constexpr int hb_off(int l) {
  return l == 0 ? 0 : l == 1 ? 1 : l == 2 ? 3 : l == 3 ? 7 : l == 4 ? 11 : 13;
}
constexpr int HB = 15;

// waits for this thread's tensor-memory loads; the registers of the last load are in-out
// operands, so no use of them is scheduled before the wait
__device__ __forceinline__ void tc_wait_ld_into(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Epilogue of layer L for one thread: node row r (TMEM lane), column half h, in chunks of 16
// columns with the next chunk's tensor-memory load in flight.  Layers 0-3 write the next A
// operand; layer 4 returns the partial attention score over its 64 columns.
template <int L>
__device__ __forceinline__ float epi_layer(const float (&hb)[HB], uint32_t trow, uint32_t act_u,
                                           int r, int h) {
  constexpr int HALF = lay_n(L) / 2, NCH = HALF / 16;
  const uint32_t tcol = trow + (uint32_t)(h * HALF);
  float part = 0.f;
  uint32_t v[2][16];
  tc_ld_32x32b_x16(tcol, v[0]);
  tc_wait_ld_into(v[0]);
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    if (ch + 1 < NCH) tc_ld_32x32b_x16(tcol + 16u * (ch + 1), v[(ch + 1) & 1]);
    const uint32_t* vv = v[ch & 1];
    float y[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = 16 * ch + i;   // column within the half
      y[i] = __uint_as_float(vv[i]) +
             __shfl_sync(0xffffffffu, hb[hb_off(L) + (k >> 5)], k & 31);
    }
    if constexpr (L == 4) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = 16 * ch + i;
        part = fmaf(__shfl_sync(0xffffffffu, hb[hb_off(5) + (k >> 5)], k & 31),
                    tanh_approx(y[i]), part);
      }
    } else {
      const int c = h * HALF + 16 * ch;
      const uint32_t blk = act_u + (uint32_t)(c >> 6) * KB_BYTES;
      const int j0 = (c & 63) >> 3;
#pragma unroll
      for (int i = 0; i < 16; ++i) y[i] = fmaxf(y[i], 0.f);
      if constexpr (L == 3) {
        // residual: f = h3 + relu(R4 h3 + b), h3 read back from the same place
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const uint4 h3 = ld_shared_v4(blk + chunk_off(r, j0 + cc));
          const uint32_t hw[4] = {h3.x, h3.y, h3.z, h3.w};
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            y[8 * cc + 2 * x] += bf_lo(hw[x]);
            y[8 * cc + 2 * x + 1] += bf_hi(hw[x]);
          }
        }
      }
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const float* z = y + 8 * cc;
        st_shared_v4(blk + chunk_off(r, j0 + cc), pack2(z[0], z[1]), pack2(z[2], z[3]),
                     pack2(z[4], z[5]), pack2(z[6], z[7]));
      }
    }
    if (ch + 1 < NCH) tc_wait_ld_into(v[(ch + 1) & 1]);
  }
  return part;
}

__global__ void __launch_bounds__(THREADS, 1) regress_tc_kernel(const __grid_constant__ RegTcArgs p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SM_BAR);
  uint64_t* empty = full + STAGES;
  uint64_t* act_ready = empty + STAGES;   // [2]: the slot's next A operand is in place
  uint64_t* acc_full = act_ready + 2;     // [2]: the slot's accumulator is complete
  uint64_t* drain = acc_full + 2;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + SM_MISC);
  volatile int* s_abort = reinterpret_cast<volatile int*>(smem + SM_MISC + 4);
  volatile int* s_never = reinterpret_cast<volatile int*>(smem + SM_MISC + 8);   // stays 0
  int* s_stop = reinterpret_cast<int*>(smem + SM_MISC + 12);   // [2]: first failed tile per slot
  const RegArgs& a = p.r;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&act_ready[s], 8);
      mbar_init(&acc_full[s], 1);
      s_stop[s] = INT_MAX;
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    *s_never = 0;
    fence_mbar_init();
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
  const int slot0 = 2 * blockIdx.x;
  const int ntile0 = p.slot_tiles[slot0], ntile1 = p.slot_tiles[slot0 + 1];
  const int jmax = ntile0 > ntile1 ? ntile0 : ntile1;

  if (warp == PROD_WARP) {
    // ---------------------------------------------------------------- weight pieces
    if (lane == 0) {
      int stage = 0, issued = 0;
      uint32_t phase = 0;
      bool stop = false;
      for (int j = 0; j < jmax && !stop; ++j)
        for (int l = 0; l < NL && !stop; ++l)
          for (int s = 0; s < 2 && !stop; ++s) {
            if (j >= (s ? ntile1 : ntile0)) continue;
            for (int kb = 0; kb < lay_nkb(l); ++kb) {
              if (!mbar_wait(&empty[stage], phase ^ 1u, s_abort, limit)) {
                *s_abort = 1;
                stop = true;
                break;
              }
              const int pc = lay_piece(l) + kb;
              const uint32_t bytes = (uint32_t)piece_bytes(pc);
              mbar_expect_tx(&full[stage], bytes);
              bulk_load(smem + SM_RING + (size_t)stage * STAGE_BYTES, p.wimg + piece_off(pc), bytes,
                        &full[stage]);
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
        for (int k = 0; k < STAGES && k < issued; ++k) {
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
      uint32_t phase = 0, actc0 = 0, actc1 = 0;
      bool any = false, stop = false;
      for (int j = 0; j < jmax && !stop; ++j)
        for (int l = 0; l < NL && !stop; ++l)
          for (int s = 0; s < 2 && !stop; ++s) {
            if (j >= (s ? ntile1 : ntile0)) continue;
            if (!mbar_wait(&act_ready[s], (s ? actc1 : actc0) & 1u, s_abort, limit)) {
              stop = true;
              break;
            }
            if (s) ++actc1;
            else ++actc0;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)s * SLOT_COLS;
            const uint32_t idesc = idesc_bf16_f32(TM, lay_n(l));
            const uint32_t a0 = smem_u32(smem + SM_ACT + (size_t)s * ACT_BYTES);
            for (int kb = 0; kb < lay_nkb(l); ++kb) {
              if (!mbar_wait(&full[stage], phase, s_abort, limit)) {
                stop = true;
                break;
              }
              tc_fence_after();
              const uint32_t b0 = smem_u32(smem + SM_RING + (size_t)stage * STAGE_BYTES);
#pragma unroll
              for (int k = 0; k < 4; ++k)
                tc_mma_bf16(d, smem_desc_sw128(a0 + (uint32_t)kb * KB_BYTES + 32u * k),
                            smem_desc_sw128(b0 + 32u * k), idesc, (kb | k) != 0 ? 1u : 0u);
              any = true;
              tc_commit(&empty[stage]);
              if (++stage == STAGES) {
                stage = 0;
                phase ^= 1u;
              }
            }
            if (stop) break;
            tc_commit(&acc_full[s]);
          }
      if (stop) *s_abort = 1;
      if (any) {
        // every MMA issued by this thread has completed once the drain barrier flips
        tc_commit(drain);
        mbar_wait(drain, 0u, s_never, limit);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogues
    const int s = warp >> 3, lw = warp & 7, q = warp & 3, h = lw >> 2;
    const int slot = slot0 + s;
    unsigned char* act = smem + SM_ACT + (size_t)s * ACT_BYTES;
    const uint32_t act_u = smem_u32(act);
    const uint32_t trow = tmem + (uint32_t)s * SLOT_COLS + ((uint32_t)(32 * q) << 16);
    const int r = 32 * q + lane;               // my node row within a tile
    const int bar_pair = 1 + 4 * s + q;        // the two warps of rows 32 q .. 32 q + 31
    const int bar_slot = 9 + s;
    float* sc = reinterpret_cast<float*>(act);
    float hb[HB];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int half = lay_n(l) / 2;
#pragma unroll
      for (int x = 0; x < half / 32; ++x) hb[hb_off(l) + x] = __ldg(a.b[l] + h * half + 32 * x + lane);
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) hb[hb_off(5) + x] = __ldg(a.W[5] + h * 64 + 32 * x + lane);
    uint32_t accc = 0;
    int round = 0;
    bool stopped = false;
    for (int pi = p.slot_off[slot]; pi < p.slot_off[slot + 1] && !stopped; ++pi) {
      const int pad = p.slot_pads[pi];
      const int t = a.pad_type[pad];
      const int t0 = a.type_off[t], n = a.type_off[t + 1] - t0;
      const long long base = a.pad_off[pad];
      float M = -INFINITY, Zl = 0.f, G0 = 0.f, G1 = 0.f, G2 = 0.f, G3 = 0.f;
      for (int j0 = 0; j0 < n; j0 += TM, ++round) {
        const int m = min(TM, n - j0);
        // ---- input rows [x_hi (9), x_lo (9), 0 ...]: warp half 0 writes columns 0-31, half 1
        // columns 32-63 (zeros)
        {
          uint32_t w[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) w[i] = 0u;
          if (h == 0 && r < m && ETAC_IN(p.status, base + j0 + r, a.num_nodes)) {
            const int node = t0 + j0 + r;
            const float* pp = a.type_pos + 3 * (size_t)node;
            const float* nn = a.type_nrm + 3 * (size_t)node;
            const float* uu = a.disp + 3 * (base + j0 + r);
            const float x[9] = {pp[0], pp[1], pp[2], nn[0], nn[1], nn[2], uu[0], uu[1], uu[2]};
            float v[18];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
              const __nv_bfloat16 hi = __float2bfloat16_rn(x[k]);
              v[k] = __bfloat162float(hi);
              v[9 + k] = x[k] - v[k];   // exact in FP32; rounded to BF16 below
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) w[k] = pack2(v[2 * k], v[2 * k + 1]);
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            st_shared_v4(act_u + chunk_off(r, 4 * h + cc), w[4 * cc], w[4 * cc + 1], w[4 * cc + 2],
                         w[4 * cc + 3]);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&act_ready[s]);
        // ---- the five layers
        float part = 0.f;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          if (!mbar_wait(&acc_full[s], accc & 1u, s_abort, limit)) {
            *s_abort = 1;
            atomicMin(&s_stop[s], round);
          }
          __syncwarp();
          ++accc;
          tc_fence_after();
          if (l == 0) epi_layer<0>(hb, trow, act_u, r, h);
          if (l == 1) epi_layer<1>(hb, trow, act_u, r, h);
          if (l == 2) epi_layer<2>(hb, trow, act_u, r, h);
          if (l == 3) epi_layer<3>(hb, trow, act_u, r, h);
          if (l == 4) part = epi_layer<4>(hb, trow, act_u, r, h);
          if (l < NL - 1) {
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&act_ready[s]);
          }
        }
        // ---- attention score: the two halves of row r meet through TMEM columns 254, 255
        tc_st_32x32b_x1(trow + XCH_COL + (uint32_t)h, __float_as_uint(part));
        tc_wait_st();
        tc_fence_before();
        named_bar_sync(bar_pair, 64);
        tc_fence_after();
        const float other = __uint_as_float(tc_ld_32x32b_x1(trow + XCH_COL + (uint32_t)(h ^ 1)));
        tc_wait_ld();
        const float score = (h == 0 ? part + other : other + part) + __ldg(a.b[5]);
        const bool valid = r < m;
        if (a.attn && h == 0 && valid && ETAC_IN(p.status, base + j0 + r, a.num_nodes))
          a.attn[base + j0 + r] = score;   // rescaled at pad end
        // ---- online softmax pooling over this warp's rows
        const int rows = min(32, m - 32 * q);
        if (rows > 0) {
          float wmax = valid ? score : -INFINITY;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
          const float Mn = fmaxf(M, wmax);
          const float scl = __expf(M - Mn);    // 0 while M = -inf
          Zl *= scl;
          G0 *= scl;
          G1 *= scl;
          G2 *= scl;
          G3 *= scl;
          M = Mn;
          const float e = valid ? __expf(score - M) : 0.f;
          Zl += e;
          // channels 128 h + 4 lane .. + 3: block 2 h + lane / 16, chunk (lane & 15) / 2
          const uint32_t cbase = act_u + (uint32_t)(2 * h + (lane >> 4)) * KB_BYTES +
                                 (uint32_t)(lane & 1) * 8u + (uint32_t)(32 * q) * 128u;
          const int jj = (lane & 15) >> 1;
#pragma unroll 4
          for (int i = 0; i < rows; ++i) {
            const float ei = __shfl_sync(0xffffffffu, e, i);
            const uint2 f2 = ld_shared_v2(cbase + (uint32_t)(i * 128 + ((jj ^ (i & 7)) << 4)));
            G0 = fmaf(ei, bf_lo(f2.x), G0);
            G1 = fmaf(ei, bf_hi(f2.x), G1);
            G2 = fmaf(ei, bf_lo(f2.y), G2);
            G3 = fmaf(ei, bf_hi(f2.y), G3);
          }
        }
        // the buffer is rewritten by the next tile's input rows only after every warp of the
        // slot is done with f; a failed wait anywhere in this tile stops the slot here
        __threadfence_block();
        named_bar_sync(bar_slot, 256);
        if (*reinterpret_cast<volatile int*>(&s_stop[s]) <= round) {
          stopped = true;
          break;
        }
      }
      if (stopped) break;
      // ---- merge the row quarters, then the head (FP32)
      float Z = Zl;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) Z += __shfl_xor_sync(0xffffffffu, Z, o);
      if (h == 0 && lane == 0) {
        sc[SC_M + q] = M;
        sc[SC_Z + q] = Z;
      }
      *reinterpret_cast<float4*>(sc + SC_G + q * 256 + 128 * h + 4 * lane) =
          make_float4(G0, G1, G2, G3);
      named_bar_sync(bar_slot, 256);
      const int c = lw * 32 + lane;
      float Mx = sc[SC_M];
#pragma unroll
      for (int k = 1; k < 4; ++k) Mx = fmaxf(Mx, sc[SC_M + k]);
      float Zt = 0.f, g = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float w = __expf(sc[SC_M + k] - Mx);
        Zt = fmaf(w, sc[SC_Z + k], Zt);
        g = fmaf(w, sc[SC_G + k * 256 + c], g);
      }
      sc[SC_g + c] = g / Zt;
      named_bar_sync(bar_slot, 256);
      {
        const float* H1 = a.W[6];
#pragma unroll 1
        for (int o = 16 * lw; o < 16 * lw + 16; ++o) {
          float acc = 0.f;
#pragma unroll
          for (int k = lane; k < 256; k += 32) acc = fmaf(__ldg(H1 + o * 256 + k), sc[SC_g + k], acc);
#pragma unroll
          for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sh);
          if (lane == 0) sc[SC_z + o] = fmaxf(acc + __ldg(a.b[6] + o), 0.f);
        }
      }
      named_bar_sync(bar_slot, 256);
      {
        const float* H2 = a.W[7];
        float acc = 0.f;
#pragma unroll
        for (int k = lane; k < 128; k += 32) acc = fmaf(__ldg(H2 + lw * 128 + k), sc[SC_z + k], acc);
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sh);
        if (lane == 0 && ETAC_IN(p.status, pad, a.num_pads))
          a.taxels[(size_t)pad * 8 + lw] = acc + __ldg(a.b[7] + lw);
      }
      if (a.attn && ETAC_IN(p.status, base + n - 1, a.num_nodes)) {
        const float invZ = 1.f / Zt;
        for (int i = c; i < n; i += 256) a.attn[base + i] = __expf(a.attn[base + i] - Mx) * invZ;
      }
      // the scratch is overwritten by the next pad's input rows
      named_bar_sync(bar_slot, 256);
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

size_t regress_tc_smem_bytes() { return SM_ALLOC; }

cudaError_t launch_regress_pack(const RegArgs& a, unsigned char* wimg, cudaStream_t s) {
  regress_pack_kernel<<<140, 256, 0, s>>>(a, wimg);
  return cudaGetLastError();
}

cudaError_t launch_regress_tc(const RegTcArgs& p, int grid, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(regress_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_ALLOC);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (grid <= 0) return cudaSuccess;
  regress_tc_kernel<<<grid, THREADS, SM_ALLOC, s>>>(p);
  return cudaGetLastError();
}

}  // namespace etac
