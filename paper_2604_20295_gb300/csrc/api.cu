// api.cu -- C ABI of libetac (declared in include/etac.h): validation, device buffers and
// the stream-ordered launch sequences.  Device memory is allocated by etac_create_pads and
// etac_set_model; etac_set_tuning and etac_autotune may grow the GEMM tile list and the
// reverse mode's work units for a new shape.  No step call (forward or reverse) allocates or
// synchronises the host.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <functional>
#include <queue>
#include <utility>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "etac.h"
#include "etac_common.cuh"
#include "etac_kernels.h"

struct etac_ctx {
  std::string err;
  int T = 0, E = 0, P = 0, K = 0, nmax = 0;
  int64_t N = 0;
  std::vector<int> type_n, type_off;
  std::vector<int> pad_type;
  std::vector<long long> pad_off;
  std::vector<float> type_pmax;
  // node blocks of every pad type for the BF16 front kernel's outside test
  std::vector<int16_t> blk_perm;     // [sum n] nodes in block order, type t at type_off[t]
  std::vector<float4> blk_sphere;    // [sum nb] block bounding spheres (centre, radius)
  std::vector<int> type_boff;        // [T] first block of each type
  int16_t* d_blk_perm = nullptr;
  float* d_blk_pos = nullptr;        // [sum n, 3] positions and normals in block order
  float* d_blk_nrm = nullptr;
  float4* d_blk_sphere = nullptr;
  int* d_type_boff = nullptr;
  // meshes of ETAC_OBJ_MESH objects (etac_set_meshes; the meshes themselves are borrowed)
  etac::MeshDev* d_meshes = nullptr;
  int num_meshes = 0, meshes_cap = 0;
  uint32_t* d_btbits = nullptr;      // nodes whose B-operand entries are nonzero (front kernel)
  // device geometry
  float* d_type_pos = nullptr;
  float* d_type_nrm = nullptr;
  float* d_type_pmax = nullptr;
  int* d_type_off = nullptr;
  int* d_pad_type = nullptr;
  long long* d_pad_off = nullptr;
  int* d_status = nullptr;
  // model
  bool has_model = false;
  etac_model_desc model{};
  float* d_params = nullptr;
  // state of the last forward (device copies of its inputs)
  bool has_forward = false;
  uint64_t step_id = 0;   // id of the last forward enqueued on this context (1, 2, ...)
  // mode B of the last forward: the caller's active set and u_hat (borrowed), else null
  const uint8_t* given_mask = nullptr;
  const float* given_uhat = nullptr;
  int* d_saved_obj_type = nullptr;
  float* d_saved_obj_dims = nullptr;
  float* d_saved_obj_pose = nullptr;
  float* d_saved_pad_pose = nullptr;
  int num_sms = 0;
  // batched algorithm: per-type tables, work queue
  std::vector<long long> omega_off;
  std::vector<int> item_pad;
  long long* d_omega_off = nullptr;
  int* d_item_pad = nullptr;
  int* d_ticket = nullptr;
  float* d_ctab = nullptr;
  float* d_f0tab = nullptr;
  float* d_h0tab = nullptr;
  int16_t* d_order = nullptr;
  float* d_omega = nullptr;
  // batched FP32: Omega from the per-type table, or on the fly (exp of the distance, in the
  // kernel) when the table would exceed kOmegaTableMaxBytes or the caller chose it
  bool omega_otf = false;
  int omega_pref = -1;   // etac_set_tuning: -1 no choice, 0 table, 1 on the fly
  void* d_omega_bf16 = nullptr;
  bool tables_ready = false;
  int batched_grid = 0;
  // BF16 tensor-core algorithm
  void* d_h0bf16 = nullptr;
  void* d_bt = nullptr;
  long long* d_bt_off = nullptr;
  int* d_pad_inst = nullptr;
  int* d_inst_off = nullptr;
  int* d_inst_pad = nullptr;
  void* d_negbeta = nullptr;
  float4* d_c0m = nullptr;
  uint32_t* d_maskbits = nullptr;
  long long* d_mask_woff = nullptr;
  int* d_pad_m = nullptr;
  float* d_g0a = nullptr;
  int* d_g0arg = nullptr;      // [E*P][64] maximising node of g0 (FP32 batched forward)
  bool fwd_recorded = false;   // the last forward recorded g0 / d_g0arg for the reverse
  float2* d_ranked = nullptr;
  etac::PadObj* d_padobj = nullptr;
  int* d_pad_bad = nullptr;
  int* d_pad_gi = nullptr;
  long long* d_inst_base = nullptr;
  long long* d_type_woff = nullptr;
  etac::GemmTile* d_tiles = nullptr;
  etac::GemmParams gemm{};
  int front_grid = 0, gemm_grid = 0, num_tiles = 0, tiles_cap = 0;
  int front_max_per_sm = 0;   // occupancy limit of the front kernel (CTAs per SM)
  long long mask_words = 0;   // contact-bit words of all pads (instance order)
  int gemm_gi = 64;      // instances per GEMM tile (tuned: 32, 64 or 80)
  int gemm_order = 0;    // GEMM tile order (tuned)
  int r3_range = 0;      // decoder-reverse node range (0: from the SM count; tuned)
  size_t r3g_cap = 0, spart_cap = 0, d2_cap = 0;
  bool bf16_ready = false, inst_ready = false;
  std::vector<long long> bt_off_h;
  std::vector<int> ninst_h;
  long long bt_total = 0;
  // staged batched reverse mode
  bool bwdb_ready = false;
  void* d_om_hi = nullptr;
  void* d_om_lo = nullptr;
  void* d_dom_hi = nullptr;
  void* d_dom_lo = nullptr;
  void* d_bg_hi = nullptr;
  void* d_bg_lo = nullptr;
  float* d_pr = nullptr;
  int* d_inst_m = nullptr;
  etac::R3Group* d_r3g = nullptr;
  float* d_a3part = nullptr;
  long long* d_a3_toff = nullptr;
  int* d_a3_tg = nullptr;
  float* d_a3 = nullptr;
  float* d_d2part = nullptr;
  float* d_r4part = nullptr;
  float* d_r4bpart = nullptr;
  float* d_r5part = nullptr;
  float* d_alpha_part = nullptr;
  float* d_gsum_part = nullptr;
  float* d_spart = nullptr;
  long long* d_s_toff = nullptr;
  int* d_s_nr = nullptr;
  int bwd_r1_grid = 0;
  int r3_parts = 0, r4_parts = 0, r4b_parts = 0, r5_parts = 0, alpha_parts = 0;
  etac::GemmParams gemm_bu{}, gemm_ba{};
  // profiling: event pairs around kernel launches
  // reverse mode workspace
  int* d_ws_idx = nullptr;
  float4* d_ws_u = nullptr;
  float4* d_ws_du = nullptr;
  float* d_pose_part = nullptr;
  float* d_param_part = nullptr;
  int bwd_grid = 0;
  // taxel regressor, tensor-core form: BF16 weight images and the slot schedule
  unsigned char* d_reg_wimg = nullptr;
  int* d_reg_sched = nullptr;        // [slots + 1] offsets | [E*P] pads | [slots] tile counts
  std::vector<int> reg_sched_h;
  int reg_grid = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev;       // 2 * ETAC_TIMING_SLOTS
  std::vector<int> ev_kernel;        // kernel id per used slot
  int ev_used = 0;
};

namespace {
const char* kKernelNames[] = {"plain_forward_kernel<float>", "batched_forward_kernel<fp32>",
                              "front_contact_kernel", "prop_gemm_kernel", "front_global_kernel",
                              "backward_kernel", "pad_obj_kernel", "bwd_pad_kernel",
                              "bwd_global_kernel", "bwd_decoder_kernel",
                              "bwd_padrev_kernel", "bwd_typenode_kernel",
                              "prop_gemm_kernel<bwd_u>", "prop_gemm_kernel<bwd_alpha>",
                              "bwd_pose_kernel(+param sums)", "bwd_reduce_a3_kernel",
                              "bwd_padsum_kernel", "regress_pack_kernel", "regress_tc_kernel",
                              "regress_plain_kernel"};
enum { K_PLAIN = 0, K_BATCHED = 1, K_FRONT = 2, K_GEMM = 3, K_GLOBAL = 4, K_BWD = 5, K_PADOBJ = 6,
       K_BWD_PAD = 7, K_BWD_GLOBAL = 8, K_BWD_DECODER = 9, K_BWD_PADREV = 10, K_BWD_TYPENODE = 11,
       K_BWD_GEMM_U = 12, K_BWD_GEMM_A = 13, K_BWD_POSE = 14, K_BWD_A3SUM = 15,
       K_BWD_PADSUM = 16, K_REG_PACK = 17, K_REG_TC = 18, K_REG_PLAIN = 19, K_COUNT = 20 };

// records the start event of a timed launch; returns the slot or -1
int timing_begin(etac_ctx* c, int kernel, cudaStream_t s) {
  nvtxRangePushA(kKernelNames[kernel]);
  if (!c->timing || c->ev_used >= ETAC_TIMING_SLOTS) return -1;
  const int slot = c->ev_used++;
  c->ev_kernel[slot] = kernel;
  cudaEventRecord(c->ev[2 * slot], s);
  return slot;
}
void timing_end(etac_ctx* c, int slot, cudaStream_t s) {
  if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], s);
  nvtxRangePop();
}

// An API call as a named NVTX range (nested around its launches' ranges).
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

// One kernel launch as a named region: an NVTX range with the kernel's name (seen by a
// profiler that attaches an NVTX tool, a no-op otherwise) and, while timing is on, a CUDA event
// pair on the launch stream.  Scoped, so an early error return still closes both.
class TimedLaunch {
 public:
  TimedLaunch(etac_ctx* c, int kernel, cudaStream_t s)
      : c_(c), s_(s), slot_(timing_begin(c, kernel, s)) {}
  ~TimedLaunch() { timing_end(c_, slot_, s_); }
  TimedLaunch(const TimedLaunch&) = delete;
  TimedLaunch& operator=(const TimedLaunch&) = delete;

 private:
  etac_ctx* c_;
  cudaStream_t s_;
  int slot_;
};
}  // namespace

namespace {

thread_local std::string g_create_err;

etac_status fail(etac_ctx* c, etac_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_err = buf;
  return s;
}

etac_status cuda_fail(etac_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? ETAC_ERR_OOM : ETAC_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define ETAC_CUDA(ctx, expr, what)                       \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

template <typename X>
cudaError_t dalloc(X** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(1, count) * sizeof(X));
}

void free_ctx(etac_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  void* ptrs[] = {c->d_type_pos, c->d_type_nrm, c->d_type_pmax, c->d_type_off, c->d_pad_type,
                  c->d_pad_off, c->d_status, c->d_params, c->d_saved_obj_type,
                  c->d_saved_obj_dims, c->d_saved_obj_pose, c->d_saved_pad_pose,
                  c->d_omega_off, c->d_item_pad, c->d_ticket, c->d_ctab, c->d_f0tab,
                  c->d_h0tab, c->d_order, c->d_omega, c->d_omega_bf16, c->d_h0bf16, c->d_bt,
                  c->d_bt_off, c->d_pad_inst, c->d_inst_off, c->d_inst_pad, c->d_negbeta,
                  c->d_c0m, c->d_tiles, c->d_maskbits, c->d_mask_woff, c->d_pad_m,
                  c->d_g0a, c->d_ranked, c->d_padobj, c->d_pad_bad, c->d_pad_gi, c->d_inst_base,
                  c->d_type_woff, c->d_om_hi, c->d_om_lo, c->d_dom_hi, c->d_dom_lo,
                  c->d_bg_hi, c->d_bg_lo, c->d_pr, c->d_inst_m, c->d_r3g, c->d_a3part,
                  c->d_a3_toff, c->d_a3_tg, c->d_a3, c->d_d2part, c->d_r4part, c->d_r4bpart,
                  c->d_r5part, c->d_alpha_part, c->d_gsum_part, c->d_spart, c->d_s_toff,
                  c->d_s_nr, c->d_ws_idx, c->d_ws_u,
                  c->d_ws_du, c->d_pose_part, c->d_param_part, c->d_g0arg,
                  c->d_blk_perm, c->d_blk_sphere, c->d_type_boff, c->d_btbits,
                  c->d_blk_pos, c->d_blk_nrm, c->d_meshes, c->d_reg_wimg, c->d_reg_sched};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

// Node blocks of one pad type for the front kernel's outside test: the nodes in Morton order
// of their pad-frame positions (10 bits per axis over the type's bounding box, ties by node
// index), 32 per block, each block with the centroid of its nodes and the largest distance
// of a node from it, rounded up.  On a grid the blocks are 4 x 8 or 8 x 4 patches.
void build_blocks(const float* pos, int n, int16_t* perm, std::vector<float4>& sph) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = 0; i < n; ++i)
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], (double)pos[3 * i + q]);
      hi[q] = std::max(hi[q], (double)pos[3 * i + q]);
    }
  std::vector<std::pair<uint64_t, int>> key(n);
  for (int i = 0; i < n; ++i) {
    uint64_t code = 0;
    uint32_t g[3];
    for (int q = 0; q < 3; ++q) {
      const double span = hi[q] - lo[q];
      g[q] = span > 0 ? (uint32_t)std::min(1023.0, std::floor((pos[3 * i + q] - lo[q]) / span * 1023.0 + 0.5)) : 0u;
    }
    for (int bit = 9; bit >= 0; --bit)
      for (int q = 0; q < 3; ++q) code = (code << 1) | ((g[q] >> bit) & 1u);
    key[i] = {code, i};
  }
  std::sort(key.begin(), key.end());
  for (int i = 0; i < n; ++i) perm[i] = (int16_t)key[i].second;
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int b1 = std::min(n, b0 + 32);
    double c[3] = {0, 0, 0};
    for (int s = b0; s < b1; ++s)
      for (int q = 0; q < 3; ++q) c[q] += pos[3 * perm[s] + q];
    float cf[3];
    for (int q = 0; q < 3; ++q) cf[q] = (float)(c[q] / (b1 - b0));
    double r = 0.0;
    for (int s = b0; s < b1; ++s) {
      double d2 = 0.0;
      for (int q = 0; q < 3; ++q) {
        const double d = (double)pos[3 * perm[s] + q] - (double)cf[q];
        d2 += d * d;
      }
      r = std::max(r, std::sqrt(d2));
    }
    sph.push_back(make_float4(cf[0], cf[1], cf[2], std::nextafter((float)r, INFINITY) + 1e-6f));
  }
}

bool valid_model(const etac_model_desc* d) {
  return d && d->hidden == ETAC_HIDDEN && d->mode >= ETAC_MODE_FULL &&
         d->mode <= ETAC_MODE_PENETRATION_ONLY && (d->precision == ETAC_PREC_FP32 ||
         d->precision == ETAC_PREC_BF16) && (d->algo == ETAC_ALGO_PLAIN ||
         d->algo == ETAC_ALGO_BATCHED);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2-D BF16 tensor [rows][cols] (cols contiguous), box of 64 columns x box_rows rows, 128B swizzle
bool encode_bf16_2d(EncodeTiledFn fn, CUtensorMap* m, const void* base, uint64_t cols,
                    uint64_t rows, uint32_t box_rows) {
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void fill_gemm_common(etac_ctx* c, etac::GemmParams& g);

// GEMM tile list for the current tile shape (instances per tile) and order: heaviest tiles
// first; order 0 walks node-row tiles innermost, so the CTAs working at one time share each B
// tile through L2; order 1 walks instance groups innermost, sharing each Omega row block
etac_status build_tiles(etac_ctx* c, cudaStream_t s) {
  const int gi = c->gemm_gi;
  std::vector<etac::GemmTile> tiles;
  for (int t = 0; t < c->T; ++t) {
    if (!c->ninst_h[t]) continue;
    const int n = c->type_n[t];
    if (c->gemm_order == 0) {
      for (int k0 = 0; k0 < c->ninst_h[t]; k0 += gi)
        for (int m0 = 0; m0 < n; m0 += 128) tiles.push_back({t, m0, k0, (n + 63) / 64});
    } else {
      for (int m0 = 0; m0 < n; m0 += 128)
        for (int k0 = 0; k0 < c->ninst_h[t]; k0 += gi) tiles.push_back({t, m0, k0, (n + 63) / 64});
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](const etac::GemmTile& x,
                                                  const etac::GemmTile& y) {
    return x.nkb > y.nkb;
  });
  cudaError_t e = cudaSuccess;
  if ((int)tiles.size() > c->tiles_cap) {
    if (c->d_tiles) cudaFree(c->d_tiles);
    c->d_tiles = nullptr;
    e = dalloc(&c->d_tiles, tiles.size());
    if (e != cudaSuccess) return cuda_fail(c, e, "GEMM tile list");
    c->tiles_cap = (int)tiles.size();
  }
  if (!tiles.empty())
    e = cudaMemcpyAsync(c->d_tiles, tiles.data(), sizeof(etac::GemmTile) * tiles.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "GEMM tile list");
  c->num_tiles = (int)tiles.size();
  c->gemm_grid = std::max(1, std::min(c->num_sms, c->num_tiles));
  for (etac::GemmParams* g : {&c->gemm, &c->gemm_bu, &c->gemm_ba}) {
    g->tiles = c->d_tiles;
    g->num_tiles = c->num_tiles;
  }
  c->alpha_parts = c->gemm_grid;
  return ETAC_OK;
}

// Instance bookkeeping shared by the tensor-core forward and the batched reverse mode (once
// per context): instance order per pad type, per-instance records' indices, contact bit words
// in instance order, the GEMM tile list, per-pad transform buffers.
etac_status setup_instances(etac_ctx* c, cudaStream_t s) {
  if (c->inst_ready) return ETAC_OK;
  const int np = c->E * c->P;
  std::vector<int> inst_off(c->T + 1, 0), pad_inst(np), ninst(c->T, 0);
  for (int p = 0; p < np; ++p) pad_inst[p] = ninst[c->pad_type[p]]++;
  for (int t = 0; t < c->T; ++t) inst_off[t + 1] = inst_off[t] + ninst[t];
  std::vector<int> inst_pad(np), fill(c->T, 0);
  for (int p = 0; p < np; ++p) {
    const int t = c->pad_type[p];
    inst_pad[inst_off[t] + fill[t]++] = p;
  }
  // contact bit words in instance order: type t's instances one after another, so a GEMM tile
  // finds its rows' words at computable addresses; by-instance record indices for the same
  std::vector<long long> type_woff(c->T, 0), woff(np + 1, 0), inst_base(np);
  std::vector<int> pad_gi(np);
  long long wtot = 0;
  for (int t = 0; t < c->T; ++t) {
    type_woff[t] = wtot;
    wtot += (long long)ninst[t] * ((c->type_n[t] + 31) / 32);
  }
  for (int p = 0; p < np; ++p) {
    const int t = c->pad_type[p];
    woff[p] = type_woff[t] + (long long)pad_inst[p] * ((c->type_n[t] + 31) / 32);
    pad_gi[p] = inst_off[t] + pad_inst[p];
    inst_base[pad_gi[p]] = c->pad_off[p];
  }
  woff[np] = wtot;
  c->bt_off_h.assign(c->T, 0);
  long long bt_total = 0;
  for (int t = 0; t < c->T; ++t) {
    c->bt_off_h[t] = bt_total;
    bt_total += ((3LL * ninst[t] * c->type_n[t]) + 127) / 128 * 128;
  }
  c->bt_total = bt_total;
  c->ninst_h = ninst;
  cudaError_t e = dalloc(&c->d_bt_off, c->T);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_inst, np);
  if (e == cudaSuccess) e = dalloc(&c->d_inst_off, c->T + 1);
  if (e == cudaSuccess) e = dalloc(&c->d_inst_pad, np);
  if (e == cudaSuccess) e = dalloc(&c->d_maskbits, (size_t)woff[np]);
  c->mask_words = woff[np];
  if (e == cudaSuccess) e = dalloc(&c->d_mask_woff, (size_t)np + 1);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_m, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->d_padobj, (size_t)np * c->K);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_bad, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_gi, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->d_inst_base, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->d_type_woff, (size_t)c->T);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_pad_gi, pad_gi.data(), sizeof(int) * np,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_inst_base, inst_base.data(),
                                            sizeof(long long) * np, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_type_woff, type_woff.data(),
                                            sizeof(long long) * c->T, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_mask_woff, woff.data(), sizeof(long long) * (np + 1),
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_bt_off, c->bt_off_h.data(),
                                            sizeof(long long) * c->T, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_pad_inst, pad_inst.data(), sizeof(int) * np,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_inst_off, inst_off.data(),
                                            sizeof(int) * (c->T + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_inst_pad, inst_pad.data(), sizeof(int) * np,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors are pageable
  if (e != cudaSuccess) return cuda_fail(c, e, "instance buffers");
  c->inst_ready = true;
  return build_tiles(c, s);
}

bool tensor_core_shapes_ok(const etac_ctx* c) {
  if (c->T > etac::GEMM_MAX_TYPES) return false;
  for (int t = 0; t < c->T; ++t)
    if (c->type_n[t] % 8 != 0) return false;
  return true;
}

EncodeTiledFn get_encode_fn() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &qr);
  if (e != cudaSuccess || !fn || qr != cudaDriverEntryPointSuccess) return nullptr;
  return reinterpret_cast<EncodeTiledFn>(fn);
}

// common GEMM fields (tile list, per-instance records) of a parameter block
void fill_gemm_common(etac_ctx* c, etac::GemmParams& g) {
  g.tiles = c->d_tiles;
  g.num_tiles = c->num_tiles;
  g.type_off = c->d_type_off;
  g.inst_off = c->d_inst_off;
  g.inst_pad = c->d_inst_pad;
  g.pad_off = c->d_pad_off;
  g.inst_base = c->d_inst_base;
  g.type_woff = c->d_type_woff;
  g.maskbits = c->d_maskbits;
  g.params = c->d_params;
  g.status = c->d_status;
  g.num_nodes = c->N;
  g.timeout_ns = 2000000000ull;   // 2 s per wait: far beyond any legitimate stall
  g.test_withhold = 0;
}

// B-operand tensor map of the forward GEMM carries the tile shape (box rows = 3 x instances)
etac_status encode_fwd_maps(etac_ctx* c) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn) return fail(c, ETAC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  etac::GemmParams& g = c->gemm;
  for (int t = 0; t < c->T; ++t) {
    const int n = c->type_n[t];
    const char* om = reinterpret_cast<const char*>(c->d_omega_bf16) + 2 * (size_t)c->omega_off[t];
    const char* bt = reinterpret_cast<const char*>(c->d_bt) + 2 * (size_t)c->bt_off_h[t];
    if (!encode_bf16_2d(fn, &g.tmA[t], om, n, n, 128) ||
        !encode_bf16_2d(fn, &g.tmB[t], bt, n, std::max(1, 3 * c->ninst_h[t]), 3 * c->gemm_gi))
      return fail(c, ETAC_ERR_CUDA, "tensor map encoding failed for pad type %d", t);
  }
  return ETAC_OK;
}

// Buffers and tensor maps of the BF16 tensor-core forward (once per context).
etac_status setup_bf16(etac_ctx* c, cudaStream_t s) {
  if (c->bf16_ready) return ETAC_OK;
  if (c->T > etac::GEMM_MAX_TYPES)
    return fail(c, ETAC_ERR_UNSUPPORTED, "BF16 algorithm supports at most %d pad types",
                etac::GEMM_MAX_TYPES);
  for (int t = 0; t < c->T; ++t)
    if (c->type_n[t] % 8 != 0)
      return fail(c, ETAC_ERR_UNSUPPORTED,
                  "BF16 algorithm needs node counts that are multiples of 8 (type %d has %d)", t,
                  c->type_n[t]);
  etac_status st = setup_instances(c, s);
  if (st != ETAC_OK) return st;
  const int np = c->E * c->P;
  const size_t tn = (size_t)c->type_off[c->T];
  cudaError_t e = dalloc(reinterpret_cast<char**>(&c->d_omega_bf16), 2 * (size_t)c->omega_off[c->T]);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_h0bf16), 2 * tn * etac::H);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_bt), 2 * (size_t)c->bt_total);
  // the front kernel rewrites only the B-operand entries of nodes that are or were active,
  // so both start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bt, 0, 2 * (size_t)c->bt_total, s);
  if (e == cudaSuccess) e = dalloc(&c->d_btbits, (size_t)c->mask_words);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_btbits, 0, sizeof(uint32_t) * c->mask_words, s);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_negbeta), 2 * (size_t)np * etac::H);
  if (e == cudaSuccess) e = dalloc(&c->d_c0m, np);
  if (e == cudaSuccess && !c->d_g0a) e = dalloc(&c->d_g0a, (size_t)np * etac::H);
  if (e != cudaSuccess) return cuda_fail(c, e, "BF16 buffers");
  etac::GemmParams& g = c->gemm;
  memset(&g, 0, sizeof g);
  if ((st = encode_fwd_maps(c)) != ETAC_OK) return st;
  fill_gemm_common(c, g);
  g.h0bf16 = c->d_h0bf16;
  g.negbeta = c->d_negbeta;
  g.c0m = c->d_c0m;
  int per_sm = 0;
  e = etac::front_occupancy(c->nmax, c->K, &per_sm);
  if (e != cudaSuccess || per_sm < 1) return cuda_fail(c, e, "front kernel occupancy");
  c->front_grid = per_sm * c->num_sms;
  c->front_max_per_sm = per_sm;
  c->bf16_ready = true;
  return ETAC_OK;
}

// B-operand tensor maps of the reverse-mode GEMMs (box rows = 3 x instances per tile)
etac_status encode_bwd_maps(etac_ctx* c) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn) return fail(c, ETAC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  for (int which = 0; which < 2; ++which) {
    etac::GemmParams& g = which == 0 ? c->gemm_bu : c->gemm_ba;
    const char* ah = reinterpret_cast<const char*>(which == 0 ? c->d_om_hi : c->d_dom_hi);
    const char* al = reinterpret_cast<const char*>(which == 0 ? c->d_om_lo : c->d_dom_lo);
    for (int t = 0; t < c->T; ++t) {
      const int n = c->type_n[t];
      const size_t oo = 2 * (size_t)c->omega_off[t], bo = 2 * (size_t)c->bt_off_h[t];
      const uint64_t rows = std::max(1, 3 * c->ninst_h[t]);
      const uint32_t box = 3 * c->gemm_gi;
      if (!encode_bf16_2d(fn, &g.tmA[t], ah + oo, n, n, 128) ||
          !encode_bf16_2d(fn, &g.tmA2[t], al + oo, n, n, 128) ||
          !encode_bf16_2d(fn, &g.tmB[t], reinterpret_cast<const char*>(c->d_bg_hi) + bo, n, rows, box) ||
          !encode_bf16_2d(fn, &g.tmB2[t], reinterpret_cast<const char*>(c->d_bg_lo) + bo, n, rows, box))
        return fail(c, ETAC_ERR_CUDA, "tensor map encoding failed for pad type %d", t);
    }
  }
  return ETAC_OK;
}

// Decoder-reverse work units: (pad type, 64-instance group, node range).  range 0 picks 256
// nodes, halved (down to 16) until there are at least four units per SM.
etac_status build_r3(etac_ctx* c, int range, cudaStream_t s) {
  std::vector<long long> a3_toff(c->T, 0);
  std::vector<int> a3_tg(c->T, 0);
  long long a3tot = 0;
  for (int t = 0; t < c->T; ++t) {
    a3_toff[t] = a3tot;
    a3_tg[t] = (c->ninst_h[t] + 63) / 64;
    a3tot += (long long)a3_tg[t] * c->type_n[t] * etac::H;
  }
  auto units = [&](int rg) {
    long long u = 0;
    for (int t = 0; t < c->T; ++t) u += (long long)a3_tg[t] * ((c->type_n[t] + rg - 1) / rg);
    return u;
  };
  if (range <= 0) {
    range = etac::R3_RANGE;
    while (range > 16 && units(range) < 4LL * c->num_sms) range /= 2;
  }
  if (range % 16 != 0 || range < 16 || range > etac::R3_RANGE)
    return fail(c, ETAC_ERR_INVALID_ARG, "decoder-reverse node range must be 16..256 in steps of 16");
  std::vector<long long> s_toff(c->T, 0);
  std::vector<int> s_nr(c->T, 0);
  long long stot = 0;
  for (int t = 0; t < c->T; ++t) {
    s_toff[t] = stot;
    s_nr[t] = (c->type_n[t] + range - 1) / range;
    stot += (long long)s_nr[t] * c->ninst_h[t];
  }
  std::vector<etac::R3Group> groups;
  for (int t = 0; t < c->T; ++t)
    for (int g = 0; g < a3_tg[t]; ++g)
      for (int r = 0; r < s_nr[t]; ++r)
        groups.push_back({t, 64 * g, r * range, std::min(c->type_n[t], (r + 1) * range), r,
                          a3_toff[t] + (long long)g * c->type_n[t] * etac::H});
  std::stable_sort(groups.begin(), groups.end(), [](const etac::R3Group& x, const etac::R3Group& y) {
    return x.i1 - x.i0 > y.i1 - y.i0;   // largest units first
  });
  cudaError_t e = cudaSuccess;
  auto grow = [&](auto** ptr, size_t& cap, size_t need) {
    if (e != cudaSuccess || need <= cap) return;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    e = dalloc(ptr, need);
    cap = e == cudaSuccess ? need : 0;
  };
  grow(&c->d_r3g, c->r3g_cap, groups.size());
  grow(&c->d_spart, c->spart_cap, (size_t)stot * etac::H);
  grow(&c->d_d2part, c->d2_cap, groups.size() * 3 * etac::H);
  if (e == cudaSuccess && !c->d_a3part) e = dalloc(&c->d_a3part, (size_t)a3tot);
  if (e == cudaSuccess && !c->d_a3_toff) e = dalloc(&c->d_a3_toff, (size_t)c->T);
  if (e == cudaSuccess && !c->d_a3_tg) e = dalloc(&c->d_a3_tg, (size_t)c->T);
  if (e == cudaSuccess && !c->d_s_toff) e = dalloc(&c->d_s_toff, (size_t)c->T);
  if (e == cudaSuccess && !c->d_s_nr) e = dalloc(&c->d_s_nr, (size_t)c->T);
  if (e == cudaSuccess && !groups.empty())
    e = cudaMemcpyAsync(c->d_r3g, groups.data(), sizeof(etac::R3Group) * groups.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_a3_toff, a3_toff.data(), sizeof(long long) * c->T,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_a3_tg, a3_tg.data(), sizeof(int) * c->T,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_s_toff, s_toff.data(), sizeof(long long) * c->T,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_s_nr, s_nr.data(), sizeof(int) * c->T,
                                            cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "decoder-reverse work units");
  c->r3_parts = (int)groups.size();
  c->r3_range = range;
  return ETAC_OK;
}

// Buffers and tensor maps of the staged batched reverse mode (once per context).
etac_status setup_bwdb(etac_ctx* c, cudaStream_t s) {
  if (c->bwdb_ready) return ETAC_OK;
  etac_status st = setup_instances(c, s);
  if (st != ETAC_OK) return st;
  const int np = c->E * c->P;
  const size_t tn = (size_t)c->type_off[c->T];
  const size_t om = (size_t)c->omega_off[c->T];
  c->r4_parts = 3 * c->num_sms;                         // CTAs of the R4 grid (8 warps each)
  c->r4b_parts = (np + 63) / 64;
  c->r5_parts = (int)((tn + 63) / 64);
  cudaError_t e = dalloc(reinterpret_cast<char**>(&c->d_om_hi), 2 * om);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_om_lo), 2 * om);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_dom_hi), 2 * om);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_dom_lo), 2 * om);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_bg_hi), 2 * (size_t)c->bt_total);
  if (e == cudaSuccess) e = dalloc(reinterpret_cast<char**>(&c->d_bg_lo), 2 * (size_t)c->bt_total);
  if (e == cudaSuccess) e = dalloc(&c->d_pr, (size_t)np * etac::PR_STRIDE);
  if (e == cudaSuccess) e = dalloc(&c->d_inst_m, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&c->d_a3, tn * etac::H);
  if (e == cudaSuccess) e = dalloc(&c->d_r4part, (size_t)c->r4_parts * (etac::OFF_W2 - etac::OFF_W1));
  if (e == cudaSuccess) e = dalloc(&c->d_r4bpart, (size_t)c->r4b_parts * (etac::OFF_W4 - etac::OFF_W2));
  if (e == cudaSuccess) e = dalloc(&c->d_r5part, (size_t)c->r5_parts * (etac::OFF_W4 - etac::OFF_W1));
  if (e == cudaSuccess) e = dalloc(&c->d_alpha_part, (size_t)c->num_sms);   // >= GEMM grid
  if (e == cudaSuccess) e = dalloc(&c->d_gsum_part, (size_t)c->r4b_parts * 3);
  if (e == cudaSuccess && !c->d_g0a) e = dalloc(&c->d_g0a, (size_t)np * etac::H);
  if (e == cudaSuccess) e = dalloc(&c->d_g0arg, (size_t)np * etac::H);
  if (e != cudaSuccess) return cuda_fail(c, e, "reverse-mode buffers");
  if ((st = build_r3(c, c->r3_range, s)) != ETAC_OK) return st;
  for (int which = 0; which < 2; ++which) {
    etac::GemmParams& g = which == 0 ? c->gemm_bu : c->gemm_ba;
    memset(&g, 0, sizeof g);
    fill_gemm_common(c, g);
    g.inst_m = c->d_inst_m;
    g.alpha_part = c->d_alpha_part;   // ws_u / ws_du are bound at launch (allocated later)
  }
  if ((st = encode_bwd_maps(c)) != ETAC_OK) return st;
  int per_sm = 0;
  e = etac::bwd_pad_occupancy(c->nmax, c->K, &per_sm);
  if (e != cudaSuccess || per_sm < 1) return cuda_fail(c, e, "reverse-mode pad kernel occupancy");
  c->bwd_r1_grid = per_sm * c->num_sms;
  c->bwdb_ready = true;
  return ETAC_OK;
}

// Largest per-type Omega table (FP32) the batched algorithm caches; beyond it (pads of
// per-instance geometry, many large types) Omega is evaluated on the fly.
constexpr size_t kOmegaTableMaxBytes = size_t(4) << 30;

etac_status build_tables(etac_ctx* c, const etac_model_desc* desc, cudaStream_t s) {
  const size_t tn = (size_t)c->type_off[c->T];
  const size_t om = (size_t)c->omega_off[c->T];
  cudaError_t e = cudaSuccess;
  if (!c->d_ctab) {
    e = dalloc(&c->d_ctab, tn * etac::H);
    if (e == cudaSuccess) e = dalloc(&c->d_f0tab, tn * etac::H);
    if (e == cudaSuccess) e = dalloc(&c->d_h0tab, tn * etac::H);
    if (e == cudaSuccess) e = dalloc(&c->d_order, tn * etac::H);
    if (e == cudaSuccess) e = dalloc(&c->d_ranked, tn * etac::H);
    if (e != cudaSuccess) return cuda_fail(c, e, "allocate per-type tables");
  }
  const bool batched = desc->algo == ETAC_ALGO_BATCHED;
  const bool fp32b = batched && desc->precision == ETAC_PREC_FP32;
  const bool fits = om * sizeof(float) <= kOmegaTableMaxBytes;
  if (fp32b && c->omega_pref == 0 && !fits)
    return fail(c, ETAC_ERR_UNSUPPORTED, "Omega table of %zu bytes exceeds %zu: on the fly only",
                om * sizeof(float), kOmegaTableMaxBytes);
  const bool need32 = fp32b && fits && c->omega_pref != 1;
  const bool need16 = batched && desc->precision == ETAC_PREC_BF16;
  c->omega_otf = fp32b && !need32;
  if (need32 && !c->d_omega) {
    e = dalloc(&c->d_omega, om);
    if (e != cudaSuccess) return cuda_fail(c, e, "allocate Omega table");
  }
  if (need16) {
    etac_status st = setup_bf16(c, s);
    if (st != ETAC_OK) return st;
  }
  // staged reverse mode (32-bit node offsets inside its kernels; otherwise the per-pad kernel)
  const bool needb = batched && tensor_core_shapes_ok(c) && 3 * c->N < (1LL << 31);
  if (needb) {
    etac_status st = setup_bwdb(c, s);
    if (st != ETAC_OK) return st;
  }
  if (batched) {   // the grid of the instantiation in effect (Omega table or on the fly)
    int per_sm = 0;
    e = etac::batched_occupancy(c->nmax, c->K, c->omega_otf, &per_sm);
    if (e != cudaSuccess) return cuda_fail(c, e, "batched occupancy");
    if (per_sm < 1) return fail(c, ETAC_ERR_UNSUPPORTED, "batched kernel does not fit an SM");
    c->batched_grid = per_sm * c->num_sms;
  }
  etac::TablesArgs a{};
  a.type_pos = c->d_type_pos;
  a.type_nrm = c->d_type_nrm;
  a.type_off = c->d_type_off;
  a.omega_off = c->d_omega_off;
  a.num_types = c->T;
  a.total_nodes = (int)tn;
  a.params = c->d_params;
  a.ctab = c->d_ctab;
  a.f0tab = c->d_f0tab;
  a.h0tab = c->d_h0tab;
  a.order = c->d_order;
  a.omega = need32 ? c->d_omega : nullptr;
  a.omega_bf16 = need16 ? c->d_omega_bf16 : nullptr;
  a.h0bf16 = need16 ? c->d_h0bf16 : nullptr;
  a.ranked = c->d_ranked;
  a.om_hi = needb ? c->d_om_hi : nullptr;
  a.om_lo = needb ? c->d_om_lo : nullptr;
  a.dom_hi = needb ? c->d_dom_hi : nullptr;
  a.dom_lo = needb ? c->d_dom_lo : nullptr;
  e = etac::launch_tables(a, c->nmax, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "per-type tables");
  c->tables_ready = true;
  return ETAC_OK;
}

// The staged reverse mode of the batched algorithms (bwd_batched.cu, prop_gemm.cu).
etac_status backward_batched(etac_ctx* c, const float* grad_disp, float* grad_obj_pose,
                             float* grad_uhat, float* grad_pen, float* grad_params,
                             cudaStream_t s) {
  const int EP = c->E * c->P;
  const bool use_l = etac::uses_propagation(c->model.mode);
  // pad -> object transforms of the differentiated step
  etac::FrontArgs f{};
  f.type_pmax = c->d_type_pmax;
  f.pad_type = c->d_pad_type;
  f.num_items = EP;
  f.P = c->P;
  f.K = c->K;
  f.obj_type = c->d_saved_obj_type;
  f.obj_dims = c->d_saved_obj_dims;
  f.obj_pose = c->d_saved_obj_pose;
  f.pad_pose = c->d_saved_pad_pose;
  f.padobj = c->d_padobj;
  f.pad_bad = c->d_pad_bad;
  f.mask_in = c->given_mask;
  f.uhat_in = c->given_uhat;
  f.meshes = c->d_meshes;
  f.num_meshes = c->num_meshes;
  {
    TimedLaunch tl_(c, K_PADOBJ, s);
    ETAC_CUDA(c, etac::launch_pad_obj(f, s), "reverse mode: pad transforms");
  }
  ETAC_CUDA(c, cudaMemsetAsync(c->d_ticket, 0, sizeof(int), s), "reset work queue");
  etac::BwdBatchedArgs b{};
  b.type_pos = c->d_type_pos;
  b.type_nrm = c->d_type_nrm;
  b.type_off = c->d_type_off;
  b.pad_type = c->d_pad_type;
  b.pad_off = c->d_pad_off;
  b.item_pad = c->d_item_pad;
  b.num_items = EP;
  b.P = c->P;
  b.K = c->K;
  b.nmax = c->nmax;
  b.total_nodes = c->type_off[c->T];
  b.pad_pose = c->d_saved_pad_pose;
  b.obj_pose = c->d_saved_obj_pose;
  b.params = c->d_params;
  b.ctab = c->d_ctab;
  b.f0tab = c->d_f0tab;
  b.h0tab = c->d_h0tab;
  b.ranked = c->d_ranked;
  b.padobj = c->d_padobj;
  b.pad_bad = c->d_pad_bad;
  b.pad_inst = c->d_pad_inst;
  b.inst_off = c->d_inst_off;
  b.inst_pad = c->d_inst_pad;
  b.pad_gi = c->d_pad_gi;
  b.inst_base = c->d_inst_base;
  b.type_woff = c->d_type_woff;
  b.mask_woff = c->d_mask_woff;
  b.maskbits = c->d_maskbits;
  b.bg_off = c->d_bt_off;
  b.bg_hi = c->d_bg_hi;
  b.bg_lo = c->d_bg_lo;
  b.mode = c->model.mode;
  b.mask_in = c->given_mask;
  b.uhat_in = c->given_uhat;
  b.g0rec = c->fwd_recorded ? c->d_g0a : nullptr;
  b.g0arg = c->fwd_recorded ? c->d_g0arg : nullptr;
  b.has_meshes = c->num_meshes > 0;
  b.grad_disp = grad_disp;
  b.grad_uhat = grad_uhat;
  b.grad_pen = grad_pen;
  b.ws_u = c->d_ws_u;
  b.ws_du = c->d_ws_du;
  b.pr = c->d_pr;
  b.pad_m = c->d_pad_m;
  b.inst_m = c->d_inst_m;
  b.r3_groups = c->d_r3g;
  b.r3_parts = c->r3_parts;
  b.a3part = c->d_a3part;
  b.a3_toff = c->d_a3_toff;
  b.a3_tgroups = c->d_a3_tg;
  b.a3 = c->d_a3;
  b.spart = c->d_spart;
  b.s_toff = c->d_s_toff;
  b.s_nr = c->d_s_nr;
  b.d2part = c->d_d2part;
  b.r4part = c->d_r4part;
  b.r4_parts = c->r4_parts;
  b.r4bpart = c->d_r4bpart;
  b.r4b_parts = c->r4b_parts;
  b.gsum_part = c->d_gsum_part;
  b.r5part = c->d_r5part;
  b.r5_parts = c->r5_parts;
  b.alpha_part = c->d_alpha_part;
  b.alpha_parts = use_l ? c->alpha_parts : 0;
  b.pose_part = c->d_pose_part;
  b.ticket = c->d_ticket;
  if (!etac::uses_residual(c->model.mode)) {   // no network: only alpha has a gradient
    b.r3_parts = b.r4_parts = b.r4b_parts = b.r5_parts = 0;
  }
  {
    const void* need[] = {b.ws_u, b.ws_du, b.pr, b.pad_m, b.inst_m, b.padobj, b.pad_bad,
                          b.maskbits, b.mask_woff, b.bg_hi, b.bg_lo, b.r3_groups, b.a3part,
                          b.a3, b.d2part, b.r4part, b.r4bpart, b.r5part, b.alpha_part, b.gsum_part, b.spart, b.s_toff, b.s_nr,
                          b.pose_part, b.ranked, b.h0tab, b.ctab, b.f0tab};
    for (const void* q : need)
      if (!q) return fail(c, ETAC_ERR_STATE, "reverse-mode buffers are not set up");
  }
  etac::BwdBatchedLaunch l{};
  l.r1_grid = c->bwd_r1_grid;
  l.r2_grid = std::max(1, std::min(4 * c->num_sms, (EP + 7) / 8));
  l.r7_grid = std::max(1, std::min(4 * c->num_sms, (EP + 7) / 8));
  auto stage = [&](int st, int slot, const char* what) -> etac_status {
    {
      TimedLaunch tl_(c, slot, s);
      ETAC_CUDA(c, etac::launch_backward_stage(b, l, st, grad_params, s), what);
    }
    return ETAC_OK;
  };
  etac_status st = stage(etac::BWD_STAGE_PAD, K_BWD_PAD, "reverse mode: pad stage");
  if (st != ETAC_OK) return st;
  if (etac::uses_residual(c->model.mode)) {
    if ((st = stage(etac::BWD_STAGE_GLOBAL, K_BWD_GLOBAL, "reverse mode: global MLP")) != ETAC_OK ||
        (st = stage(etac::BWD_STAGE_DECODER, K_BWD_DECODER, "reverse mode: decoder")) != ETAC_OK ||
        (st = stage(etac::BWD_STAGE_A3SUM, K_BWD_A3SUM, "reverse mode: decoder sums")) != ETAC_OK ||
        (st = stage(etac::BWD_STAGE_PADREV, K_BWD_PADREV, "reverse mode: pad reverse")) != ETAC_OK ||
        (st = stage(etac::BWD_STAGE_PADSUM, K_BWD_PADSUM, "reverse mode: pad sums")) != ETAC_OK ||
        (st = stage(etac::BWD_STAGE_TYPENODE, K_BWD_TYPENODE, "reverse mode: type nodes")) != ETAC_OK)
      return st;
  }
  if (use_l) {
    for (etac::GemmParams* g : {&c->gemm_bu, &c->gemm_ba}) {
      g->ws_u = c->d_ws_u;
      g->ws_du = c->d_ws_du;
      if (!g->ws_u || !g->ws_du || !g->inst_m || !g->alpha_part || !g->tiles)
        return fail(c, ETAC_ERR_STATE, "reverse-mode GEMM buffers are not set up");
    }
    {
      TimedLaunch tl_(c, K_BWD_GEMM_U, s);
      ETAC_CUDA(c, etac::launch_prop_gemm(c->gemm_bu, c->gemm_grid, s, etac::GEMM_BWD_U, c->gemm_gi),
                "reverse mode: propagation GEMM");
    }
    {
      TimedLaunch tl_(c, K_BWD_GEMM_A, s);
      ETAC_CUDA(c, etac::launch_prop_gemm(c->gemm_ba, c->gemm_grid, s, etac::GEMM_BWD_ALPHA, c->gemm_gi),
                "reverse mode: alpha GEMM");
    }
  }
  if ((st = stage(etac::BWD_STAGE_POSE, K_BWD_POSE, "reverse mode: outputs")) != ETAC_OK ||
      (st = stage(etac::BWD_STAGE_PARAMS, K_BWD_POSE, "reverse mode: parameter sums")) != ETAC_OK)
    return st;
  if (grad_obj_pose)
    ETAC_CUDA(c, etac::launch_reduce_pose(c->d_pose_part, c->E, c->P, c->K, grad_obj_pose, s),
              "reverse mode: pose sums");
  return ETAC_OK;
}

}  // namespace

namespace etac {
// message of a failed call that has no context (read back with etac_last_error(NULL))
void set_context_free_error(const std::string& msg) { g_create_err = msg; }
}  // namespace etac

extern "C" {

size_t etac_param_count(const etac_model_desc* desc) {
  if (desc && desc->hidden != ETAC_HIDDEN) return 0;
  return (size_t)etac::NPARAM;
}

int64_t etac_total_nodes(const etac_pads_desc* d) {
  if (!d || d->num_types < 1 || !d->type_num_nodes || !d->pad_type || d->num_envs < 1 ||
      d->pads_per_env < 1)
    return 0;
  int64_t N = 0;
  for (int64_t p = 0; p < (int64_t)d->num_envs * d->pads_per_env; ++p) {
    int t = d->pad_type[p];
    if (t < 0 || t >= d->num_types) return 0;
    int n = d->type_num_nodes[t];
    if (n < 1 || n > ETAC_MAX_PAD_NODES) return 0;
    N += n;
  }
  return N;
}

etac_status etac_create_pads(etac_ctx** out, const etac_pads_desc* d, void* stream) {
  NvtxScope nvtx_("etac_create_pads");
  if (!out) return fail(nullptr, ETAC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(nullptr, ETAC_ERR_INVALID_ARG, "desc is NULL");
  if (d->num_types < 1 || !d->type_num_nodes || !d->type_pos || !d->type_nrm || !d->pad_type)
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "pad types: num_types < 1 or NULL array");
  if (d->num_envs < 1 || d->pads_per_env < 1)
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "num_envs and pads_per_env must be >= 1");
  if (d->max_objects < 1 || d->max_objects > ETAC_MAX_OBJECTS)
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "max_objects must be in [1, %d]",
                ETAC_MAX_OBJECTS);
  int64_t np = (int64_t)d->num_envs * d->pads_per_env;
  if (np > (int64_t)INT32_MAX / 2)
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "too many pads");
  etac_ctx* c = new etac_ctx();
  c->T = d->num_types;
  c->E = d->num_envs;
  c->P = d->pads_per_env;
  c->K = d->max_objects;
  c->type_n.assign(d->type_num_nodes, d->type_num_nodes + c->T);
  c->type_off.resize(c->T + 1, 0);
  for (int t = 0; t < c->T; ++t) {
    int n = c->type_n[t];
    if (n < 1 || n > ETAC_MAX_PAD_NODES) {
      free_ctx(c);
      return fail(nullptr, ETAC_ERR_INVALID_ARG, "pad type %d has %d nodes (allowed 1..%d)", t,
                  n, ETAC_MAX_PAD_NODES);
    }
    c->type_off[t + 1] = c->type_off[t] + n;
    c->nmax = std::max(c->nmax, n);
  }
  const int total_type_nodes = c->type_off[c->T];
  c->type_pmax.assign(c->T, 0.f);
  // type_pmax: the largest Euclidean |p| of the type's nodes (the screening margin's bound)
  for (int t = 0; t < c->T; ++t)
    for (int i = c->type_off[t]; i < c->type_off[t + 1]; ++i) {
      double p2 = 0.0;
      for (int q = 0; q < 3; ++q) {
        float v = d->type_pos[3 * i + q], w = d->type_nrm[3 * i + q];
        if (!std::isfinite(v) || !std::isfinite(w)) {
          free_ctx(c);
          return fail(nullptr, ETAC_ERR_INVALID_ARG, "non-finite node geometry (type %d)", t);
        }
        p2 += (double)v * v;
      }
      // rounded up so that the FP32 value is never below the exact norm
      c->type_pmax[t] = std::max(c->type_pmax[t], std::nextafter((float)std::sqrt(p2), INFINITY));
    }
  c->blk_perm.resize(total_type_nodes);
  c->type_boff.assign(c->T, 0);
  for (int t = 0; t < c->T; ++t) {
    c->type_boff[t] = (int)c->blk_sphere.size();
    build_blocks(d->type_pos + 3 * (size_t)c->type_off[t], c->type_n[t],
                 c->blk_perm.data() + c->type_off[t], c->blk_sphere);
  }
  c->pad_type.assign(d->pad_type, d->pad_type + np);
  c->pad_off.resize(np + 1, 0);
  for (int64_t p = 0; p < np; ++p) {
    int t = c->pad_type[p];
    if (t < 0 || t >= c->T) {
      free_ctx(c);   // the message takes the type count from the description, not from c
      return fail(nullptr, ETAC_ERR_INVALID_ARG, "pad %lld has type %d (num_types %d)",
                  (long long)p, t, d->num_types);
    }
    c->pad_off[p + 1] = c->pad_off[p] + c->type_n[t];
  }
  c->N = c->pad_off[np];
  // work items of the batched algorithm: pads by decreasing node count (stable)
  c->item_pad.resize(np);
  for (int64_t p = 0; p < np; ++p) c->item_pad[p] = (int)p;
  std::stable_sort(c->item_pad.begin(), c->item_pad.end(), [&](int x, int y) {
    return c->type_n[c->pad_type[x]] > c->type_n[c->pad_type[y]];
  });
  c->omega_off.assign(c->T + 1, 0);
  for (int t = 0; t < c->T; ++t)
    c->omega_off[t + 1] = c->omega_off[t] + (long long)c->type_n[t] * c->type_n[t];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = dalloc(&c->d_type_pos, 3 * (size_t)total_type_nodes);
  if (e == cudaSuccess) e = dalloc(&c->d_type_nrm, 3 * (size_t)total_type_nodes);
  if (e == cudaSuccess) e = dalloc(&c->d_type_pmax, c->T);
  if (e == cudaSuccess) e = dalloc(&c->d_type_off, c->T + 1);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_type, np);
  if (e == cudaSuccess) e = dalloc(&c->d_pad_off, np + 1);
  if (e == cudaSuccess) e = dalloc(&c->d_status, 1);
  if (e == cudaSuccess) e = dalloc(&c->d_params, etac::NPARAM);
  if (e == cudaSuccess) e = dalloc(&c->d_saved_obj_type, (size_t)c->E * c->K);
  if (e == cudaSuccess) e = dalloc(&c->d_saved_obj_dims, (size_t)c->E * c->K * 3);
  if (e == cudaSuccess) e = dalloc(&c->d_saved_obj_pose, (size_t)c->E * c->K * 7);
  if (e == cudaSuccess) e = dalloc(&c->d_saved_pad_pose, (size_t)np * 7);
  if (e == cudaSuccess) e = dalloc(&c->d_omega_off, c->T + 1);
  if (e == cudaSuccess) e = dalloc(&c->d_item_pad, np);
  if (e == cudaSuccess) e = dalloc(&c->d_ticket, 4);
  if (e == cudaSuccess) e = dalloc(&c->d_blk_perm, c->blk_perm.size());
  if (e == cudaSuccess) e = dalloc(&c->d_blk_sphere, c->blk_sphere.size());
  if (e == cudaSuccess) e = dalloc(&c->d_type_boff, c->T);
  std::vector<float> bpos(3 * (size_t)total_type_nodes), bnrm(3 * (size_t)total_type_nodes);
  for (int t = 0; t < c->T; ++t)
    for (int s = 0; s < c->type_n[t]; ++s) {
      const size_t src = c->type_off[t] + (size_t)c->blk_perm[c->type_off[t] + s];
      for (int q = 0; q < 3; ++q) {
        bpos[3 * ((size_t)c->type_off[t] + s) + q] = d->type_pos[3 * src + q];
        bnrm[3 * ((size_t)c->type_off[t] + s) + q] = d->type_nrm[3 * src + q];
      }
    }
  if (e == cudaSuccess) e = dalloc(&c->d_blk_pos, bpos.size());
  if (e == cudaSuccess) e = dalloc(&c->d_blk_nrm, bnrm.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_blk_pos, bpos.data(), sizeof(float) * bpos.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_blk_nrm, bnrm.data(), sizeof(float) * bnrm.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_blk_perm, c->blk_perm.data(), sizeof(int16_t) * c->blk_perm.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_blk_sphere, c->blk_sphere.data(),
                        sizeof(float4) * c->blk_sphere.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_type_boff, c->type_boff.data(), sizeof(int) * c->T,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_omega_off, c->omega_off.data(), sizeof(long long) * (c->T + 1),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_item_pad, c->item_pad.data(), sizeof(int) * np,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_type_pos, d->type_pos, sizeof(float) * 3 * total_type_nodes,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_type_nrm, d->type_nrm, sizeof(float) * 3 * total_type_nodes,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_type_pmax, c->type_pmax.data(), sizeof(float) * c->T,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_type_off, c->type_off.data(), sizeof(int) * (c->T + 1),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_pad_type, c->pad_type.data(), sizeof(int) * np,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_pad_off, c->pad_off.data(), sizeof(long long) * (np + 1),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
  // host vectors are pageable: the copies above complete before returning
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    etac_status st = cuda_fail(nullptr, e, "etac_create_pads");
    free_ctx(c);
    return st;
  }
  if (etac::plain_smem_f32(c->nmax, c->K) > 227 * 1024) {
    free_ctx(c);
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "pad type too large for the plain algorithm");
  }
  *out = c;
  return ETAC_OK;
}

etac_status etac_set_model(etac_ctx* c, const etac_model_desc* desc, const float* params,
                           void* stream) {
  NvtxScope nvtx_("etac_set_model");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!valid_model(desc))
    return fail(c, ETAC_ERR_INVALID_ARG,
                "model desc: hidden must be %d; mode, precision, algo must be known values",
                ETAC_HIDDEN);
  if (!params || !aligned(params, 4)) return fail(c, ETAC_ERR_INVALID_ARG, "params NULL/misaligned");
  if (desc->precision == ETAC_PREC_BF16 && desc->algo != ETAC_ALGO_BATCHED)
    return fail(c, ETAC_ERR_UNSUPPORTED, "BF16 precision is implemented by the batched algorithm");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float alpha = 0.f;
  ETAC_CUDA(c, cudaMemcpyAsync(&alpha, params, sizeof(float), cudaMemcpyDeviceToHost, s),
            "read alpha");
  ETAC_CUDA(c, cudaStreamSynchronize(s), "read alpha");
  if (!(std::isfinite(alpha) && alpha > 0.f))
    return fail(c, ETAC_ERR_INVALID_ARG, "alpha must be finite and > 0 (got %g)", alpha);
  ETAC_CUDA(c, cudaMemcpyAsync(c->d_params, params, sizeof(float) * etac::NPARAM,
                               cudaMemcpyDeviceToDevice, s), "copy params");
  etac_status st = build_tables(c, desc, s);   // also used by the reverse mode
  if (st != ETAC_OK) return st;
  if (!c->d_ws_idx) {
    const size_t np = (size_t)c->E * c->P;
    if (etac::backward_smem_bytes(c->nmax, c->K) > 227 * 1024)
      return fail(c, ETAC_ERR_UNSUPPORTED, "pad type too large for the reverse mode");
    c->bwd_grid = c->num_sms;
    cudaError_t e = dalloc(&c->d_ws_idx, (size_t)c->N);
    if (e == cudaSuccess) e = dalloc(&c->d_ws_u, (size_t)c->N);
    if (e == cudaSuccess) e = dalloc(&c->d_ws_du, (size_t)c->N);
    if (e == cudaSuccess) e = dalloc(&c->d_pose_part, np * c->K * 6);
    if (e == cudaSuccess) e = dalloc(&c->d_param_part, (size_t)c->bwd_grid * etac::NPARAM);
    if (e != cudaSuccess) return cuda_fail(c, e, "reverse-mode workspace");
  }
  c->model = *desc;
  c->has_model = true;
  return ETAC_OK;
}

etac_status etac_step_forward(etac_ctx* c, const etac_step_in* in, const etac_step_out* out,
                              void* stream) {
  NvtxScope nvtx_("etac_step_forward");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_model) return fail(c, ETAC_ERR_STATE, "etac_set_model has not been called");
  if (!in || !out) return fail(c, ETAC_ERR_INVALID_ARG, "in/out is NULL");
  const bool given = in->active_mask_in != nullptr;
  if (given != (in->active_disp_in != nullptr))
    return fail(c, ETAC_ERR_INVALID_ARG,
                "active_mask_in and active_disp_in must be given together (or neither)");
  if ((!given && (!in->obj_type || !in->obj_dims || !in->obj_pose || !in->pad_pose)) ||
      !out->disp)
    return fail(c, ETAC_ERR_INVALID_ARG, "required input/output pointer is NULL");
  if ((!given && (!aligned(in->obj_type, 4) || !aligned(in->obj_dims, 4) ||
                  !aligned(in->obj_pose, 4) || !aligned(in->pad_pose, 4))) ||
      (given && !aligned(in->active_disp_in, 4)) || !aligned(out->disp, 4) ||
      (out->penetration && !aligned(out->penetration, 4)) ||
      (out->active_count && !aligned(out->active_count, 4)))
    return fail(c, ETAC_ERR_INVALID_ARG, "pointer not 4-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t EK = (size_t)c->E * c->K, EP = (size_t)c->E * c->P;
  // keep this step's inputs for the reverse mode (mode B: the caller's buffers, borrowed)
  if (!given) {
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_saved_obj_type, in->obj_type, sizeof(int) * EK,
                                 cudaMemcpyDeviceToDevice, s), "save inputs");
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_saved_obj_dims, in->obj_dims, sizeof(float) * EK * 3,
                                 cudaMemcpyDeviceToDevice, s), "save inputs");
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_saved_obj_pose, in->obj_pose, sizeof(float) * EK * 7,
                                 cudaMemcpyDeviceToDevice, s), "save inputs");
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_saved_pad_pose, in->pad_pose, sizeof(float) * EP * 7,
                                 cudaMemcpyDeviceToDevice, s), "save inputs");
  }
  // a forward that fails from here on leaves no state to differentiate
  c->has_forward = false;
  c->fwd_recorded = false;
  c->given_mask = in->active_mask_in;
  c->given_uhat = in->active_disp_in;
  if (c->model.algo == ETAC_ALGO_BATCHED) {
    etac::BatchedArgs b{};
    b.type_pos = c->d_type_pos;
    b.type_nrm = c->d_type_nrm;
    b.type_pmax = c->d_type_pmax;
    b.type_off = c->d_type_off;
    b.omega_off = c->d_omega_off;
    b.num_nodes = c->N;
    b.pad_type = c->d_pad_type;
    b.pad_off = c->d_pad_off;
    b.item_pad = c->d_item_pad;
    b.num_items = (int)EP;
    b.P = c->P;
    b.K = c->K;
    b.nmax = c->nmax;
    b.obj_type = c->d_saved_obj_type;
    b.obj_dims = c->d_saved_obj_dims;
    b.obj_pose = c->d_saved_obj_pose;
    b.pad_pose = c->d_saved_pad_pose;
    b.params = c->d_params;
    b.ctab = c->d_ctab;
    b.f0tab = c->d_f0tab;
    b.h0tab = c->d_h0tab;
    b.order = c->d_order;
    b.omega = c->omega_otf ? nullptr : c->d_omega;
    b.mode = c->model.mode;
    b.disp = out->disp;
    b.mask = out->active_mask;
    b.pen = out->penetration;
    b.count = out->active_count;
    b.ticket = c->d_ticket;
    b.status = c->d_status;
    b.mask_in = c->given_mask;
    b.uhat_in = c->given_uhat;
    b.meshes = c->d_meshes;
    b.num_meshes = c->num_meshes;
    // the FP32 forward records each pad's max-pool state for the staged reverse mode
    const bool record = c->bwdb_ready && c->d_g0arg && c->model.precision == ETAC_PREC_FP32;
    b.g0rec = record ? c->d_g0a : nullptr;
    b.g0arg = record ? c->d_g0arg : nullptr;
    c->fwd_recorded = record;
    ETAC_CUDA(c, cudaMemsetAsync(c->d_ticket, 0, sizeof(int), s), "reset work queue");
    if (c->model.precision == ETAC_PREC_BF16) {
      etac::FrontArgs f{};
      f.type_pos = c->d_type_pos;
      f.type_nrm = c->d_type_nrm;
      f.type_pmax = c->d_type_pmax;
      f.type_off = c->d_type_off;
      f.pad_type = c->d_pad_type;
      f.pad_off = c->d_pad_off;
      f.item_pad = c->d_item_pad;
      f.num_nodes = c->N;
      f.bt_total = c->bt_total;
      f.mask_words = c->mask_words;
      f.num_items = (int)EP;
      f.P = c->P;
      f.K = c->K;
      f.nmax = c->nmax;
      f.obj_type = c->d_saved_obj_type;
      f.obj_dims = c->d_saved_obj_dims;
      f.obj_pose = c->d_saved_obj_pose;
      f.pad_pose = c->d_saved_pad_pose;
      f.params = c->d_params;
      f.ctab = c->d_ctab;
      f.f0tab = c->d_f0tab;
      f.order = c->d_order;
      f.ranked = c->d_ranked;
      f.mode = c->model.mode;
      f.disp = out->disp;
      f.mask = out->active_mask;
      f.pen = out->penetration;
      f.count = out->active_count;
      f.ticket = c->d_ticket;
      f.status = c->d_status;
      f.bt = c->d_bt;
      f.bt_off = c->d_bt_off;
      f.pad_inst = c->d_pad_inst;
      f.maskbits = c->d_maskbits;
      f.mask_woff = c->d_mask_woff;
      f.pad_m = c->d_pad_m;
      f.g0a = c->d_g0a;
      f.negbeta = c->d_negbeta;
      f.c0m = c->d_c0m;
      f.pad_gi = c->d_pad_gi;
      f.padobj = c->d_padobj;
      f.pad_bad = c->d_pad_bad;
      f.mask_in = c->given_mask;
      f.uhat_in = c->given_uhat;
      f.meshes = c->d_meshes;
      f.num_meshes = c->num_meshes;
      f.blk_perm = c->d_blk_perm;
      f.blk_pos = c->d_blk_pos;
      f.blk_nrm = c->d_blk_nrm;
      f.blk_sphere = c->d_blk_sphere;
      f.type_boff = c->d_type_boff;
      f.btbits = c->d_btbits;
      if (!f.blk_perm || !f.blk_pos || !f.blk_nrm || !f.blk_sphere || !f.type_boff || !f.btbits || !f.padobj || !f.pad_bad || !f.pad_gi || !c->gemm.inst_base || !c->gemm.type_woff || !f.bt || !f.bt_off || !f.pad_inst || !f.negbeta || !f.c0m || !f.maskbits ||
          !f.mask_woff || !f.pad_m || !f.g0a || !f.ranked || !c->gemm.tiles || !c->gemm.h0bf16 ||
          !c->gemm.maskbits)
        return fail(c, ETAC_ERR_STATE, "BF16 buffers are not set up");
      {
        TimedLaunch tl_(c, K_PADOBJ, s);
        ETAC_CUDA(c, etac::launch_pad_obj(f, s), "pad transforms launch");
      }
      {
        TimedLaunch tl_(c, K_FRONT, s);
        ETAC_CUDA(c, etac::launch_front_contact(f, std::min<int>(c->front_grid, (int)EP), s),
                  "BF16 front launch");
      }
      {
        TimedLaunch tl_(c, K_GLOBAL, s);
        ETAC_CUDA(c, etac::launch_front_global(f, c->num_sms, s),
                  "BF16 global-feature launch");
      }
      etac::GemmParams& g = c->gemm;
      g.disp = out->disp;
      g.use_l = etac::uses_propagation(c->model.mode);
      g.use_r = etac::uses_residual(c->model.mode);
      {
        TimedLaunch tl_(c, K_GEMM, s);
        ETAC_CUDA(c, etac::launch_prop_gemm(g, c->gemm_grid, s, etac::GEMM_FWD, c->gemm_gi), "BF16 propagation GEMM launch");
      }
      c->has_forward = true;
      ++c->step_id;
      return ETAC_OK;
    }
    {
      TimedLaunch tl_(c, K_BATCHED, s);
      ETAC_CUDA(c, etac::launch_batched_forward(b, std::min<int>(c->batched_grid, (int)EP), s),
                "batched forward launch");
    }
    c->has_forward = true;
    ++c->step_id;
    return ETAC_OK;
  }
  etac::PlainArgs<float> a{};
  a.num_nodes = c->N;
  a.type_pos = c->d_type_pos;
  a.type_nrm = c->d_type_nrm;
  a.type_pmax = c->d_type_pmax;
  a.type_off = c->d_type_off;
  a.pad_type = c->d_pad_type;
  a.pad_off = c->d_pad_off;
  a.P = c->P;
  a.K = c->K;
  a.nmax = c->nmax;
  a.obj_type = c->d_saved_obj_type;
  a.obj_dims = c->d_saved_obj_dims;
  a.obj_pose = c->d_saved_obj_pose;
  a.pad_pose = c->d_saved_pad_pose;
  a.params = c->d_params;
  a.mode = c->model.mode;
  a.disp = out->disp;
  a.mask = out->active_mask;
  a.pen = out->penetration;
  a.count = out->active_count;
  a.status = c->d_status;
  a.mask_in = c->given_mask;
  a.uhat_in = c->given_uhat;
  a.meshes = c->d_meshes;
  a.num_meshes = c->num_meshes;
  {
    TimedLaunch tl_(c, K_PLAIN, s);
    ETAC_CUDA(c, etac::launch_plain_forward<float>(a, (int)EP, s), "plain forward launch");
  }
  c->has_forward = true;
  ++c->step_id;
  return ETAC_OK;
}

etac_status etac_set_meshes(etac_ctx* c, const etac_mesh_gpu* const* meshes, int32_t count,
                            void* stream) {
  NvtxScope nvtx_("etac_set_meshes");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (count < 0 || (count > 0 && !meshes))
    return fail(c, ETAC_ERR_INVALID_ARG, "meshes: count %d with %s list", count,
                meshes ? "a" : "a NULL");
  std::vector<etac::MeshDev> h(count);
  for (int i = 0; i < count; ++i) {
    if (!meshes[i]) return fail(c, ETAC_ERR_INVALID_ARG, "mesh %d is NULL", i);
    etac::mesh_dev_view(meshes[i], &h[i]);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (count > c->meshes_cap) {
    if (c->d_meshes) {
      ETAC_CUDA(c, cudaStreamSynchronize(s), "mesh table");
      cudaFree(c->d_meshes);
      c->d_meshes = nullptr;
      c->meshes_cap = 0;
    }
    cudaError_t e = dalloc(&c->d_meshes, (size_t)count);
    if (e != cudaSuccess) return cuda_fail(c, e, "mesh table");
    c->meshes_cap = count;
  }
  if (count > 0)
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_meshes, h.data(), sizeof(etac::MeshDev) * count,
                                 cudaMemcpyHostToDevice, s), "mesh table");
  ETAC_CUDA(c, cudaStreamSynchronize(s), "mesh table");   // h is pageable and goes away
  c->num_meshes = count;
  return ETAC_OK;
}

etac_status etac_test_withhold_load(etac_ctx* c, int32_t tile, uint64_t wait_limit_ns) {
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_model || c->model.algo != ETAC_ALGO_BATCHED ||
      c->model.precision != ETAC_PREC_BF16 || !c->bf16_ready)
    return fail(c, ETAC_ERR_STATE, "the load hook applies to a batched BF16 model");
  if (tile < -1 || tile >= c->num_tiles)
    return fail(c, ETAC_ERR_INVALID_ARG, "tile %d outside [-1, %d)", tile, c->num_tiles);
  if (wait_limit_ns > 2000000000ull)
    return fail(c, ETAC_ERR_INVALID_ARG, "wait limit above 2 s");
  c->gemm.test_withhold = tile + 1;
  c->gemm.timeout_ns = wait_limit_ns ? wait_limit_ns : 2000000000ull;
  return ETAC_OK;
}

etac_status etac_last_step(const etac_ctx* c, uint64_t* step_id) {
  if (!c || !step_id) return fail(nullptr, ETAC_ERR_INVALID_ARG, "NULL argument");
  *step_id = c->has_forward ? c->step_id : 0;
  return ETAC_OK;
}

etac_status etac_step_backward(etac_ctx* c, uint64_t step_id, const float* grad_disp,
                               float* grad_obj_pose, float* grad_uhat, float* grad_penetration,
                               float* grad_params, void* stream) {
  NvtxScope nvtx_("etac_step_backward");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!c->has_forward) return fail(c, ETAC_ERR_STATE, "no forward step to differentiate");
  if (step_id != 0 && step_id != c->step_id)
    return fail(c, ETAC_ERR_STATE,
                "step %llu is not the last forward on this context (last: %llu); its saved "
                "state has been overwritten",
                (unsigned long long)step_id, (unsigned long long)c->step_id);
  if (!grad_disp) return fail(c, ETAC_ERR_INVALID_ARG, "grad_disp is NULL");
  if (!aligned(grad_disp, 4) || (grad_obj_pose && !aligned(grad_obj_pose, 4)) ||
      (grad_uhat && !aligned(grad_uhat, 4)) || (grad_penetration && !aligned(grad_penetration, 4)) ||
      (grad_params && !aligned(grad_params, 4)))
    return fail(c, ETAC_ERR_INVALID_ARG, "pointer not 4-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (c->model.algo == ETAC_ALGO_BATCHED && c->bwdb_ready)
    return backward_batched(c, grad_disp, grad_obj_pose, grad_uhat, grad_penetration, grad_params, s);
  etac::BackwardArgs b{};
  b.type_pos = c->d_type_pos;
  b.type_nrm = c->d_type_nrm;
  b.type_pmax = c->d_type_pmax;
  b.type_off = c->d_type_off;
  b.pad_type = c->d_pad_type;
  b.pad_off = c->d_pad_off;
  b.item_pad = c->d_item_pad;
  b.num_items = c->E * c->P;
  b.E = c->E;
  b.P = c->P;
  b.K = c->K;
  b.nmax = c->nmax;
  b.obj_type = c->d_saved_obj_type;
  b.obj_dims = c->d_saved_obj_dims;
  b.obj_pose = c->d_saved_obj_pose;
  b.pad_pose = c->d_saved_pad_pose;
  b.params = c->d_params;
  b.ctab = c->d_ctab;
  b.f0tab = c->d_f0tab;
  b.h0tab = c->d_h0tab;
  b.order = c->d_order;
  b.ranked = c->d_ranked;
  b.mode = c->model.mode;
  b.grad_disp = grad_disp;
  b.grad_uhat = grad_uhat;
  b.grad_pen = grad_penetration;
  b.grad_params = grad_params;
  b.grad_obj_pose = grad_obj_pose;
  b.ws_idx = c->d_ws_idx;
  b.ws_u = c->d_ws_u;
  b.ws_du = c->d_ws_du;
  b.pose_part = c->d_pose_part;
  b.param_part = c->d_param_part;
  b.mask_in = c->given_mask;
  b.uhat_in = c->given_uhat;
  b.meshes = c->d_meshes;
  b.num_meshes = c->num_meshes;
  {
    TimedLaunch tl_(c, K_BWD, s);
    ETAC_CUDA(c, etac::launch_backward(b, c->bwd_grid, s), "reverse-mode launch");
  }
  return ETAC_OK;
}

etac_status etac_set_tuning(etac_ctx* c, const etac_tuning* t, void* stream) {
  if (!c || !t) return fail(c, ETAC_ERR_INVALID_ARG, "NULL argument");
  if (!c->has_model || c->model.algo != ETAC_ALGO_BATCHED)
    return fail(c, ETAC_ERR_STATE, "tuning applies to a batched model");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (c->model.precision == ETAC_PREC_FP32) {
    if (t->omega_source < ETAC_OMEGA_AUTO || t->omega_source > ETAC_OMEGA_ON_THE_FLY)
      return fail(c, ETAC_ERR_INVALID_ARG, "omega_source %d unknown", t->omega_source);
    const int pref = t->omega_source == ETAC_OMEGA_TABLE ? 0
                     : t->omega_source == ETAC_OMEGA_ON_THE_FLY ? 1 : -1;
    if (pref != c->omega_pref) {
      const int old = c->omega_pref;
      c->omega_pref = pref;
      etac_status st = build_tables(c, &c->model, s);   // builds the table if now needed
      if (st != ETAC_OK) {
        c->omega_pref = old;
        return st;
      }
    }
  }
  if (c->inst_ready) {
    if ((t->gemm_inst_per_tile != 32 && t->gemm_inst_per_tile != 64 &&
         t->gemm_inst_per_tile != 80) ||
        (t->gemm_tile_order != 0 && t->gemm_tile_order != 1))
      return fail(c, ETAC_ERR_INVALID_ARG, "GEMM shape: 32, 64 or 80 instances, order 0 or 1");
    c->gemm_gi = t->gemm_inst_per_tile;
    c->gemm_order = t->gemm_tile_order;
    etac_status st = build_tiles(c, s);
    if (st == ETAC_OK && c->bf16_ready) st = encode_fwd_maps(c);
    if (st == ETAC_OK && c->bwdb_ready) st = encode_bwd_maps(c);
    if (st != ETAC_OK) return st;
  }
  if (c->bf16_ready && c->model.precision == ETAC_PREC_BF16) {
    if (t->front_ctas_per_sm < 0 || t->front_ctas_per_sm > c->front_max_per_sm)
      return fail(c, ETAC_ERR_INVALID_ARG, "front_ctas_per_sm %d outside [0, %d]",
                  t->front_ctas_per_sm, c->front_max_per_sm);
    c->front_grid =
        (t->front_ctas_per_sm ? t->front_ctas_per_sm : c->front_max_per_sm) * c->num_sms;
  }
  if (c->bwdb_ready && t->bwd_node_range) return build_r3(c, t->bwd_node_range, s);
  return ETAC_OK;
}

etac_status etac_autotune(etac_ctx* c, const etac_step_in* in, const etac_step_out* out,
                          const float* grad_disp, etac_tuning* r, void* stream) {
  NvtxScope nvtx_("etac_autotune");
  if (!c || !in || !out || !r) return fail(c, ETAC_ERR_INVALID_ARG, "NULL argument");
  if (!c->has_model || c->model.algo != ETAC_ALGO_BATCHED)
    return fail(c, ETAC_ERR_STATE, "autotuning needs a batched model");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  memset(r, 0, sizeof *r);
  r->gemm_inst_per_tile = c->gemm_gi;
  r->gemm_tile_order = c->gemm_order;
  r->bwd_node_range = c->r3_range;
  r->front_ctas_per_sm = c->num_sms ? c->front_grid / c->num_sms : 0;
  r->omega_source = c->omega_pref == 0   ? ETAC_OMEGA_TABLE
                    : c->omega_pref == 1 ? ETAC_OMEGA_ON_THE_FLY
                                         : ETAC_OMEGA_AUTO;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ETAC_CUDA(c, cudaEventCreate(&e0), "autotune events");
  ETAC_CUDA(c, cudaEventCreate(&e1), "autotune events");
  etac_status st = ETAC_OK;
  auto timed = [&](auto&& once, int warm, int reps, float* ms) -> etac_status {
    for (int i = 0; i < warm; ++i) {
      etac_status q = once();
      if (q != ETAC_OK) return q;
    }
    ETAC_CUDA(c, cudaEventRecord(e0, s), "autotune event");
    for (int i = 0; i < reps; ++i) {
      etac_status q = once();
      if (q != ETAC_OK) return q;
    }
    ETAC_CUDA(c, cudaEventRecord(e1, s), "autotune event");
    ETAC_CUDA(c, cudaEventSynchronize(e1), "autotune event");
    ETAC_CUDA(c, cudaEventElapsedTime(ms, e0, e1), "autotune event");
    *ms /= reps;
    return ETAC_OK;
  };
  auto fwd = [&]() { return etac_step_forward(c, in, out, stream); };
  auto bwd = [&]() {
    return etac_step_backward(c, 0, grad_disp, nullptr, nullptr, nullptr, nullptr, stream);
  };
  etac_tuning t = *r;
  if (c->bf16_ready && c->model.precision == ETAC_PREC_BF16) {
    const int cand[6][2] = {{64, 0}, {64, 1}, {80, 0}, {80, 1}, {32, 0}, {32, 1}};
    int best = -1;
    for (int k = 0; k < 6 && st == ETAC_OK; ++k) {
      t.gemm_inst_per_tile = cand[k][0];
      t.gemm_tile_order = cand[k][1];
      t.bwd_node_range = 0;
      if ((st = etac_set_tuning(c, &t, stream)) != ETAC_OK) break;
      float ms = 0.f;
      if ((st = timed(fwd, 2, 5, &ms)) != ETAC_OK) break;
      r->fwd_cand[k][0] = cand[k][0];
      r->fwd_cand[k][1] = cand[k][1];
      r->fwd_ms[k] = ms;
      r->num_fwd = k + 1;
      if (best < 0 || ms < r->fwd_ms[best]) best = k;
    }
    if (st == ETAC_OK) {
      t.gemm_inst_per_tile = cand[best][0];
      t.gemm_tile_order = cand[best][1];
      t.bwd_node_range = 0;
      st = etac_set_tuning(c, &t, stream);
      r->gemm_inst_per_tile = t.gemm_inst_per_tile;
      r->gemm_tile_order = t.gemm_tile_order;
    }
    // then the front kernel's CTAs per SM (its persistent grid) with the chosen GEMM tiles
    int bestf = -1;
    for (int k = 1; k <= c->front_max_per_sm && k <= ETAC_TUNE_MAX && st == ETAC_OK; ++k) {
      t.front_ctas_per_sm = k;
      if ((st = etac_set_tuning(c, &t, stream)) != ETAC_OK) break;
      float ms = 0.f;
      if ((st = timed(fwd, 2, 5, &ms)) != ETAC_OK) break;
      r->front_cand[k - 1] = k;
      r->front_ms[k - 1] = ms;
      r->num_front = k;
      if (bestf < 0 || ms < r->front_ms[bestf]) bestf = k - 1;
    }
    if (st == ETAC_OK && bestf >= 0) {
      t.front_ctas_per_sm = bestf + 1;
      st = etac_set_tuning(c, &t, stream);
      r->front_ctas_per_sm = t.front_ctas_per_sm;
    }
  }
  if (st == ETAC_OK && c->model.precision == ETAC_PREC_FP32 &&
      (size_t)c->omega_off[c->T] * sizeof(float) <= kOmegaTableMaxBytes) {
    // the batched FP32 step: Omega from the table against on the fly
    const int src[2] = {ETAC_OMEGA_TABLE, ETAC_OMEGA_ON_THE_FLY};
    for (int k = 0; k < 2 && st == ETAC_OK; ++k) {
      t.omega_source = src[k];
      if ((st = etac_set_tuning(c, &t, stream)) != ETAC_OK) break;
      if ((st = timed(fwd, 2, 5, &r->omega_ms[k])) != ETAC_OK) break;
    }
    if (st == ETAC_OK) {
      t.omega_source = r->omega_ms[1] < r->omega_ms[0] ? ETAC_OMEGA_ON_THE_FLY : ETAC_OMEGA_TABLE;
      st = etac_set_tuning(c, &t, stream);
      r->omega_source = t.omega_source;
    }
  }
  if (st == ETAC_OK && grad_disp && c->bwdb_ready && etac::uses_residual(c->model.mode)) {
    st = fwd();
    const int cand[4] = {32, 64, 128, 256};
    int best = -1;
    for (int k = 0; k < 4 && st == ETAC_OK; ++k) {
      if ((st = build_r3(c, cand[k], s)) != ETAC_OK) break;
      float ms = 0.f;
      if ((st = timed(bwd, 1, 3, &ms)) != ETAC_OK) break;
      r->bwd_cand[k] = cand[k];
      r->bwd_ms[k] = ms;
      r->num_bwd = k + 1;
      if (best < 0 || ms < r->bwd_ms[best]) best = k;
    }
    if (st == ETAC_OK) st = build_r3(c, cand[best], s);
  }
  r->bwd_node_range = c->r3_range;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

etac_status etac_pose_grad_to_quat(const float* poses, const float* twist_grad, float* pose_grad,
                                   int64_t count, void* stream) {
  if (!poses || !twist_grad || !pose_grad || count < 0 || !aligned(poses, 4) ||
      !aligned(twist_grad, 4) || !aligned(pose_grad, 4))
    return fail(nullptr, ETAC_ERR_INVALID_ARG, "etac_pose_grad_to_quat: bad argument");
  cudaError_t e = etac::launch_pose_grad_to_quat(poses, twist_grad, pose_grad, (long long)count,
                                                 reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "etac_pose_grad_to_quat");
  return ETAC_OK;
}

etac_status etac_poll_status(etac_ctx* c, int32_t* device_status, void* stream) {
  if (!c || !device_status) return fail(c, ETAC_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  ETAC_CUDA(c, cudaMemcpyAsync(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s),
            "read status");
  ETAC_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s), "clear status");
  ETAC_CUDA(c, cudaStreamSynchronize(s), "read status");
  *device_status = v;
  return ETAC_OK;
}

etac_status etac_forward_f64(etac_ctx* c, const etac_model_desc* desc, const int32_t* obj_type,
                             const double* obj_dims, const double* obj_pose,
                             const double* pad_pose, const double* params, double* disp,
                             void* stream) {
  NvtxScope nvtx_("etac_forward_f64");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!valid_model(desc)) return fail(c, ETAC_ERR_INVALID_ARG, "bad model desc");
  if (!obj_type || !obj_dims || !obj_pose || !pad_pose || !params || !disp ||
      !aligned(obj_dims, 8) || !aligned(obj_pose, 8) || !aligned(pad_pose, 8) ||
      !aligned(params, 8) || !aligned(disp, 8) || !aligned(obj_type, 4))
    return fail(c, ETAC_ERR_INVALID_ARG, "NULL or misaligned pointer");
  if (etac::plain_smem_f64(c->nmax, c->K) > 227 * 1024)
    return fail(c, ETAC_ERR_UNSUPPORTED, "pad type too large for the FP64 check (max ~1500 nodes)");
  etac::PlainArgs<double> a{};
  a.num_nodes = c->N;
  a.type_pos = c->d_type_pos;
  a.type_nrm = c->d_type_nrm;
  a.type_pmax = c->d_type_pmax;
  a.type_off = c->d_type_off;
  a.pad_type = c->d_pad_type;
  a.pad_off = c->d_pad_off;
  a.P = c->P;
  a.K = c->K;
  a.nmax = c->nmax;
  a.obj_type = obj_type;
  a.obj_dims = obj_dims;
  a.obj_pose = obj_pose;
  a.pad_pose = pad_pose;
  a.params = params;
  a.mode = desc->mode;
  a.disp = disp;
  a.status = c->d_status;
  ETAC_CUDA(c, etac::launch_plain_forward<double>(a, c->E * c->P,
                                                  reinterpret_cast<cudaStream_t>(stream)),
            "fp64 forward launch");
  return ETAC_OK;
}

namespace {

// Work of the tensor-core regressor: whole pads to slots (two per CTA, one CTA per SM), the
// longest first, each to the slot with the fewest 128-node tiles so far (LPT).
void build_regress_schedule(etac_ctx* c) {
  const int num_pads = c->E * c->P;
  const int grid = std::max(1, std::min(c->num_sms, (num_pads + 1) / 2));
  const int slots = 2 * grid;
  std::vector<int> tiles(num_pads), order(num_pads);
  for (int p = 0; p < num_pads; ++p) {
    tiles[p] = (c->type_n[c->pad_type[p]] + 127) / 128;
    order[p] = p;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tiles[x] > tiles[y]; });
  using Load = std::pair<long long, int>;   // (tiles so far, slot)
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int s = 0; s < slots; ++s) heap.push({0, s});
  std::vector<std::vector<int>> lists(slots);
  for (int p : order) {
    Load l = heap.top();
    heap.pop();
    lists[l.second].push_back(p);
    heap.push({l.first + tiles[p], l.second});
  }
  std::vector<int>& h = c->reg_sched_h;
  h.assign((size_t)slots + 1 + num_pads + slots, 0);
  int at = 0;
  for (int s = 0; s < slots; ++s) {
    h[s] = at;
    int nt = 0;
    for (int p : lists[s]) {
      h[slots + 1 + at++] = p;
      nt += tiles[p];
    }
    h[slots + 1 + num_pads + s] = nt;
  }
  h[slots] = at;
  c->reg_grid = grid;
}

}  // namespace

etac_status etac_regress(etac_ctx* c, const float* disp, const float* rparams, float* taxels,
                         float* attn, int32_t precision, void* stream) {
  NvtxScope nvtx_("etac_regress");
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (!disp || !rparams || !taxels || !aligned(disp, 4) || !aligned(rparams, 16) ||
      !aligned(taxels, 4) || !aligned(attn, 4))
    return fail(c, ETAC_ERR_INVALID_ARG, "NULL or misaligned pointer");
  if (precision != ETAC_PREC_FP32 && precision != ETAC_PREC_BF16)
    return fail(c, ETAC_ERR_INVALID_ARG, "precision must be ETAC_PREC_FP32 or ETAC_PREC_BF16");
  // layer shapes (out, in) in the order of the flat vector: R1 R2 R3 R4 A1 A2 H1 H2
  static const int dims[8][2] = {{64, 9}, {128, 64}, {256, 128}, {256, 256},
                                 {128, 256}, {1, 128}, {128, 256}, {ETAC_TAXELS, 128}};
  etac::RegArgs a{};
  size_t off = 0;
  for (int l = 0; l < 8; ++l) {
    a.W[l] = rparams + off;
    off += (size_t)dims[l][0] * dims[l][1];
    a.b[l] = rparams + off;
    off += (size_t)dims[l][0];
  }
  if (off != ETAC_REGRESSOR_PARAMS) return fail(c, ETAC_ERR_STATE, "regressor layout mismatch");
  a.type_pos = c->d_type_pos;
  a.type_nrm = c->d_type_nrm;
  a.type_off = c->d_type_off;
  a.pad_type = c->d_pad_type;
  a.pad_off = c->d_pad_off;
  a.num_pads = c->E * c->P;
  a.num_nodes = c->N;
  a.disp = disp;
  a.taxels = taxels;
  a.attn = attn;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == ETAC_PREC_FP32) {
    {
      TimedLaunch tl_(c, K_REG_PLAIN, s);
      ETAC_CUDA(c, etac::launch_regress_plain(a, c->num_sms, s), "regressor launch");
    }
    return ETAC_OK;
  }
  if (!c->d_reg_sched) {
    build_regress_schedule(c);
    ETAC_CUDA(c, dalloc(&c->d_reg_wimg, (size_t)etac::REG_TC_IMAGE_BYTES), "regressor weights");
    ETAC_CUDA(c, dalloc(&c->d_reg_sched, c->reg_sched_h.size()), "regressor schedule");
    ETAC_CUDA(c, cudaMemcpyAsync(c->d_reg_sched, c->reg_sched_h.data(),
                                 c->reg_sched_h.size() * sizeof(int), cudaMemcpyHostToDevice, s),
              "regressor schedule copy");
  }
  const int slots = 2 * c->reg_grid, num_pads = c->E * c->P;
  etac::RegTcArgs t{};
  t.r = a;
  t.wimg = c->d_reg_wimg;
  t.slot_off = c->d_reg_sched;
  t.slot_pads = c->d_reg_sched + slots + 1;
  t.slot_tiles = c->d_reg_sched + slots + 1 + num_pads;
  t.status = c->d_status;
  t.timeout_ns = c->gemm.timeout_ns ? c->gemm.timeout_ns : 2000000000ull;
  {
    TimedLaunch tl_(c, K_REG_PACK, s);
    ETAC_CUDA(c, etac::launch_regress_pack(a, c->d_reg_wimg, s), "regressor weight images");
  }
  {
    TimedLaunch tl_(c, K_REG_TC, s);
    ETAC_CUDA(c, etac::launch_regress_tc(t, c->reg_grid, s), "regressor launch");
  }
  return ETAC_OK;
}

etac_status etac_enable_timing(etac_ctx* c, int32_t enable) {
  if (!c) return fail(nullptr, ETAC_ERR_INVALID_ARG, "ctx is NULL");
  if (enable && c->ev.empty()) {
    c->ev.assign(2 * ETAC_TIMING_SLOTS, nullptr);
    c->ev_kernel.assign(ETAC_TIMING_SLOTS, 0);
    for (auto& e : c->ev) ETAC_CUDA(c, cudaEventCreate(&e), "create timing events");
  }
  c->timing = enable != 0;
  c->ev_used = 0;
  return ETAC_OK;
}

etac_status etac_kernel_times(etac_ctx* c, etac_kernel_time* out, int32_t max, int32_t* count) {
  if (!c || !count || (max > 0 && !out)) return fail(c, ETAC_ERR_INVALID_ARG, "NULL argument");
  ETAC_CUDA(c, cudaDeviceSynchronize(), "synchronise for timing");
  int launches[K_COUNT] = {0};
  double total[K_COUNT] = {0};
  for (int i = 0; i < c->ev_used; ++i) {
    float ms = 0.f;
    ETAC_CUDA(c, cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]), "event time");
    launches[c->ev_kernel[i]] += 1;
    total[c->ev_kernel[i]] += ms;
  }
  int n = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (!launches[k]) continue;
    if (n < max) {
      memset(&out[n], 0, sizeof(out[n]));
      snprintf(out[n].name, sizeof(out[n].name), "%s", kKernelNames[k]);
      out[n].launches = launches[k];
      out[n].total_ms = (float)total[k];
    }
    ++n;
  }
  *count = n < max ? n : max;
  c->ev_used = 0;
  return ETAC_OK;
}

const char* etac_last_error(const etac_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

void etac_destroy(etac_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  free_ctx(c);
}

}  // extern "C"
