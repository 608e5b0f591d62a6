// etac_kernels.h -- launch interfaces between the C-ABI host code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "etac_common.cuh"

struct etac_mesh_gpu;

namespace etac {

// device view of a mesh made by etac_mesh_gpu_create (mesh_query.cu)
void mesh_dev_view(const etac_mesh_gpu* g, MeshDev* d);

// ---------------------------------------------------------------- plain algorithm
template <typename T>
struct PlainArgs {
  const float* type_pos;      // [sum n, 3]
  const float* type_nrm;      // [sum n, 3]
  const float* type_pmax;     // [T] max |p| per pad type
  const int* type_off;        // [T+1] node offsets of pad types
  const int* pad_type;        // [E*P]
  const long long* pad_off;   // [E*P+1] node offsets of pad instances
  int P, K, nmax;
  const int* obj_type;
  const T* obj_dims;
  const T* obj_pose;
  const T* pad_pose;
  const T* params;            // flat parameter vector
  int mode;
  T* disp;
  uint8_t* mask;              // optional
  T* pen;                     // optional
  int* count;                 // optional
  int* status;                // device status word
  long long num_nodes;         // nodes of all pad instances (index checks of the bounds build)
  const uint8_t* mask_in;     // mode B (both or neither): caller's active set [N] and
  const float* uhat_in;       //   u_hat [N*3]; objects are then not read (FP32 only)
  const MeshDev* meshes;      // the context's meshes (OBJ_MESH objects), may be null
  int num_meshes;
};

template <typename T>
cudaError_t launch_plain_forward(const PlainArgs<T>& a, int num_pads, cudaStream_t stream);
size_t plain_smem_f32(int nmax, int K);
size_t plain_smem_f64(int nmax, int K);

}  // namespace etac

namespace etac {

// ---------------------------------------------------------------- per-type tables
struct TablesArgs {
  const float* type_pos;
  const float* type_nrm;
  const int* type_off;          // [T+1]
  const long long* omega_off;   // [T+1] element offsets of each type's n x n Omega
  int num_types, total_nodes;
  const float* params;
  float* ctab;                  // [sum n][64]
  float* f0tab;                 // [sum n][64]
  float* h0tab;                 // [sum n][64]
  int16_t* order;               // [64 * sum n]: type t at 64*type_off[t], channel-major
  float* omega;                 // [sum n^2] FP32 (optional)
  void* omega_bf16;             // [sum n^2] BF16 (optional)
  void* h0bf16;                 // [sum n][64] BF16 copy of h0 (optional)
  float2* ranked;               // [64 * sum n] (f0 value, node as int bits) in rank order (optional)
  // reverse mode of the batched algorithms (optional): Omega and d * Omega split into BF16
  // hi and lo parts
  void* om_hi;
  void* om_lo;
  void* dom_hi;
  void* dom_lo;
  const int* skip;              // optional: when *skip != 0 the kernels return at once
};
cudaError_t launch_tables(const TablesArgs& a, int nmax, cudaStream_t s);

// ---------------------------------------------------------------- batched FP32 forward
struct BatchedArgs {
  const float* type_pos;
  const float* type_nrm;
  const float* type_pmax;
  const int* type_off;
  const long long* omega_off;
  const int* pad_type;
  const long long* pad_off;
  const int* item_pad;          // pad instance of each work item, heaviest first
  int num_items, P, K, nmax;
  const int* obj_type;
  const float* obj_dims;
  const float* obj_pose;
  const float* pad_pose;
  const float* params;
  const float* ctab;
  const float* f0tab;
  const float* h0tab;
  const int16_t* order;
  const float* omega;
  int mode;
  float* disp;
  uint8_t* mask;
  float* pen;
  int* count;
  int* ticket;                  // work-queue counter, zero at launch
  int* status;
  long long num_nodes;         // nodes of all pad instances (index checks of the bounds build)
  const int* skip;              // optional: when *skip != 0 the kernel returns at once
  const uint8_t* mask_in;       // mode B: caller's active set [N] and u_hat [N*3]
  const float* uhat_in;
  float* g0rec;                 // optional [E*P][64]: each pad's max-pooled feature g0 and
  int* g0arg;                   //   its lowest-index maximising node (for the reverse mode)
  const MeshDev* meshes;        // the context's meshes (OBJ_MESH objects), may be null
  int num_meshes;
};
cudaError_t launch_batched_forward(const BatchedArgs& a, int grid, cudaStream_t s);

// ---------------------------------------------------------------- BF16 front kernels
struct FrontArgs {
  const float* type_pos;
  const float* type_nrm;
  const float* type_pmax;
  const int* type_off;
  const int* pad_type;
  const long long* pad_off;
  const int* item_pad;
  int num_items, P, K, nmax;
  const int* obj_type;
  const float* obj_dims;
  const float* obj_pose;
  const float* pad_pose;
  const float* params;
  const float* ctab;
  const float* f0tab;
  const int16_t* order;
  const float2* ranked;         // per type and channel: (f0, node) in descending f0 order
  int mode;
  float* disp;
  uint8_t* mask;
  float* pen;
  int* count;
  int* ticket;
  int* status;
  long long num_nodes;         // nodes of all pad instances (index checks of the bounds build)
  long long bt_total;          // B-operand entries (BF16) of all types
  long long mask_words;        // contact-bit words of all pads
  void* bt;                     // BF16 B operand, type t at bt_off[t]: [3 * I_t][n_t]
  const long long* bt_off;
  const int* pad_inst;
  uint32_t* maskbits;
  const long long* mask_woff;
  int* pad_m;                   // [E*P] active count
  float* g0a;                   // [E*P][64] max-pooled global feature g0 of each pad
  const int* pad_gi;            // [E*P] global instance index (type's first instance + k)
  void* negbeta;                // [sum I_t][64] BF16 in MMA-fragment word order (by instance)
  float4* c0m;                  // [sum I_t] by instance
  PadObj* padobj;               // [E*P][K] pad -> object transforms
  int* pad_bad;                 // [E*P] 1 when a pose or size held NaN / Inf
  const uint8_t* mask_in;       // mode B: caller's active set [N] and u_hat [N*3]
  const float* uhat_in;
  const int16_t* blk_perm;      // [sum n] nodes of each type in block order (32 per block)
  const float* blk_pos;         // [sum n, 3] positions and normals in that order
  const float* blk_nrm;
  const float4* blk_sphere;     // [sum nb] block bounding spheres: centroid, radius
  const int* type_boff;         // [T] first block of each type
  uint32_t* btbits;             // nodes whose B-operand entries are nonzero (mask_woff layout)
  const MeshDev* meshes;        // the context's meshes (OBJ_MESH objects), may be null
  int num_meshes;
};
size_t front_smem_bytes(int nmax, int K);
cudaError_t launch_pad_obj(const FrontArgs& a, cudaStream_t s);
cudaError_t front_occupancy(int nmax, int K, int* blocks_per_sm);
cudaError_t launch_front_contact(const FrontArgs& a, int grid, cudaStream_t s);
cudaError_t launch_front_global(const FrontArgs& a, int num_sms, cudaStream_t s);

size_t batched_smem_bytes(int nmax, int K, bool otf = false);
int batched_threads();
cudaError_t batched_occupancy(int nmax, int K, bool otf, int* blocks_per_sm);

}  // namespace etac

#include <cuda.h>

namespace etac {

// ---------------------------------------------------------------- BF16 propagation GEMM
constexpr int GEMM_MAX_TYPES = 16;

struct GemmTile {
  int type, m0, k0, nkb;   // pad type, first node row, first instance, K blocks of 64 nodes
};

struct GemmParams {
  CUtensorMap tmA[GEMM_MAX_TYPES];   // Omega_t BF16 [n_t][n_t], box 64 x 128, 128B swizzle
  CUtensorMap tmB[GEMM_MAX_TYPES];   // B_t BF16 [3 I_t][n_t], box 64 x 192, 128B swizzle
  // reverse modes only: the low BF16 parts (A: Omega_t or d * Omega_t, B: dL/dU of passive
  // nodes); the K loop runs the segments (A hi, B hi), (A hi, B lo), (A lo, B hi)
  CUtensorMap tmA2[GEMM_MAX_TYPES];
  CUtensorMap tmB2[GEMM_MAX_TYPES];
  const GemmTile* tiles;
  int num_tiles;
  const int* type_off;               // [T+1]
  const int* inst_off;               // [T+1]
  const int* inst_pad;               // [sum I_t] pad index of instance k of type t
  const long long* pad_off;
  const void* h0bf16;                // [sum n][64]
  const void* negbeta;               // [sum I_t][64] BF16 by instance, MMA-fragment word order
  const float4* c0m;                 // [sum I_t] (D2 beta + b_D2, m) by instance
  const long long* inst_base;        // [sum I_t] first node of each instance's pad
  const uint32_t* maskbits;          // contact bits, instance order: type t, instance k at
  const long long* type_woff;        //   type_woff[t] + k * ceil(n_t / 32)
  const float* params;
  float* disp;
  int use_l, use_r;
  int* status;
  long long num_nodes;         // nodes of all pad instances (index checks of the bounds build)
  unsigned long long timeout_ns;
  // failure-path tests only: 1 + the tile whose first K block the producer withholds (its
  // TMA loads are never issued, so the MMA issuer's bounded wait runs out); 0 = off
  int test_withhold;
  // reverse modes
  const int* inst_m;                 // [sum I_t] active count by instance
  const float4* ws_u;                // [N] (u_hat, phi) of active nodes
  float4* ws_du;                     // [N] dL/du_hat of active nodes (accumulated into)
  float* alpha_part;                 // [grid] per-CTA sums of u_hat . (d Omega G)
};

enum { GEMM_FWD = 0, GEMM_BWD_U = 1, GEMM_BWD_ALPHA = 2 };
// gi: instances per tile (32 or 64; the tile list and B-operand tensor maps must match)
cudaError_t launch_prop_gemm(const GemmParams& p, int grid, cudaStream_t s, int mode, int gi);
size_t prop_gemm_smem_bytes();

}  // namespace etac

namespace etac {

// ---------------------------------------------------------------- reverse mode (FP32)
struct BackwardArgs {
  const float* type_pos;
  const float* type_nrm;
  const float* type_pmax;
  const int* type_off;
  const int* pad_type;
  const long long* pad_off;
  const int* item_pad;
  int num_items, E, P, K, nmax;
  const int* obj_type;
  const float* obj_dims;
  const float* obj_pose;
  const float* pad_pose;
  const float* params;
  const float* ctab;
  const float* f0tab;
  const float* h0tab;
  const int16_t* order;
  const float2* ranked;        // per type and channel: (f0, node) in descending f0 order
  int mode;
  const float* grad_disp;      // [N*3]
  float* grad_uhat;            // [N*3] or null
  float* grad_pen;             // [N] or null
  float* grad_params;          // [NPARAM] or null
  float* grad_obj_pose;        // [E*K*6] or null
  int* ws_idx;                 // [N] active lists (per pad at its node offset)
  float4* ws_u;                // [N]
  float4* ws_du;               // [N]
  float* pose_part;            // [E*P*K*6]
  float* param_part;           // [grid * NPARAM]
  const uint8_t* mask_in;      // mode B: the forward's caller-supplied active set and u_hat
  const float* uhat_in;
  const MeshDev* meshes;       // the context's meshes (OBJ_MESH objects), may be null
  int num_meshes;
};
size_t backward_smem_bytes(int nmax, int K);
cudaError_t launch_backward(const BackwardArgs& a, int grid, cudaStream_t s);
cudaError_t launch_pose_grad_to_quat(const float* poses, const float* tw, float* out,
                                     long long count, cudaStream_t s);
cudaError_t launch_reduce_pose(const float* part, int E, int P, int K, float* out, cudaStream_t s);

// ---------------------------------------------------------------- batched reverse mode (FP32)
// per-pad records of the staged reverse mode (floats; PR_ROUTE holds int bits)
constexpr int PR_G0 = 0, PR_AG = 64, PR_G = 128, PR_BETA = 192, PR_S = 256, PR_DAG = 320,
              PR_ROUTE = 384, PR_GSUM = 448, PR_D = 452, PR_SLOT = 516, PR_X = 580,
              PR_STRIDE = PR_X + 64 * 9 + 4;

struct R3Group {
  int type, k0;        // pad type, first instance of the 64-instance group
  int i0, i1;          // node range of this work unit
  int srange;          // index of the node range within the type
  long long a3off;     // float offset of the group's A3 partial block [n_t][64]
};
constexpr int R3_RANGE = 256;   // nodes per decoder-reverse work unit (at most; host picks)

struct BwdBatchedArgs {
  const float* type_pos;
  const float* type_nrm;
  const int* type_off;
  const int* pad_type;
  const long long* pad_off;
  const int* item_pad;
  int num_items, P, K, nmax, total_nodes;
  const float* pad_pose;
  const float* obj_pose;
  const float* params;
  const float* ctab;
  const float* f0tab;
  const float* h0tab;
  const float2* ranked;
  const PadObj* padobj;
  const int* pad_bad;
  const int* pad_inst;
  const int* inst_off;
  const int* inst_pad;
  const int* pad_gi;
  const long long* inst_base;
  const long long* type_woff;
  const long long* mask_woff;
  uint32_t* maskbits;
  const long long* bg_off;     // [T] element offset of each type's [3 I_t][n_t] block
  void* bg_hi;                 // passive dL/dU, BF16 hi part, propagation-reverse B operand
  void* bg_lo;                 // the BF16 remainders
  int mode;
  const float* grad_disp;
  float* grad_uhat;
  float* grad_pen;
  float4* ws_u;                // [N] (u_hat, phi) of active nodes
  float4* ws_du;               // [N] dL/du_hat of active nodes
  float* pr;                   // [E*P][PR_STRIDE]
  int* pad_m;
  int* inst_m;                 // [sum I_t] active count by instance
  const R3Group* r3_groups;
  int r3_parts;
  float* a3part;
  const long long* a3_toff;    // [T] float offset of type t's first group block
  const int* a3_tgroups;       // [T] groups of type t
  float* spart;                // dL/dbeta partials per (node range, instance) [.][64]
  const long long* s_toff;     // [T] first partial row of type t (rows: range-major, then instance)
  const int* s_nr;             // [T] node ranges of type t
  float* a3;                   // [sum n][64]
  float* d2part;               // [r3_parts][3 * 64]
  float* r4part;
  int r4_parts;
  float* r4bpart;
  int r4b_parts;
  float* gsum_part;            // [r4b_parts][3] sums of G over passive nodes per pad chunk
  float* r5part;
  int r5_parts;
  float* alpha_part;
  int alpha_parts;
  float* pose_part;
  int* ticket;
  const uint8_t* mask_in;      // mode B: the forward's caller-supplied active set and u_hat
  const float* uhat_in;
  const float* g0rec;          // the forward's recorded g0 and maximising nodes [E*P][64], or
  const int* g0arg;            //   null: R1 recomputes the active nodes' encoder
  int has_meshes;               // the context has mesh objects (selects the kernels' build)
};
struct BwdBatchedLaunch {
  int r1_grid, r2_grid, r7_grid;
};
size_t bwd_pad_smem_bytes(int nmax, int K);
cudaError_t bwd_pad_occupancy(int nmax, int K, int* blocks_per_sm);
enum { BWD_STAGE_PAD = 0, BWD_STAGE_GLOBAL, BWD_STAGE_DECODER, BWD_STAGE_A3SUM,
       BWD_STAGE_PADREV, BWD_STAGE_PADSUM, BWD_STAGE_TYPENODE, BWD_STAGE_POSE,
       BWD_STAGE_PARAMS };
cudaError_t launch_backward_stage(const BwdBatchedArgs& a, const BwdBatchedLaunch& l, int stage,
                                  float* grad_params, cudaStream_t s);

}  // namespace etac

namespace etac {

// ---------------------------------------------------------------- taxel regressor
struct RegArgs {
  const float* type_pos;      // [sum n, 3]
  const float* type_nrm;      // [sum n, 3]
  const int* type_off;        // [T+1]
  const int* pad_type;        // [E*P]
  const long long* pad_off;   // [E*P+1]
  int num_pads;
  const float* disp;          // [N, 3] pad frame
  const float* W[8];          // R1, R2, R3, R4, A1, A2, H1, H2 (row-major, out x in)
  const float* b[8];
  float* taxels;              // [E*P, 8]
  float* attn;                // [N] softmax weights (optional)
  long long num_nodes;        // N (index checks of the bounds build)
};

cudaError_t launch_regress_plain(const RegArgs& a, int num_sms, cudaStream_t s);

// Tensor-core regressor (regress_tc.cu).  Slot s (two per CTA) runs the encoder over the pads
// slot_pads[slot_off[s] .. slot_off[s + 1]) in order; slot_tiles[s] is their number of
// 128-node tiles.  wimg holds the BF16 weight images of the five per-node layers
// (REG_TC_IMAGE_BYTES, written by launch_regress_pack).
constexpr int REG_TC_IMAGE_BYTES = 286720;
struct RegTcArgs {
  RegArgs r;
  const unsigned char* wimg;
  const int* slot_off;        // [num_slots + 1]
  const int* slot_pads;       // [num_pads]
  const int* slot_tiles;      // [num_slots]
  int* status;
  unsigned long long timeout_ns;
};
cudaError_t launch_regress_pack(const RegArgs& a, unsigned char* wimg, cudaStream_t s);
cudaError_t launch_regress_tc(const RegTcArgs& a, int grid, cudaStream_t s);
size_t regress_tc_smem_bytes();

}  // namespace etac
