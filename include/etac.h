/*
 * etac.h -- C ABI of the GB300 (sm_103a) ETac tactile step library (libetac.so).
 *
 * ETac (Sec. III-A) simulates elastomer tactile pads: every surface node of every pad is
 * tested against the environment's rigid objects with signed distance fields; nodes inside
 * an object are "active" and take a local displacement u_hat; every other ("passive") node
 * gets the decay-based propagation of Eq. 1 (Omega U_a) plus the PointNet residual Phi_p of
 * Sec. III-A 2, summed as in Eq. 4.  This library runs that step for a whole batch of
 * environments on one GPU, and its reverse mode.
 *
 * Conventions shared by every entry point:
 *   - millimetres; quaternions are (x, y, z, w) and need not be normalised; a pose is
 *     t(3) followed by q(4), 7 floats;
 *   - a pad type is a fixed set of n surface nodes with undeformed positions P and unit
 *     normals N in the pad frame; node order within a pad is the caller's (row-major grids);
 *   - pad instances are env-major, pad-minor; the flat node index of node i of pad instance
 *     p is offset[p] + i, offset being the prefix sum of the instances' node counts;
 *   - displacements are returned in the pad frame of their pad (undeformed frame, Sec. III-A);
 *   - "host" pointers are read during the call only; "device" pointers are borrowed: they
 *     must stay valid, and untouched by other work, until the work enqueued on the given
 *     stream has completed.  Nothing is retained after the call returns except where stated;
 *   - every call returns an etac_status; on failure etac_last_error() describes it.  Calls
 *     that enqueue GPU work never synchronise; conditions found on the GPU (bounded waits
 *     that ran out, non-finite poses) are latched in a device status word read with
 *     etac_poll_status().
 *   - a context is not thread-safe; use one context per stream.
 */
#ifndef ETAC_H_
#define ETAC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ETAC_HIDDEN 64          /* hidden width of every network layer (global feature: 64) */
#define ETAC_MAX_OBJECTS 8      /* rigid objects per environment                            */
#define ETAC_MAX_PAD_NODES 4096 /* nodes per pad type                                       */

typedef enum {
  ETAC_OK = 0,
  ETAC_ERR_INVALID_ARG = 1,  /* bad pointer, size, alignment or value                      */
  ETAC_ERR_STATE = 2,        /* call out of order (e.g. step before set_model)             */
  ETAC_ERR_CUDA = 3,         /* a CUDA call failed; the context should be destroyed        */
  ETAC_ERR_OOM = 4,          /* device allocation failed                                   */
  ETAC_ERR_TIMEOUT = 5,      /* device status: a bounded wait gave up                      */
  ETAC_ERR_NONFINITE = 6,    /* device status: a pose held NaN / Inf (those pads output 0) */
  ETAC_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement               */
  ETAC_ERR_BOUNDS = 8        /* device status, ETAC_BOUNDS build only: an index check failed
                                (the access was skipped)                                    */
} etac_status;

enum { ETAC_OBJ_NONE = 0, ETAC_OBJ_SPHERE = 1, ETAC_OBJ_BOX = 2, ETAC_OBJ_CYLINDER = 3,
       ETAC_OBJ_CAPSULE = 4, ETAC_OBJ_MESH = 5 };

/* which terms of Eq. 4 are evaluated (the ablations of Table II): both, the decay propagation
 * of Eq. 1 alone, the residual network alone, or neither (penetration only: active nodes take
 * u_hat and passive nodes stay at zero, the propagation-free baseline the paper compares with) */
enum { ETAC_MODE_FULL = 0, ETAC_MODE_LINEAR_ONLY = 1, ETAC_MODE_RESIDUAL_ONLY = 2,
       ETAC_MODE_PENETRATION_ONLY = 3 };

/* arithmetic of the dense contractions: FP32, or BF16 operands with FP32 accumulation */
enum { ETAC_PREC_FP32 = 0, ETAC_PREC_BF16 = 1 };

/* ETAC_ALGO_PLAIN: one CTA per pad, Eq. 1 / Eq. 4 evaluated literally on every node with the
 * exponential computed per pair (the unoptimised reference form).
 * ETAC_ALGO_BATCHED: one persistent launch over all pads, per-pad-type tables, the network
 * factored through the passive nodes' constant inputs, FP32 or BF16 contractions. */
enum { ETAC_ALGO_PLAIN = 0, ETAC_ALGO_BATCHED = 1 };

typedef struct etac_ctx etac_ctx;   /* opaque, owned by the library */

/* Pads of the whole batch (host arrays, read during etac_create_pads only). */
typedef struct {
  int32_t num_types;               /* >= 1                                                 */
  const int32_t* type_num_nodes;   /* [num_types], each in [1, ETAC_MAX_PAD_NODES]          */
  const float* type_pos;           /* [sum n, 3] undeformed positions, pad frame (mm)       */
  const float* type_nrm;           /* [sum n, 3] unit outward normals, pad frame            */
  int32_t num_envs;                /* >= 1                                                 */
  int32_t pads_per_env;            /* >= 1                                                 */
  const int32_t* pad_type;         /* [num_envs * pads_per_env], each in [0, num_types)     */
  int32_t max_objects;             /* K, objects per environment, in [1, ETAC_MAX_OBJECTS]  */
} etac_pads_desc;

/* Propagation model configuration.  Parameters are one flat FP32 vector (etac_param_count
 * floats): alpha (1/mm, > 0), then for each layer W (row-major, out x in) followed by b, in
 * the order E1 (9->64), E2 (64->64), G1 (64->64), D1 (128->64, input [f_i ; g]),
 * D2 (64->3).  Activations are ReLU except after D2. */
typedef struct {
  int32_t hidden;      /* must be ETAC_HIDDEN                                              */
  int32_t mode;        /* ETAC_MODE_*                                                      */
  int32_t precision;   /* ETAC_PREC_*                                                      */
  int32_t algo;        /* ETAC_ALGO_*                                                      */
} etac_model_desc;

/* Per-step inputs (device pointers, borrowed).
 *
 * Mode A (active_mask_in and active_disp_in NULL): the library finds the contact itself, with
 * the SDFs of the env's objects (Sec. III-A "Overview"); the four object / pad arrays are
 * required.
 * Mode B (both given): the caller supplies the contact result of an external pipeline (a mesh
 * or FEM contact solver, recorded data): the active set and the active nodes' local
 * displacements u_hat, which are the propagation input U_a of Eq. 1 and Eq. 4.  No SDF is
 * evaluated and the object / pad arrays are not read (they may be NULL); the penetration
 * output reads 0 for every node; in the reverse mode dL/du_hat is the gradient with respect
 * to active_disp_in, and the object-pose and penetration gradients are zero.  The reverse mode
 * of a mode-B step reads these two buffers again: they are retained (borrowed) until the
 * step's etac_step_backward has been enqueued, and must not change before then.  Giving only
 * one of the two is ETAC_ERR_INVALID_ARG. */
typedef struct {
  const int32_t* obj_type;   /* [E*K] ETAC_OBJ_*; ETAC_OBJ_NONE slots are ignored           */
  const float* obj_dims;     /* [E*K*3] sphere (r,-,-); box half-extents (hx,hy,hz);
                                cylinder / capsule (r, half-length along local z, -);
                                mesh (index among etac_set_meshes' meshes, -, -)           */
  const float* obj_pose;     /* [E*K*7] world pose of each object                           */
  const float* pad_pose;     /* [E*P*7] world pose of each pad instance                     */
  const float* active_disp_in;     /* mode B: [N*3] u_hat of active nodes, pad frame (mm);
                                      entries of passive nodes are ignored                  */
  const uint8_t* active_mask_in;   /* mode B: [N] nonzero = active                         */
} etac_step_in;

/* Per-step outputs (device pointers, borrowed; NULL = not wanted, except disp). */
typedef struct {
  float* disp;               /* [N*3] node displacement, pad frame (required)               */
  uint8_t* active_mask;      /* [N] 1 if the node is in contact                             */
  float* penetration;        /* [N] max(0, -signed distance)                                */
  int32_t* active_count;     /* [E*P] active nodes per pad (the n_a of the contact reward)  */
} etac_step_out;

/* Number of floats in the flat parameter vector for this configuration (0 if invalid). */
size_t etac_param_count(const etac_model_desc* desc);

/* Total node count N of a pad description (0 if invalid). */
int64_t etac_total_nodes(const etac_pads_desc* desc);

/* Create a context for a fixed batch of pads: the surface nodes P and their normals N of
 * every pad type (Sec. III-A: the sensor skin's node set, undeformed, pad frame) and the type
 * of each pad instance.  Copies the geometry to the device and allocates every buffer a later
 * step needs (steps never allocate).  `stream` orders the copies.  On success *out owns
 * device memory until etac_destroy. */
etac_status etac_create_pads(etac_ctx** out, const etac_pads_desc* desc, void* stream);

/* Set (or replace) the propagation model: the decay rate alpha of Eq. 1 and the residual
 * network of Sec. III-A 2 (encoder, max-pool, global MLP, decoder; Eq. 4 sums the two terms).
 * `params` is a device FP32 vector of etac_param_count(desc) floats, copied on `stream` (the
 * caller may reuse it once the call returns).  Synchronises `stream` once to validate alpha (finite and > 0, else
 * ETAC_ERR_INVALID_ARG and the previous model stays).  Rebuilds the per-pad-type tables of
 * the batched algorithm.  Not capturable in a CUDA graph. */
etac_status etac_set_model(etac_ctx* ctx, const etac_model_desc* desc, const float* params,
                           void* stream);

/* Closed triangle meshes for ETAC_OBJ_MESH objects (ETac Sec. III-A "Overview": contact by
 * signed distance between the nodes and object meshes).  `meshes` [count] are device meshes
 * from etac_mesh_gpu_create (declared below); an object of type ETAC_OBJ_MESH names one by
 * its index in obj_dims[0] (an index outside [0, count) leaves the slot empty).  The meshes
 * are borrowed: they must outlive every step that uses them.  Replaces the previous list;
 * count 0 clears it.  Copies a small table to the device and synchronises `stream`; not
 * capturable.  The FP32 screen and the FP32 path for nodes certainly inside use the mesh's
 * grid and candidate lists (Voronoi-region nearest points, pseudo-normal sign); nodes within
 * a few um of the surface, or with two nearly equal nearest triangles, take the decision
 * and u_hat in FP64.  The FP64 finite-difference evaluation (etac_forward_f64) treats mesh
 * slots as empty.  Errors: ETAC_ERR_INVALID_ARG (NULL ctx, count < 0, a NULL mesh),
 * ETAC_ERR_OOM, ETAC_ERR_CUDA. */
typedef struct etac_mesh_gpu etac_mesh_gpu;
etac_status etac_set_meshes(etac_ctx* ctx, const etac_mesh_gpu* const* meshes, int32_t count,
                            void* stream);

/* One forward step (ETac Sec. III-A, Eq. 1 and Eq. 4) for every pad of the batch.  Enqueues
 * work on `stream` only (no host synchronisation, no allocation), so it can be captured in
 * a CUDA graph.  Pads whose env has no object in contact output zero displacement.  Keeps
 * a device copy of the poses for etac_step_backward. */
etac_status etac_step_forward(etac_ctx* ctx, const etac_step_in* in, const etac_step_out* out,
                              void* stream);

/* Id of the last etac_step_forward enqueued on this context: 1 for the first, then 2, 3, ...
 * (0 before any).  Host-side bookkeeping: no GPU work. */
etac_status etac_last_step(const etac_ctx* ctx, uint64_t* step_id);

/* Reverse mode (FP32, hand-written) of the forward step `step_id` on this context (the id
 * etac_last_step gave right after that forward).  The context keeps the saved state of its
 * last forward only, so any other id is refused with ETAC_ERR_STATE (nothing is enqueued):
 * a caller that ran several forwards before differentiating them must re-run the one it
 * differentiates.  step_id = 0 means "the last forward", unchecked.
 * grad_disp [N*3] is dL/d(disp).  Outputs are overwritten (not accumulated); any may be
 * NULL: grad_obj_pose [E*K*6] = (dL/dt world, dL/d omega) with the rotation increment
 * exp([omega]x) applied on the left about the object origin; grad_uhat [N*3] = dL/d u_hat of
 * active nodes (pad frame, 0 on passive nodes); grad_penetration [N] = dL/d(penetration)
 * with u_hat = penetration * outward normal (0 on passive nodes); grad_params [P] for the
 * flat parameter vector.  The contact set is held fixed.  ETAC_ERR_STATE without a prior
 * forward. */
etac_status etac_step_backward(etac_ctx* ctx, uint64_t step_id, const float* grad_disp,
                               float* grad_obj_pose, float* grad_uhat, float* grad_penetration,
                               float* grad_params, void* stream);

/* Chain rule from the pose gradient of etac_step_backward to the 7-float pose layout: given
 * poses [count*7] (t, q) and their twist gradients [count*6] (dL/dt, dL/d omega with the
 * left world-frame rotation increment), writes dL/d(pose) [count*7], where the quaternion
 * part is the gradient with respect to the raw (not normalised) quaternion components.
 * Device pointers; enqueued on `stream`. */
etac_status etac_pose_grad_to_quat(const float* poses, const float* twist_grad, float* pose_grad,
                                   int64_t count, void* stream);

/* ---- Failure-path test hook (the paper has no counterpart; for tests only).
 * Every wait inside the library's kernels is bounded: a wait that runs out latches
 * ETAC_ERR_TIMEOUT in the device status word, and the kernel winds down (it waits, bounded,
 * for its own copies and tensor-core operations in flight and frees its tensor memory) and
 * returns, leaving the context usable.  This hook lets a test make such a wait run out
 * without any fault: for the following forward steps of a batched BF16 model, the
 * propagation GEMM's load producer does not issue the loads of the first K block of GEMM
 * tile `tile` (nothing else is loaded by that CTA), so its MMA issuer's wait on them gives up
 * after `wait_limit_ns` (0: the default 2 s; at most 2 s); the pads of that CTA's tiles are
 * left unwritten.  tile = -1 turns the hook off and restores the default limit.
 * ETAC_ERR_STATE without a batched BF16 model; ETAC_ERR_INVALID_ARG for a tile outside
 * [-1, number of tiles) or a limit above 2 s. */
etac_status etac_test_withhold_load(etac_ctx* ctx, int32_t tile, uint64_t wait_limit_ns);

/* Reads and clears the device status word (synchronises `stream`).  *device_status receives
 * ETAC_OK or the first latched ETAC_ERR_TIMEOUT / ETAC_ERR_NONFINITE (or, in the ETAC_BOUNDS
 * build, ETAC_ERR_BOUNDS). */
etac_status etac_poll_status(etac_ctx* ctx, int32_t* device_status, void* stream);

/* ---- Per-kernel timing (profiling aid; the paper has no counterpart).
 * When enabled, every later step records a CUDA event pair on its stream around each kernel
 * it launches (at most ETAC_TIMING_SLOTS launches are kept until read).  etac_kernel_times
 * synchronises the device, writes up to `max` entries (kernel name, launches, summed
 * milliseconds) and clears the record.  Enabling creates events (do it outside any stream
 * capture); timing adds event records to captured graphs. */
#define ETAC_TIMING_SLOTS 4096
typedef struct {
  char name[48];
  int32_t launches;
  float total_ms;
} etac_kernel_time;
etac_status etac_enable_timing(etac_ctx* ctx, int32_t enable);
etac_status etac_kernel_times(etac_ctx* ctx, etac_kernel_time* out, int32_t max, int32_t* count);

/* ---- Tile and block shapes picked by measurement (the paper has no counterpart).
 * gemm_inst_per_tile: pad instances per tile of the BF16 propagation GEMM (32, 64 or 80; the
 * tile is 128 node rows x 3 * that many columns); gemm_tile_order: 0 walks node-row tiles
 * innermost (tiles running together share a B tile in L2), 1 walks instance groups
 * innermost (they share an Omega row block); bwd_node_range: nodes per work unit of the
 * batched reverse mode's decoder stage (16..256, a multiple of 16); front_ctas_per_sm: CTAs
 * per SM of the BF16 step's persistent contact / encoder kernel (1 .. the occupancy maximum,
 * which is also what 0 selects); omega_source: where the batched FP32 step takes Omega
 * (ETAC_OMEGA_*, below; etac_autotune times the table against on the fly when the table fits).
 *
 * etac_autotune times every candidate on the caller's own step: the forward shapes
 * (ETAC_ALGO_BATCHED with ETAC_PREC_BF16: GEMM tiles, then the front kernel's CTAs per SM)
 * on `in` / `out`, and, when grad_disp is not NULL,
 * the reverse-mode node ranges on that upstream gradient [N*3].  It leaves the fastest
 * choice in effect, writes the candidates and their milliseconds per step to *result
 * (host), synchronises `stream`, and overwrites `out`.  Not to be called during stream
 * capture.  etac_set_tuning applies a stored choice (fields that do not apply to the
 * model's algorithm are ignored).  Both may grow the GEMM tile list and the reverse mode's
 * work-unit list (device memory) for a new shape; steps never allocate.  Errors:
 * ETAC_ERR_STATE without a batched model, ETAC_ERR_INVALID_ARG for NULL in/out/result or
 * out-of-range fields, ETAC_ERR_OOM if that growth fails. */
#define ETAC_TUNE_MAX 8
typedef struct {
  int32_t gemm_inst_per_tile;
  int32_t gemm_tile_order;
  int32_t bwd_node_range;
  int32_t num_fwd;                     /* forward candidates timed */
  int32_t fwd_cand[ETAC_TUNE_MAX][2];  /* (instances per tile, tile order) */
  float fwd_ms[ETAC_TUNE_MAX];
  int32_t num_bwd;                     /* reverse-mode candidates timed */
  int32_t bwd_cand[ETAC_TUNE_MAX];     /* node range */
  float bwd_ms[ETAC_TUNE_MAX];
  int32_t front_ctas_per_sm;
  int32_t num_front;                   /* front-kernel candidates timed */
  int32_t front_cand[ETAC_TUNE_MAX];   /* CTAs per SM */
  float front_ms[ETAC_TUNE_MAX];
  int32_t omega_source;                /* ETAC_OMEGA_* (batched FP32 only) */
  float omega_ms[2];                   /* forward ms with the table, on the fly (0: not timed) */
} etac_tuning;
/* Source of Omega (Eq. 1) in the batched FP32 step: AUTO takes the per-type table when all
 * tables together fit in 4 GiB (otherwise, e.g. for pads of per-instance geometry, the kernel
 * evaluates exp(-alpha |p_j - p_i|) on the fly, with the table's own FP32 expression, so both
 * give the same bits); TABLE insists on the table (ETAC_ERR_UNSUPPORTED when too large);
 * ON_THE_FLY never builds it. */
enum { ETAC_OMEGA_AUTO = 0, ETAC_OMEGA_TABLE = 1, ETAC_OMEGA_ON_THE_FLY = 2 };
etac_status etac_autotune(etac_ctx* ctx, const etac_step_in* in, const etac_step_out* out,
                          const float* grad_disp, etac_tuning* result, void* stream);
etac_status etac_set_tuning(etac_ctx* ctx, const etac_tuning* tuning, void* stream);

/* FP64 evaluation of the plain algorithm, for finite-difference gradient checks only.
 * Device arrays as in etac_step_in but double; params [etac_param_count] double; writes
 * disp [N*3] double.  Uses the context's pads and the mode of `desc`. */
etac_status etac_forward_f64(etac_ctx* ctx, const etac_model_desc* desc,
                             const int32_t* obj_type, const double* obj_dims,
                             const double* obj_pose, const double* pad_pose,
                             const double* params, double* disp, void* stream);

/* ---- Real-to-sim taxel regressor (appendix "Modeling Real Sensors").
 * A PointNet-style network from each pad's displacement field to the outputs of its real
 * sensor's ETAC_TAXELS pressure taxels, with a residual layer and softmax attention pooling:
 *   x_i = [p_i, n_i, U_i] (pad frame);  h1 = relu(R1 x + b) (64);  h2 = relu(R2 h1 + b) (128);
 *   h3 = relu(R3 h2 + b) (256);  f_i = h3 + relu(R4 h3 + b) (256);
 *   a_i = A2 tanh(A1 f_i + b) + b (A1: 256 -> 128, the appendix's [256, 128, 1] MLP);
 *   alpha = softmax of a over the pad's nodes;  g = sum_i alpha_i f_i;
 *   y = H2 relu(H1 g + b) + b (256 -> 128 -> ETAC_TAXELS).
 * rparams: device FP32 [ETAC_REGRESSOR_PARAMS] (16-byte aligned), each layer's W (row-major,
 * out x in) then b, in the order R1, R2, R3, R4, A1, A2, H1, H2.  disp: device [N*3], e.g. the
 * output of etac_step_forward.  Writes taxels [E*P*ETAC_TAXELS] and, when attn is not NULL, each
 * node's softmax weight attn [N].  Uses the context's pads; needs no model.  Enqueued on
 * `stream`; all pointers are borrowed.
 * precision ETAC_PREC_BF16: the per-node layers R1..A1 on the tensor cores (BF16 weights and
 *   activations, FP32 accumulation; x enters split into two BF16 parts), score, softmax, pooling
 *   and head in FP32.  Two launches (the BF16 weight images, then the network); the first call
 *   on a context also builds its pad-to-SM schedule.  A device-side wait that runs out latches
 *   ETAC_ERR_TIMEOUT in the status word (etac_poll_status).
 * precision ETAC_PREC_FP32: every layer in FP32 on the CUDA cores (the unoptimised rung).
 * Errors: ETAC_ERR_INVALID_ARG (NULL or misaligned pointer, unknown precision), ETAC_ERR_OOM,
 * ETAC_ERR_CUDA. */
#define ETAC_TAXELS 8
#define ETAC_REGRESSOR_PARAMS 174729
etac_status etac_regress(etac_ctx* ctx, const float* disp, const float* rparams, float* taxels,
                         float* attn, int32_t precision, void* stream);

/* Message of the last failed call on this context (or, when ctx is NULL, of the last failed
 * etac_create_pads / etac_step_forward_noalloc on this thread).  Valid until the next call
 * on the same context. */
const char* etac_last_error(const etac_ctx* ctx);

/* Frees the context and its device memory (synchronises the device first). NULL is a no-op. */
void etac_destroy(etac_ctx* ctx);

/* ---- Triangle-mesh objects: acceleration structure (host side).
 *
 * ETac detects contact with signed distance fields between the nodes and object meshes
 * (Sec. III-A, "Overview").  For a closed triangle mesh the signed distance at a point q is
 * the distance to the nearest surface point c, negative inside; the sign follows from the
 * pseudo-normal n_F of the feature F (face, edge or vertex) that holds c: q is inside iff
 * (q - c) . n_F < 0 (Baerentzen and Aanaes, 2005).  A query visits the triangles listed for
 * the grid cell that holds q, never the whole mesh.
 *
 * etac_mesh_accel_build validates a mesh and builds, on the host, a uniform grid of cubic
 * cells over the mesh's bounding box.  Every cell is classified by the exact distance d from
 * its centre to the surface against its half-diagonal r:
 *   ETAC_CELL_OUTSIDE  no surface point within r and the centre is outside: every point of
 *                      the cell is outside (no candidates);
 *   ETAC_CELL_INSIDE   no surface point within r and the centre is inside: every point of
 *                      the cell is inside;
 *   ETAC_CELL_SURFACE  the surface may cross the cell.
 * INSIDE and SURFACE cells list every triangle whose distance from the centre is at most
 * d + 2r (+ a slack of 1e-5 cell + 1e-6 mm), which contains the nearest triangle of every
 * point of the cell.  Points outside the grid are outside the mesh.
 *
 * The mesh (host arrays, read during the call): vertices [V*3] in the object frame (mm);
 * triangles [T*3] vertex indices wound counter-clockwise seen from outside.  It must be
 * closed and consistently oriented: every directed edge occurs exactly once and its
 * reverse exactly once; no triangle may have zero area.  `grid` is the number of cells
 * along the longest side of the bounding box, in [1, 512] (0 picks 32).  Errors:
 * ETAC_ERR_INVALID_ARG (message from etac_last_error(NULL)) for a NULL pointer, an index
 * out of range, a degenerate triangle, an open or inconsistently wound mesh, or a grid whose
 * cell or candidate count exceeds 2^24 cells / 2^28 candidates; ETAC_ERR_OOM if host memory
 * runs out.  The structure is owned by the caller until etac_mesh_accel_destroy (NULL is a
 * no-op); etac_mesh_accel_get_view fills *view with pointers into it, valid until then.
 * Host-only: needs no GPU.  Building is deterministic (same mesh, same bytes). */
enum { ETAC_CELL_OUTSIDE = 0, ETAC_CELL_INSIDE = 1, ETAC_CELL_SURFACE = 2 };
typedef struct {
  int32_t num_verts;
  int32_t num_tris;
  const float* verts;      /* host [V*3] */
  const int32_t* tris;     /* host [T*3] */
  int32_t grid;            /* cells along the longest side, 0 = 32 */
} etac_mesh_desc;

typedef struct {
  float origin[3];             /* object-frame corner of cell (0, 0, 0)                       */
  float cell;                  /* cell edge (mm); cell (i, j, k) spans origin + [i, i+1) cell  */
  int32_t dims[3];             /* cells along x, y, z; cell index = (k * dims[1] + j) * dims[0] + i */
  int32_t num_tris;
  int64_t num_cand;            /* total candidate entries                                      */
  const int32_t* cell_start;   /* [C+1] first candidate of each cell, C = dims product         */
  const uint8_t* cell_kind;    /* [C] ETAC_CELL_*                                              */
  const int32_t* cand;         /* [num_cand] triangle indices, ascending within a cell         */
  const float* tri;            /* [T*16] per triangle: a, b, c, unit face normal (xyz + 0)     */
  const float* pseudo;         /* [T*24] per triangle: unit pseudo-normals of edges ab, bc, ca
                                  and vertices a, b, c (xyz + 0); an edge's is the normalised
                                  sum of its two faces' normals, a vertex's the normalised
                                  angle-weighted sum of its faces' normals                   */
} etac_mesh_accel_view;

typedef struct etac_mesh_accel etac_mesh_accel;
etac_status etac_mesh_accel_build(etac_mesh_accel** out, const etac_mesh_desc* desc);
etac_status etac_mesh_accel_get_view(const etac_mesh_accel* accel, etac_mesh_accel_view* view);
void etac_mesh_accel_destroy(etac_mesh_accel* accel);

/* Device copy of a mesh's acceleration structure, and the signed-distance query on it.
 *
 * etac_mesh_gpu_create allocates device memory for the arrays of `accel` and copies them on
 * `stream`, then synchronises `stream` (the accel may be destroyed once it returns).  Errors:
 * ETAC_ERR_INVALID_ARG (NULL), ETAC_ERR_OOM, ETAC_ERR_CUDA.  etac_mesh_gpu_destroy
 * synchronises the device and frees it (NULL is a no-op).
 *
 * etac_mesh_sdf_query evaluates, for n points q [n*3] (device, object frame, mm), the signed
 * distance phi [n] to the mesh (negative inside) and, when grad is not NULL, its outward
 * unit gradient grad [n*3], in FP32 on `stream` (no synchronisation).  A point outside the
 * grid or in an ETAC_CELL_OUTSIDE cell is outside and gets phi = +INFINITY and a zero
 * gradient (its distance is not computed); a non-finite point counts as outside.  Ties
 * between equally near triangles go to the lowest index.  The nearest surface point is
 * q - phi * grad.  Arrays must be 4-byte aligned and must not overlap.  Errors:
 * ETAC_ERR_INVALID_ARG (NULL, n < 0, misalignment), ETAC_ERR_CUDA (launch failure). */
etac_status etac_mesh_gpu_create(etac_mesh_gpu** out, const etac_mesh_accel* accel, void* stream);
etac_status etac_mesh_sdf_query(const etac_mesh_gpu* mesh, int64_t n, const float* q, float* phi,
                                float* grad, void* stream);
void etac_mesh_gpu_destroy(etac_mesh_gpu* mesh);

/* ---- Forward step for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this entry point exists for integration.  Some callers must
 * not allocate GPU memory while they run: a host application that hands the whole device
 * heap to its own pool allocator up front (physics engines commonly do), a real-time
 * control loop in which an allocation's latency or failure is not acceptable, or a plugin
 * that its host program hands device pointers and no allocator.  Such callers cannot use
 * etac_create_pads / etac_set_model, which allocate.
 *
 * etac_step_forward_noalloc runs the batched FP32 forward (ETAC_ALGO_BATCHED,
 * ETAC_PREC_FP32) from device pointers only.  The caller passes every input (pad geometry,
 * parameters, poses) and every output; the scratch the step needs (work-queue counter, status
 * words, per-pad-type tables) lives in one static device array of ETAC_NOALLOC_SCRATCH_BYTES
 * inside the library, which every GPU that loads the library holds until the process exits.
 * The call allocates and frees nothing.  Limits: the scratch must hold
 * 896 bytes per pad-type node, 4 bytes per (node, node) pair of every pad type, and 4 bytes
 * per pad instance (plus alignment); larger batches are rejected with ETAC_ERR_INVALID_ARG
 * and a message giving the bytes needed.  A pad type too large for the batched kernel's
 * shared memory gives ETAC_ERR_UNSUPPORTED, as etac_set_model does.
 *
 * What is checked, and where:
 *   - on the host, before anything is enqueued: NULL pointers, mode, num_types, num_envs,
 *     pads_per_env, max_objects and every type_num_nodes entry (range), and the scratch size
 *     those imply;
 *   - on the device, by the first kernel of the call, before any other kernel indexes with
 *     them: type_off must start at 0 and its differences must be node counts in
 *     [1, max type_num_nodes] whose sum and sum of squares equal those of type_num_nodes;
 *     every pad_type must lie in [0, num_types); pad_off must start at 0 and step by each
 *     pad's node count.  If any of these fails, no output is written and the status word
 *     reads ETAC_ERR_INVALID_ARG;
 *   - trusted, not checked: that every device array holds the number of elements given
 *     below (type_pos / type_nrm [sum n, 3], pad_type [E*P], pad_off [E*P+1], params
 *     [etac_param_count], the step inputs, and outputs of pad_off[E*P] nodes), that alpha
 *     > 0, and that the arrays do not overlap the outputs.
 *
 * device_status (optional, device int32 [1]) receives, in stream order after the step,
 * ETAC_OK, ETAC_ERR_INVALID_ARG (device-side geometry checks failed, nothing written) or
 * ETAC_ERR_NONFINITE (a pose held NaN / Inf; those pads output zero).
 *
 * The first call on each device looks up the device address of the static array (once, with
 * that device current) and keeps it for the life of the process, so make that first call
 * before any stream capture, and do not call this entry point after a cudaDeviceReset (the
 * kept address would be stale).  Every call rebuilds the tables from `params` and clears the
 * words it needs, so calls are independent, but all calls share the one array: calls that
 * overlap on the GPU (different streams, or different host threads on one device) race and
 * give wrong results.  Errors found on the host are read with etac_last_error(NULL). */
#define ETAC_NOALLOC_SCRATCH_BYTES (32u << 20)

typedef struct {
  int32_t num_types;             /* T >= 1                                                    */
  const int32_t* type_num_nodes; /* HOST [T] node count per pad type (sizes and validation)    */
  const int32_t* type_off;       /* device [T+1] prefix sums of type_num_nodes (checked)        */
  const float* type_pos;         /* device [sum n, 3] undeformed positions, pad frame (mm)     */
  const float* type_nrm;         /* device [sum n, 3] unit outward normals                      */
  int32_t num_envs;              /* >= 1                                                        */
  int32_t pads_per_env;          /* >= 1                                                        */
  int32_t max_objects;           /* K in [1, ETAC_MAX_OBJECTS]                                  */
  const int32_t* pad_type;       /* device [E*P] pad type of each pad instance (checked)        */
  const int64_t* pad_off;        /* device [E*P+1] first flat node index of each pad (checked)  */
} etac_noalloc_pads;

/* mode: ETAC_MODE_*; params: device FP32 [etac_param_count] (alpha must be > 0, unchecked);
 * in / out as for etac_step_forward (device pointers); device_status optional (see above).
 * Enqueues work on `stream` only. */
etac_status etac_step_forward_noalloc(const etac_noalloc_pads* pads, int32_t mode,
                                      const float* params, const etac_step_in* in,
                                      const etac_step_out* out, int32_t* device_status,
                                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ETAC_H_ */
