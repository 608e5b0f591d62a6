// noalloc.cu -- etac_step_forward_noalloc: the batched FP32 forward for callers that cannot
// allocate device memory (see include/etac.h).
//
// The batched kernel needs scratch beyond its inputs and outputs: a work-queue counter, a
// status word and the per-pad-type tables built from the parameters.  Here that scratch is
// one file-scope __device__ array of ETAC_NOALLOC_SCRATCH_BYTES, which every GPU that loads
// the library holds until the process exits.  Host code cannot use the array's name as a
// device address (in host code it names a host-side stand-in), so the first call on each
// device, with that device current, looks the address up with cudaGetSymbolAddress and
// caches it for the life of the process (a cudaDeviceReset invalidates it; the entry point
// must not be used after one); kernels receive that address.  No call here allocates or
// frees memory.
#include <cuda_runtime.h>

#include <climits>

#include <mutex>
#include <string>

#include "etac.h"
#include "etac_common.cuh"
#include "etac_kernels.h"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[ETAC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
std::mutex g_setup_mutex;

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// byte layout of the scratch array for one call
struct Layout {
  size_t ticket, status, bad, omega_off, pmax, items, ctab, f0tab, h0tab, order, omega, total;
  Layout(int T, long long tn, long long nn2, long long np) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = up256(o + bytes);
      return r;
    };
    ticket = take(sizeof(int));
    status = take(sizeof(int));
    bad = take(sizeof(int));
    omega_off = take(sizeof(long long) * (size_t)(T + 1));
    pmax = take(sizeof(float) * (size_t)T);
    items = take(sizeof(int) * (size_t)np);
    ctab = take(sizeof(float) * etac::H * (size_t)tn);
    f0tab = take(sizeof(float) * etac::H * (size_t)tn);
    h0tab = take(sizeof(float) * etac::H * (size_t)tn);
    order = take(sizeof(int16_t) * etac::H * (size_t)tn);
    omega = take(sizeof(float) * (size_t)nn2);
    total = o;
  }
};

// Checks the caller's device-side geometry against the sizes the host side derived from
// type_num_nodes, before any kernel indexes with it: type_off must start at 0 with every
// type's node count in [1, nmax], sum tn and sum of squares nn2 (so the tables and Omega stay
// inside the regions sized from those sums, and every pad fits the shared-memory staging);
// every pad_type must lie in [0, T); pad_off must start at 0 and step by its pad's node
// count.  On a mismatch *bad = 1 and *status = ETAC_ERR_INVALID_ARG, and the later kernels of
// the call return without touching anything.  Otherwise fills the per-call arrays: Omega
// offsets (prefix of n_t^2), the largest |p| per pad type, the identity work order, and
// clears the queue counter and status word.
__global__ void noalloc_prepare_kernel(const int* type_off, const float* type_pos, int T,
                                       int nmax, long long tn, long long nn2,
                                       const int* pad_type, const long long* pad_off,
                                       int num_pads, long long* omega_off, float* pmax,
                                       int* items, int* ticket, int* status, int* bad) {
  const int tid = threadIdx.x;
  __shared__ int s_bad;
  if (tid == 0) {
    int b = type_off[0] != 0;
    long long acc = 0, sum = 0;
    omega_off[0] = 0;
    for (int t = 0; t < T && !b; ++t) {
      const long long n = (long long)type_off[t + 1] - type_off[t];
      if (n < 1 || n > nmax) b = 1;
      sum += n;
      acc += n * n;
      omega_off[t + 1] = acc;
    }
    if (sum != tn || acc != nn2) b = 1;
    if (pad_off[0] != 0) b = 1;
    s_bad = b;
    *ticket = 0;
  }
  __syncthreads();
  if (!s_bad) {
    int b = 0;
    for (int p = tid; p < num_pads; p += blockDim.x) {
      const int t = pad_type[p];
      if (t < 0 || t >= T) {
        b = 1;
        continue;
      }
      if (pad_off[p + 1] - pad_off[p] != (long long)(type_off[t + 1] - type_off[t])) b = 1;
      items[p] = p;
    }
    if (b) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  if (tid == 0) {
    *bad = s_bad;
    *status = s_bad ? ETAC_ERR_INVALID_ARG : 0;
  }
  if (s_bad) return;
  // Euclidean |p|, rounded up so that the FP32 value is never below the exact norm
  __shared__ float red[256];
  for (int t = 0; t < T; ++t) {
    float m = 0.f;
    for (int i = type_off[t] + tid; i < type_off[t + 1]; i += blockDim.x) {
      const float x = type_pos[3 * i], y = type_pos[3 * i + 1], z = type_pos[3 * i + 2];
      m = fmaxf(m, __fsqrt_ru(__fmaf_ru(x, x, __fmaf_ru(y, y, __fmul_ru(z, z)))));
    }
    red[tid] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (tid < s) red[tid] = fmaxf(red[tid], red[tid + s]);
      __syncthreads();
    }
    if (tid == 0) pmax[t] = red[0];
    __syncthreads();
  }
}

}  // namespace

namespace etac {
void set_context_free_error(const std::string& msg);   // api.cu: read by etac_last_error(NULL)
}

namespace {
etac_status noalloc_fail(etac_status s, const std::string& msg) {
  etac::set_context_free_error(msg);
  return s;
}
}  // namespace

extern "C" etac_status etac_step_forward_noalloc(const etac_noalloc_pads* pads, int32_t mode,
                                                 const float* params, const etac_step_in* in,
                                                 const etac_step_out* out,
                                                 int32_t* device_status, void* stream) {
  if (!pads || !pads->type_num_nodes || !pads->type_off || !pads->type_pos || !pads->type_nrm ||
      !pads->pad_type || !pads->pad_off || !params || !in || !out || !out->disp)
    return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: NULL argument");
  const bool given = in->active_mask_in != nullptr;
  if (given != (in->active_disp_in != nullptr))
    return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: active_mask_in and "
                                              "active_disp_in must be given together (or neither)");
  if (!given && (!in->obj_type || !in->obj_dims || !in->obj_pose || !in->pad_pose))
    return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: NULL argument");
  if (mode < ETAC_MODE_FULL || mode > ETAC_MODE_PENETRATION_ONLY)
    return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: unknown mode");
  const int T = pads->num_types;
  if (T < 1 || pads->num_envs < 1 || pads->pads_per_env < 1 || pads->max_objects < 1 ||
      pads->max_objects > ETAC_MAX_OBJECTS)
    return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: bad sizes");
  long long tn = 0, nn2 = 0;
  int nmax = 0;
  for (int t = 0; t < T; ++t) {
    const int n = pads->type_num_nodes[t];
    if (n < 1 || n > ETAC_MAX_PAD_NODES)
      return noalloc_fail(ETAC_ERR_INVALID_ARG, "etac_step_forward_noalloc: pad type size");
    tn += n;
    nn2 += (long long)n * n;
    nmax = n > nmax ? n : nmax;
  }
  const long long np = (long long)pads->num_envs * pads->pads_per_env;
  const Layout L(T, tn, nn2, np);
  if (L.total > (size_t)ETAC_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(ETAC_ERR_INVALID_ARG,
                        "etac_step_forward_noalloc: these pads need " + std::to_string(L.total) +
                            " bytes of scratch; the static scratch holds " +
                            std::to_string((size_t)ETAC_NOALLOC_SCRATCH_BYTES) + " bytes");
  if (etac::batched_smem_bytes(nmax, pads->max_objects) > 227 * 1024)
    return noalloc_fail(ETAC_ERR_UNSUPPORTED,
                        "etac_step_forward_noalloc: a pad type of " + std::to_string(nmax) +
                            " nodes does not fit the batched kernel's shared memory");

  // once per device, with that device current: device address of the static scratch
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(ETAC_ERR_CUDA, "etac_step_forward_noalloc: no current CUDA device");
  unsigned char* base = nullptr;
  int nsm = 0;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return noalloc_fail(ETAC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                               cudaGetErrorString(e));
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess)
        return noalloc_fail(ETAC_ERR_CUDA, std::string("SM count: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
      g_num_sms[dev] = sms;
    }
    base = g_scratch_ptr[dev];
    nsm = g_num_sms[dev];
  }
  int per_sm = 0;
  e = etac::batched_occupancy(nmax, pads->max_objects, false, &per_sm);
  if (e != cudaSuccess)
    return noalloc_fail(ETAC_ERR_CUDA, std::string("etac_step_forward_noalloc: occupancy query: ") +
                                           cudaGetErrorString(e));
  if (per_sm < 1)
    return noalloc_fail(ETAC_ERR_UNSUPPORTED,
                        "etac_step_forward_noalloc: the batched kernel does not fit an SM for "
                        "these pad sizes");

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  long long* omega_off = reinterpret_cast<long long*>(base + L.omega_off);
  int* ticket = reinterpret_cast<int*>(base + L.ticket);
  int* status = reinterpret_cast<int*>(base + L.status);
  int* bad = reinterpret_cast<int*>(base + L.bad);
  float* pmax = reinterpret_cast<float*>(base + L.pmax);
  int* items = reinterpret_cast<int*>(base + L.items);
  noalloc_prepare_kernel<<<1, 256, 0, s>>>(
      pads->type_off, pads->type_pos, T, nmax, tn, nn2, pads->pad_type,
      reinterpret_cast<const long long*>(pads->pad_off), (int)np, omega_off, pmax, items, ticket,
      status, bad);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return noalloc_fail(ETAC_ERR_CUDA, std::string("prepare launch: ") + cudaGetErrorString(e));

  etac::TablesArgs ta{};
  ta.type_pos = pads->type_pos;
  ta.type_nrm = pads->type_nrm;
  ta.type_off = pads->type_off;
  ta.omega_off = omega_off;
  ta.num_types = T;
  ta.total_nodes = (int)tn;
  ta.params = params;
  ta.ctab = reinterpret_cast<float*>(base + L.ctab);
  ta.f0tab = reinterpret_cast<float*>(base + L.f0tab);
  ta.h0tab = reinterpret_cast<float*>(base + L.h0tab);
  ta.order = reinterpret_cast<int16_t*>(base + L.order);
  ta.omega = reinterpret_cast<float*>(base + L.omega);
  ta.omega_bf16 = nullptr;
  ta.skip = bad;
  e = etac::launch_tables(ta, nmax, s);
  if (e != cudaSuccess)
    return noalloc_fail(ETAC_ERR_CUDA, std::string("tables launch: ") + cudaGetErrorString(e));

  etac::BatchedArgs b{};
  // the instance offsets are checked against the type sizes by the prepare kernel (a mismatch
  // stops the step), so the index checks of the bounds build only bound each pad's own range
  b.num_nodes = LLONG_MAX;
  b.type_pos = pads->type_pos;
  b.type_nrm = pads->type_nrm;
  b.type_pmax = pmax;
  b.type_off = pads->type_off;
  b.omega_off = omega_off;
  b.pad_type = pads->pad_type;
  b.pad_off = reinterpret_cast<const long long*>(pads->pad_off);
  b.item_pad = items;
  b.num_items = (int)np;
  b.P = pads->pads_per_env;
  b.K = pads->max_objects;
  b.nmax = nmax;
  b.obj_type = in->obj_type;
  b.obj_dims = in->obj_dims;
  b.obj_pose = in->obj_pose;
  b.pad_pose = in->pad_pose;
  b.params = params;
  b.ctab = ta.ctab;
  b.f0tab = ta.f0tab;
  b.h0tab = ta.h0tab;
  b.order = ta.order;
  b.omega = ta.omega;
  b.mode = mode;
  b.disp = out->disp;
  b.mask = out->active_mask;
  b.pen = out->penetration;
  b.count = out->active_count;
  b.ticket = ticket;
  b.status = status;
  b.skip = bad;
  b.mask_in = in->active_mask_in;
  b.uhat_in = in->active_disp_in;
  const long long grid = (long long)per_sm * nsm;
  e = etac::launch_batched_forward(b, (int)(grid < np ? grid : np), s);
  if (e != cudaSuccess)
    return noalloc_fail(ETAC_ERR_CUDA, std::string("forward launch: ") + cudaGetErrorString(e));
  if (device_status) {
    e = cudaMemcpyAsync(device_status, status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
      return noalloc_fail(ETAC_ERR_CUDA, std::string("status copy: ") + cudaGetErrorString(e));
  }
  return ETAC_OK;
}
