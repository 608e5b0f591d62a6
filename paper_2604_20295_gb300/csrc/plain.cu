// plain.cu -- the unoptimised ("plain") ETac step: one CTA per pad, Eq. 1 and Eq. 4
// evaluated literally.
//
// Per pad (ETac Sec. III-A): contact detection on every node; the active set in node order;
// the residual network Phi on every node (per-node shared MLP E1, E2 on [P, N, U_hat], channel
// max-pool to the 64-d global feature, global MLP G1, broadcast + concat, decoder D1, D2);
// for each passive node the decay propagation sum_j exp(-alpha |p_j - p_i|) u_hat_j over the
// active nodes with the exponential evaluated per pair (Eq. 1); output Eq. 4.  Only the
// decoder's global half (W_g g + b) is hoisted out of the node loop.  Instantiated in FP32
// (the plain metric path) and FP64 (finite-difference gradient checks only).
#include "etac_common.cuh"
#include "etac_kernels.h"

namespace etac {

constexpr int PLAIN_THREADS = 256;

// padded shared-memory copy of the parameters (16-byte aligned tensors; G1 stays global)
constexpr int S_W1 = 0;
constexpr int S_B1 = S_W1 + H * NIN;   // 576
constexpr int S_W2 = S_B1 + H;         // 640
constexpr int S_B2 = S_W2 + H * H;     // 4736
constexpr int S_WD = S_B2 + H;         // 4800
constexpr int S_BD = S_WD + H * 2 * H; // 12992
constexpr int S_W4 = S_BD + H;         // 13056
constexpr int S_B4 = S_W4 + 3 * H;     // 13248
constexpr int S_TOTAL = S_B4 + 4;      // 13252 (multiple of 4)

template <typename T>
struct PlainTraits;
template <>
struct PlainTraits<float> {
  using PO = PadObj;
};
template <>
struct PlainTraits<double> {
  using PO = PadObj64;
};

template <typename T>
static size_t plain_smem_bytes(int nmax, int K) {
  size_t b = sizeof(T) * ((size_t)S_TOTAL + 6 * (size_t)nmax + 8 * H + 2 * H);
  b = (b + 15) & ~size_t(15);
  b += sizeof(int16_t) * (size_t)nmax;
  b = (b + 15) & ~size_t(15);
  b += sizeof(int) * (PLAIN_THREADS + 8);
  b = (b + 15) & ~size_t(15);
  b += sizeof(typename PlainTraits<T>::PO) * (size_t)K;
  return b;
}

template <typename T>
__device__ __forceinline__ T relu(T x) {
  return x > T(0) ? x : T(0);
}

template <typename T>
__device__ __forceinline__ void encode1(const T* sp, const T X[NIN], T z1[H]) {
#pragma unroll
  for (int c = 0; c < H; ++c) {
    T acc = sp[S_B1 + c];
#pragma unroll
    for (int k = 0; k < NIN; ++k) acc = fma(sp[S_W1 + c * NIN + k], X[k], acc);
    z1[c] = relu(acc);
  }
}

template <typename T>
__device__ __forceinline__ T encode2_channel(const T* sp, const T z1[H], int c) {
  T acc = sp[S_B2 + c];
#pragma unroll
  for (int k = 0; k < H; ++k) acc = fma(sp[S_W2 + c * H + k], z1[k], acc);
  return relu(acc);
}

template <typename T>
__device__ __forceinline__ void encode(const T* sp, const T X[NIN], T f[H]) {
  T z1[H];
  encode1<T>(sp, X, z1);
#pragma unroll
  for (int c = 0; c < H; ++c) f[c] = encode2_channel<T>(sp, z1, c);
}

template <typename T>
__device__ __forceinline__ void decode(const T* sp, const T* beta, const T f[H], T r[3]) {
  r[0] = sp[S_B4 + 0];
  r[1] = sp[S_B4 + 1];
  r[2] = sp[S_B4 + 2];
#pragma unroll 1
  for (int c = 0; c < H; ++c) {
    T acc = beta[c];
#pragma unroll
    for (int k = 0; k < H; ++k) acc = fma(sp[S_WD + c * 2 * H + k], f[k], acc);
    acc = relu(acc);
    r[0] = fma(sp[S_W4 + c], acc, r[0]);
    r[1] = fma(sp[S_W4 + H + c], acc, r[1]);
    r[2] = fma(sp[S_W4 + 2 * H + c], acc, r[2]);
  }
}

template <typename T>
__device__ __forceinline__ T texp(T x);
template <>
__device__ __forceinline__ float texp<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double texp<double>(double x) { return exp(x); }

template <typename T>
__global__ void __launch_bounds__(PLAIN_THREADS, 1)
plain_forward_kernel(PlainArgs<T> a) {
  using PO = typename PlainTraits<T>::PO;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pad = blockIdx.x;
  const int env = pad / a.P;
  const int ty = a.pad_type[pad];
  const int n = a.type_off[ty + 1] - a.type_off[ty];
  const float* tpos = a.type_pos + 3 * (size_t)a.type_off[ty];
  const float* tnrm = a.type_nrm + 3 * (size_t)a.type_off[ty];
  const long long base = a.pad_off[pad];
  if (!ETAC_IN(a.status, base + n - 1, a.num_nodes)) return;   // block-uniform

  T* sp = reinterpret_cast<T*>(smem);
  T* sap = sp + S_TOTAL;              // [nmax][6] active nodes: p, u_hat
  T* sred = sap + 6 * a.nmax;         // [8][H]
  T* sg = sred + 8 * H;               // [H] g0, later g
  T* sbeta = sg + H;                  // [H]
  size_t off = sizeof(T) * ((size_t)S_TOTAL + 6 * (size_t)a.nmax + 8 * H + 2 * H);
  off = (off + 15) & ~size_t(15);
  int16_t* sidx = reinterpret_cast<int16_t*>(smem + off);   // [nmax] active slot or -1
  off += sizeof(int16_t) * (size_t)a.nmax;
  off = (off + 15) & ~size_t(15);
  int* scnt = reinterpret_cast<int*>(smem + off);           // [PLAIN_THREADS + 8]
  off += sizeof(int) * (PLAIN_THREADS + 8);
  off = (off + 15) & ~size_t(15);
  PO* spo = reinterpret_cast<PO*>(smem + off);               // [K]

  const T* gp = a.params;
  for (int i = tid; i < S_TOTAL; i += PLAIN_THREADS) {
    int src = -1;
    if (i < S_B1) src = OFF_W1 + i;
    else if (i < S_W2) src = OFF_B1 + (i - S_B1);
    else if (i < S_B2) src = OFF_W2 + (i - S_W2);
    else if (i < S_WD) src = OFF_B2 + (i - S_B2);
    else if (i < S_BD) src = OFF_WD + (i - S_WD);
    else if (i < S_W4) src = OFF_BD + (i - S_BD);
    else if (i < S_B4) src = OFF_W4 + (i - S_W4);
    else if (i < S_B4 + 3) src = OFF_B4 + (i - S_B4);
    sp[i] = src >= 0 ? gp[src] : T(0);
  }
  const T alpha = gp[OFF_ALPHA];
  if (tid == 0) scnt[PLAIN_THREADS + 1] = 0;   // invalid-input flag
  __syncthreads();
  const bool given = a.mask_in != nullptr;     // mode B: contact supplied by the caller
  if (tid < a.K && !given) {
    const int o = env * a.K + tid;
    const T* op = a.obj_pose + 7 * (size_t)o;
    const T* pp = a.pad_pose + 7 * (size_t)pad;
    const T* od = a.obj_dims + 3 * (size_t)o;
    int type = a.obj_type[o];
    bool ok = true;
    for (int i = 0; i < 7; ++i) ok &= isfinite(op[i]) && isfinite(pp[i]);
    for (int i = 0; i < 3; ++i) ok &= isfinite(od[i]);
    ok &= (op[3] != T(0) || op[4] != T(0) || op[5] != T(0) || op[6] != T(0));
    ok &= (pp[3] != T(0) || pp[4] != T(0) || pp[5] != T(0) || pp[6] != T(0));
    if (type < OBJ_NONE || type > OBJ_MESH) type = OBJ_NONE;
    if (!ok && type != OBJ_NONE) {
      scnt[PLAIN_THREADS + 1] = 1;
      type = OBJ_NONE;
    }
    if constexpr (sizeof(T) == 4) {
      const MeshDev* mesh = nullptr;
      if (type == OBJ_MESH && !(mesh = object_mesh(od, a.meshes, a.num_meshes))) type = OBJ_NONE;
      setup_pad_obj(op, type, od, pp, a.type_pmax[ty], &spo[tid], mesh);
    } else {
      if (type == OBJ_MESH) type = OBJ_NONE;   // the FP64 check covers the primitives
      setup_pad_obj64(op, type, od, pp, &spo[tid]);
    }
  }
  __syncthreads();
  if (scnt[PLAIN_THREADS + 1]) {
    if (tid == 0) latch_status(a.status, STATUS_NONFINITE);
    for (int i = tid; i < n; i += PLAIN_THREADS) {
      a.disp[3 * (base + i) + 0] = T(0);
      a.disp[3 * (base + i) + 1] = T(0);
      a.disp[3 * (base + i) + 2] = T(0);
      if (a.mask) a.mask[base + i] = 0;
      if (a.pen) a.pen[base + i] = T(0);
    }
    if (tid == 0 && a.count) a.count[pad] = 0;
    return;
  }

  // ---- contact on a contiguous chunk of nodes per thread (node order is kept)
  const int chunk = (n + PLAIN_THREADS - 1) / PLAIN_THREADS;
  const int i0 = min(n, tid * chunk), i1 = min(n, i0 + chunk);
  unsigned bits = 0;
  int cnt = 0;
  for (int i = i0; i < i1; ++i) {
    T u[3];
    T pen = T(0);
    bool act;
    if constexpr (sizeof(T) == 4) {
      float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
      float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
      NodeContact c = given ? contact_given(a.mask_in, a.uhat_in, base + i)
                            : contact_node(spo, a.K, p, nr);
      act = c.active;
      u[0] = c.u[0]; u[1] = c.u[1]; u[2] = c.u[2];
      pen = act ? -c.phi : 0.f;
    } else {
      double p[3] = {tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]};
      double nr[3] = {tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]};
      act = contact_node64(spo, a.K, p, nr, u);
      pen = act ? sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) : 0.0;
    }
    // active nodes keep u_hat (Eq. 4 covers the passive ones); disp doubles as scratch
    a.disp[3 * (base + i) + 0] = u[0];
    a.disp[3 * (base + i) + 1] = u[1];
    a.disp[3 * (base + i) + 2] = u[2];
    if (a.mask) a.mask[base + i] = act ? 1 : 0;
    if (a.pen) a.pen[base + i] = pen;
    if (act) {
      bits |= 1u << (i - i0);
      ++cnt;
    }
  }
  // exclusive scan of the per-thread counts
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) scnt[warp] = incl;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int w = 0; w < PLAIN_THREADS / 32; ++w) {
      int v = scnt[w];
      scnt[w] = run;
      run += v;
    }
    scnt[PLAIN_THREADS] = run;
  }
  __syncthreads();
  const int m = scnt[PLAIN_THREADS];
  {
    int slot = scnt[warp] + incl - cnt;
    for (int i = i0; i < i1; ++i) {
      if (bits & (1u << (i - i0))) {
        sidx[i] = (int16_t)slot;
        sap[6 * slot + 0] = (T)tpos[3 * i];
        sap[6 * slot + 1] = (T)tpos[3 * i + 1];
        sap[6 * slot + 2] = (T)tpos[3 * i + 2];
        sap[6 * slot + 3] = a.disp[3 * (base + i) + 0];
        sap[6 * slot + 4] = a.disp[3 * (base + i) + 1];
        sap[6 * slot + 5] = a.disp[3 * (base + i) + 2];
        ++slot;
      } else {
        sidx[i] = -1;
      }
    }
  }
  if (tid == 0 && a.count) a.count[pad] = m;
  __syncthreads();
  if (m == 0) {   // no contact: zero displacement everywhere (u_hat is already zero)
    return;
  }

  // ---- residual network, pass 1: per-node encoder on every node and channel max-pool
  if (uses_residual(a.mode)) {
    // per-warp running channel maxima in shared memory (ReLU outputs are >= 0)
    for (int c = lane; c < H; c += 32) sred[warp * H + c] = T(0);
    __syncwarp();
    const int nround = (n + PLAIN_THREADS - 1) / PLAIN_THREADS;
    for (int rnd = 0; rnd < nround; ++rnd) {
      const int i = rnd * PLAIN_THREADS + tid;
      const bool live = i < n;
      T X[NIN], z1[H];
      const int s = live ? sidx[i] : -1;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        X[q] = live ? (T)tpos[3 * i + q] : T(0);
        X[3 + q] = live ? (T)tnrm[3 * i + q] : T(0);
        X[6 + q] = s >= 0 ? sap[6 * s + 3 + q] : T(0);
      }
      encode1<T>(sp, X, z1);
#pragma unroll 1
      for (int c = 0; c < H; ++c) {
        T v = live ? encode2_channel<T>(sp, z1, c) : T(0);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          T o = __shfl_xor_sync(0xffffffffu, v, d);
          v = o > v ? o : v;
        }
        if (lane == 0 && v > sred[warp * H + c]) sred[warp * H + c] = v;
      }
    }
    __syncthreads();
    if (tid < H) {
      T v = sred[tid];
      for (int w = 1; w < PLAIN_THREADS / 32; ++w) v = sred[w * H + tid] > v ? sred[w * H + tid] : v;
      sg[tid] = v;   // g0
    }
    __syncthreads();
    T gv = T(0);
    if (tid < H) {
      T acc = gp[OFF_BG + tid];
      for (int k = 0; k < H; ++k) acc = fma(gp[OFF_WG + tid * H + k], sg[k], acc);
      gv = relu(acc);
    }
    __syncthreads();
    if (tid < H) sg[tid] = gv;   // g
    __syncthreads();
    if (tid < H) {
      T acc = sp[S_BD + tid];
      for (int k = 0; k < H; ++k) acc = fma(sp[S_WD + tid * 2 * H + H + k], sg[k], acc);
      sbeta[tid] = acc;
    }
    __syncthreads();
  }

  // ---- pass 2: passive nodes, Eq. 4 = Omega U_a (Eq. 1) + Phi_p
  for (int i = tid; i < n; i += PLAIN_THREADS) {
    if (sidx[i] >= 0) continue;
    const T px = (T)tpos[3 * i], py = (T)tpos[3 * i + 1], pz = (T)tpos[3 * i + 2];
    T out[3] = {T(0), T(0), T(0)};
    if (uses_propagation(a.mode)) {
      for (int j = 0; j < m; ++j) {
        const T* q = sap + 6 * j;
        T dx = q[0] - px, dy = q[1] - py, dz = q[2] - pz;
        T w = texp<T>(-alpha * sqrt(dx * dx + dy * dy + dz * dz));
        out[0] = fma(w, q[3], out[0]);
        out[1] = fma(w, q[4], out[1]);
        out[2] = fma(w, q[5], out[2]);
      }
    }
    if (uses_residual(a.mode)) {
      T X[NIN], f[H], r[3];
      X[0] = px; X[1] = py; X[2] = pz;
      X[3] = (T)tnrm[3 * i]; X[4] = (T)tnrm[3 * i + 1]; X[5] = (T)tnrm[3 * i + 2];
      X[6] = X[7] = X[8] = T(0);
      encode<T>(sp, X, f);
      decode<T>(sp, sbeta, f, r);
      out[0] += r[0];
      out[1] += r[1];
      out[2] += r[2];
    }
    a.disp[3 * (base + i) + 0] = out[0];
    a.disp[3 * (base + i) + 1] = out[1];
    a.disp[3 * (base + i) + 2] = out[2];
  }
}

template <typename T>
cudaError_t launch_plain_forward(const PlainArgs<T>& a, int num_pads, cudaStream_t stream) {
  size_t smem = plain_smem_bytes<T>(a.nmax, a.K);
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(plain_forward_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  plain_forward_kernel<T><<<num_pads, PLAIN_THREADS, smem, stream>>>(a);
  return cudaGetLastError();
}

size_t plain_smem_f32(int nmax, int K) { return plain_smem_bytes<float>(nmax, K); }
size_t plain_smem_f64(int nmax, int K) { return plain_smem_bytes<double>(nmax, K); }

template cudaError_t launch_plain_forward<float>(const PlainArgs<float>&, int, cudaStream_t);
template cudaError_t launch_plain_forward<double>(const PlainArgs<double>&, int, cudaStream_t);

}  // namespace etac
