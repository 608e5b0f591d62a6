// tables.cu -- per-pad-type tables of the batched algorithm, rebuilt by etac_set_model.
//
// The residual network's input for node i is X_i = [p_i, n_i, u_hat_i] (ETac Sec. III-A 2)
// and u_hat_i = 0 on passive nodes.  P and N are fixed per pad type, so for every node of a
// type the first layer's geometric part c_i = W1[:, 0:6] [p_i; n_i] + b1, the passive encoder
// output f0_i = ReLU(W2 ReLU(c_i) + b2) and the decoder's local half for that output,
// h0_i = D1[:, 0:64] f0_i + b_D1, are constants of the model.  A per-channel ordering of f0
// (descending, ties by lower node index) lets the max-pool over passive nodes stop at the
// first passive node in that order.  Omega_t[j][i] = exp(-alpha |p_j - p_i|) (Eq. 1) is
// tabulated per type in FP32 (and BF16 for the tensor-core path).
#include <cuda_bf16.h>

#include "etac_common.cuh"
#include "etac_kernels.h"

namespace etac {

// Evaluated in FP64 and rounded once to FP32: the passive max-pool takes, per channel, the
// first passive node of the descending f0 order, so that order must be the exact one.  Two
// nodes of a type can hold f0 values a few 1e-6 apart (measured on the flat 16 x 16 pad), within
// the error of an FP32 evaluation; rounding the FP64 values keeps their order (rounding is
// monotone) unless they are within half an FP32 ulp.  Once per etac_set_model.
__global__ void __launch_bounds__(128) tables_node_kernel(TablesArgs a) {
  if (a.skip && *a.skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.total_nodes) return;
  const float* W = a.params;
  double X[6];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    X[q] = a.type_pos[3 * i + q];
    X[3 + q] = a.type_nrm[3 * i + q];
  }
  double z[H], f[H];
#pragma unroll 4
  for (int c = 0; c < H; ++c) {
    double acc = W[OFF_B1 + c];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc = fma((double)W[OFF_W1 + c * NIN + k], X[k], acc);
    a.ctab[(size_t)i * H + c] = (float)acc;
    z[c] = acc > 0.0 ? acc : 0.0;
  }
#pragma unroll 1
  for (int c = 0; c < H; ++c) {
    double acc = W[OFF_B2 + c];
#pragma unroll 8
    for (int k = 0; k < H; ++k) acc = fma((double)W[OFF_W2 + c * H + k], z[k], acc);
    f[c] = acc > 0.0 ? acc : 0.0;
    a.f0tab[(size_t)i * H + c] = (float)f[c];
  }
#pragma unroll 1
  for (int c = 0; c < H; ++c) {
    double acc = W[OFF_BD + c];
#pragma unroll 8
    for (int k = 0; k < H; ++k) acc = fma((double)W[OFF_WD + c * 2 * H + k], f[k], acc);
    a.h0tab[(size_t)i * H + c] = (float)acc;
    if (a.h0bf16) reinterpret_cast<__nv_bfloat16*>(a.h0bf16)[(size_t)i * H + c] = __double2bfloat16(acc);
  }
}

// one block per (type, channel): rank of every node in descending f0 order, ties -> lower index
__global__ void __launch_bounds__(256) tables_order_kernel(TablesArgs a) {
  extern __shared__ float col[];
  if (a.skip && *a.skip) return;
  const int t = blockIdx.x, u = blockIdx.y;
  const int o = a.type_off[t], n = a.type_off[t + 1] - o;
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a.f0tab[(size_t)(o + i) * H + u];
  __syncthreads();
  int16_t* ord = a.order + (size_t)H * o + (size_t)u * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = col[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const float w = col[j];
      rank += (w > v) || (w == v && j < i);
    }
    ord[rank] = (int16_t)i;
    if (a.ranked) a.ranked[(size_t)H * o + (size_t)u * n + rank] = make_float2(v, __int_as_float(i));
  }
}

__global__ void __launch_bounds__(256) tables_omega_kernel(TablesArgs a) {
  if (a.skip && *a.skip) return;
  const float alpha = a.params[OFF_ALPHA];
  const long long total = a.omega_off[a.num_types];
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int t = 0;
    while (idx >= a.omega_off[t + 1]) ++t;
    const int o = a.type_off[t], n = a.type_off[t + 1] - o;
    const long long r = idx - a.omega_off[t];
    const int j = (int)(r / n), i = (int)(r % n);
    const float* pj = a.type_pos + 3 * (size_t)(o + j);
    const float* pi = a.type_pos + 3 * (size_t)(o + i);
    const float dx = pj[0] - pi[0], dy = pj[1] - pi[1], dz = pj[2] - pi[2];
    const float d = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
    const float w = expf(-alpha * d);
    if (a.omega) a.omega[idx] = w;
    if (a.omega_bf16) reinterpret_cast<__nv_bfloat16*>(a.omega_bf16)[idx] = __float2bfloat16_rn(w);
    if (a.om_hi) {
      const __nv_bfloat16 h = __float2bfloat16_rn(w);
      reinterpret_cast<__nv_bfloat16*>(a.om_hi)[idx] = h;
      reinterpret_cast<__nv_bfloat16*>(a.om_lo)[idx] = __float2bfloat16_rn(w - __bfloat162float(h));
      const float dw = d * w;
      const __nv_bfloat16 dh = __float2bfloat16_rn(dw);
      reinterpret_cast<__nv_bfloat16*>(a.dom_hi)[idx] = dh;
      reinterpret_cast<__nv_bfloat16*>(a.dom_lo)[idx] = __float2bfloat16_rn(dw - __bfloat162float(dh));
    }
  }
}

cudaError_t launch_tables(const TablesArgs& a, int nmax, cudaStream_t s) {
  tables_node_kernel<<<(a.total_nodes + 127) / 128, 128, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tables_order_kernel<<<dim3(a.num_types, H), 256, sizeof(float) * nmax, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.omega || a.omega_bf16 || a.om_hi) {
    tables_omega_kernel<<<1024, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace etac
