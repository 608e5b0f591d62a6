// regress.cu -- real-to-sim taxel regressor (ETac appendix, "Modeling Real Sensors"), plain
// FP32 form.
//
// The regressor maps a pad's displacement field to the outputs of its real sensor's eight
// taxels: a per-node encoder on x_i = [p_i, n_i, U_i] (R1 9->64, R2 64->128, R3 128->256,
// ReLU, then the residual layer f = h3 + relu(R4 h3 + b) at width 256), an attention score
// a_i = A2 tanh(A1 f_i + b) + b (the appendix's [256, 128, 1] MLP with tanh), softmax weights
// over the pad's nodes, the weighted feature g = sum_i alpha_i f_i, and the head
// y = H2 relu(H1 g + b) + b.
//
// One CTA of 256 threads per pad (grid-stride over pads).  Nodes go through the encoder in
// chunks of 16 rows staged in shared memory, layer by layer (each thread computes
// 16 * width / 256 outputs of a layer as FP32 dot products).  The softmax pooling runs
// online across chunks: a running maximum M of the scores, the sum Z of exp(a - M) and the
// 256-wide sum of exp(a - M) f_i (thread k holds channel k), both rescaled by exp(M_old - M)
// when the maximum grows.  The head runs once per pad.  This is the unoptimised rung
// (280 kFLOP per node on the FP32 pipes); the tensor-core form replaces the encoder chain.
#include <cuda_runtime.h>

#include <cmath>

#include "etac.h"
#include "etac_kernels.h"

namespace {

constexpr int RC = 16;   // node rows per chunk
enum { ACT_RELU = 0, ACT_TANH = 1 };

// out[i][o] = act(b[o] + sum_c W[o][c] in[i][c]) for rows i < m; rows m..RC-1 are zeroed
template <int IN, int OUT, int ACT>
__device__ __forceinline__ void layer(const float* __restrict__ W, const float* __restrict__ b,
                                      const float* in, float* out, int m) {
  for (int idx = threadIdx.x; idx < RC * OUT; idx += blockDim.x) {
    const int i = idx / OUT, o = idx - i * OUT;
    float v = 0.f;
    if (i < m) {
      float acc = b[o];
      const float* w = W + (size_t)o * IN;
      const float* x = in + i * IN;
#pragma unroll 8
      for (int c = 0; c < IN; ++c) acc = fmaf(w[c], x[c], acc);
      v = ACT == ACT_RELU ? fmaxf(acc, 0.f) : tanhf(acc);
    }
    out[idx] = v;
  }
}

__global__ void __launch_bounds__(256) regress_plain_kernel(etac::RegArgs a) {
  __shared__ float sX[RC * 9];
  __shared__ float sH1[RC * 64];
  __shared__ float sH2[RC * 128];     // also the attention hidden layer
  __shared__ float sH3[RC * 256];
  __shared__ float sF[RC * 256];
  __shared__ float sA[RC];
  __shared__ float sG[256];
  __shared__ float sZ[128];
  const int tid = threadIdx.x;
  for (int p = blockIdx.x; p < a.num_pads; p += gridDim.x) {
    const int t = a.pad_type[p];
    const int t0 = a.type_off[t], n = a.type_off[t + 1] - t0;
    const long long base = a.pad_off[p];
    float M = -INFINITY, Z = 0.f, g = 0.f;   // g: channel tid of the weighted sum
    for (int c0 = 0; c0 < n; c0 += RC) {
      const int m = min(RC, n - c0);
      for (int idx = tid; idx < RC * 9; idx += blockDim.x) {
        const int i = idx / 9, k = idx - i * 9;
        float v = 0.f;
        if (i < m) {
          const int node = t0 + c0 + i;
          v = k < 3 ? a.type_pos[3 * node + k]
                    : (k < 6 ? a.type_nrm[3 * node + k - 3] : a.disp[3 * (base + c0 + i) + k - 6]);
        }
        sX[idx] = v;
      }
      __syncthreads();
      layer<9, 64, ACT_RELU>(a.W[0], a.b[0], sX, sH1, m);
      __syncthreads();
      layer<64, 128, ACT_RELU>(a.W[1], a.b[1], sH1, sH2, m);
      __syncthreads();
      layer<128, 256, ACT_RELU>(a.W[2], a.b[2], sH2, sH3, m);
      __syncthreads();
      layer<256, 256, ACT_RELU>(a.W[3], a.b[3], sH3, sF, m);
      __syncthreads();
      for (int idx = tid; idx < RC * 256; idx += blockDim.x) sF[idx] += sH3[idx];   // residual
      __syncthreads();
      layer<256, 128, ACT_TANH>(a.W[4], a.b[4], sF, sH2, m);
      __syncthreads();
      // scores: warp w handles rows w and w + 8 (a 128-long dot, lane-strided, then shuffles)
      {
        const int w = tid >> 5, lane = tid & 31;
        for (int i = w; i < RC; i += 8) {
          float acc = 0.f;
          for (int c = lane; c < 128; c += 32) acc = fmaf(a.W[5][c], sH2[i * 128 + c], acc);
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) sA[i] = acc + a.b[5][0];
        }
      }
      __syncthreads();
      // online softmax pooling over the chunk's m rows (every thread reads the same scores)
      float cm = -INFINITY;
      for (int i = 0; i < m; ++i) cm = fmaxf(cm, sA[i]);
      const float Mn = fmaxf(M, cm);
      const float scale = expf(M - Mn);      // M = -inf on the first chunk: scale 0
      Z *= scale;
      g *= scale;
      for (int i = 0; i < m; ++i) {
        const float e = expf(sA[i] - Mn);
        Z += e;
        g = fmaf(e, sF[i * 256 + tid], g);
      }
      M = Mn;
      if (a.attn && tid < m) a.attn[base + c0 + tid] = sA[tid];   // raw score, scaled below
      __syncthreads();
    }
    sG[tid] = g / Z;
    __syncthreads();
    if (tid < 128) {
      float acc = a.b[6][tid];
      const float* w = a.W[6] + (size_t)tid * 256;
      for (int c = 0; c < 256; ++c) acc = fmaf(w[c], sG[c], acc);
      sZ[tid] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    if (tid < 8) {
      float acc = a.b[7][tid];
      const float* w = a.W[7] + (size_t)tid * 128;
      for (int c = 0; c < 128; ++c) acc = fmaf(w[c], sZ[c], acc);
      a.taxels[(size_t)p * 8 + tid] = acc;
    }
    if (a.attn) {
      // the raw scores of this pad were written by this CTA; make them visible block-wide
      __threadfence_block();
      __syncthreads();
      const float invZ = 1.f / Z;
      for (int i = tid; i < n; i += blockDim.x)
        a.attn[base + i] = expf(a.attn[base + i] - M) * invZ;
    }
    __syncthreads();
  }
}

}  // namespace

namespace etac {

cudaError_t launch_regress_plain(const RegArgs& a, int num_sms, cudaStream_t s) {
  if (a.num_pads <= 0) return cudaSuccess;
  const int grid = a.num_pads < 8 * num_sms ? a.num_pads : 8 * num_sms;
  regress_plain_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace etac
