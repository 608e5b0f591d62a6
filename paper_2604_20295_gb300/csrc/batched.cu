// batched.cu -- the batched FP32 ETac step: one persistent launch over every pad of the batch.
//
// Work items are pad instances ordered heaviest first (largest node count); persistent CTAs
// take them from a device ticket counter, so pads of uneven size balance across the SMs.
// Per pad (ETac Sec. III-A):
//   1. contact on every node (df32 decisions), active set compacted in node order with warp
//      ballots; active nodes keep u_hat (Eq. 4 only covers passive ones);
//   2. residual network, factored through the per-type tables: only active nodes run the
//      encoder (their first layer is c_i + W1[:, 6:9] u_hat_i); passive nodes' encoder
//      outputs f0_i are table entries, so the channel max-pool over them is the first
//      passive node in the table's per-channel order; global MLP; decoder global half
//      beta = D1[:, 64:128] g;
//   3. every passive node: Omega U_a (Eq. 1, Omega from the per-type table, or evaluated on
//      the fly, exp(-alpha |p_j - p_i|) with the table's own FP32 expression, when the table
//      would not fit or is not wanted: pads of per-instance geometry defeat caching) plus
//      Phi_p = D2 ReLU(h0_i + beta) + b (Eq. 4).
// The algebra equals the literal network exactly; only rounding order differs.
#include "etac_common.cuh"
#include "etac_kernels.h"

namespace etac {

constexpr int BT = 256;
constexpr int BW = BT / 32;

struct BatchedSmem {
  // byte offsets of every shared array for a given nmax / K
  size_t w2, b2, w1u, w4, b4, g, beta, red, redi, actu, actp, actidx, mask, warp, po, total;
  __host__ __device__ BatchedSmem(int nmax, int K, bool otf) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
      size_t r = o;
      o = (o + bytes + 15) & ~size_t(15);
      return r;
    };
    w2 = take(sizeof(float) * H * H);
    b2 = take(sizeof(float) * H);
    w1u = take(sizeof(float) * H * 4);
    w4 = take(sizeof(float) * 3 * H);
    b4 = take(sizeof(float) * 4);
    g = take(sizeof(float) * H);
    beta = take(sizeof(float) * H);
    red = take(sizeof(float) * BW * H);
    redi = take(sizeof(int) * BW * H);
    actu = take(sizeof(float4) * (size_t)nmax);     // u_hat (and, on the fly, p.x in w)
    actp = take(otf ? sizeof(float2) * (size_t)nmax : 0);   // on the fly: p.y, p.z
    actidx = take(sizeof(int16_t) * (size_t)nmax);
    mask = take(sizeof(uint8_t) * (size_t)nmax);
    warp = take(sizeof(int) * (BW + 4));
    po = take(sizeof(PadObj) * (size_t)K);
    total = o;
  }
};

// MESH: the context has mesh objects (the mesh queries are compiled in); OTF: Omega on the fly
// (a.omega is null)
template <bool MESH, bool OTF>
__global__ void __launch_bounds__(BT, 2) batched_forward_kernel(BatchedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.skip && *a.skip) return;
  __shared__ int s_item;
  const BatchedSmem L(a.nmax, a.K, OTF);
  float* sW2 = reinterpret_cast<float*>(smem + L.w2);
  float* sB2 = reinterpret_cast<float*>(smem + L.b2);
  float* sW1u = reinterpret_cast<float*>(smem + L.w1u);   // [H][4]: weights on u_hat
  float* sW4 = reinterpret_cast<float*>(smem + L.w4);
  float* sB4 = reinterpret_cast<float*>(smem + L.b4);
  float* sG = reinterpret_cast<float*>(smem + L.g);
  float* sBeta = reinterpret_cast<float*>(smem + L.beta);
  float* sRed = reinterpret_cast<float*>(smem + L.red);
  int* sRedI = reinterpret_cast<int*>(smem + L.redi);   // maximising node per (warp, channel)
  float4* sActU = reinterpret_cast<float4*>(smem + L.actu);
  float2* sActP = reinterpret_cast<float2*>(smem + L.actp);   // OTF only
  int16_t* sActIdx = reinterpret_cast<int16_t*>(smem + L.actidx);
  uint8_t* sMask = reinterpret_cast<uint8_t*>(smem + L.mask);
  int* sWarp = reinterpret_cast<int*>(smem + L.warp);
  PadObj* spo = reinterpret_cast<PadObj*>(smem + L.po);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* W = a.params;
  for (int i = tid; i < H * H; i += BT) sW2[i] = W[OFF_W2 + i];
  for (int i = tid; i < H; i += BT) {
    sB2[i] = W[OFF_B2 + i];
    sW1u[4 * i + 0] = W[OFF_W1 + i * NIN + 6];
    sW1u[4 * i + 1] = W[OFF_W1 + i * NIN + 7];
    sW1u[4 * i + 2] = W[OFF_W1 + i * NIN + 8];
    sW1u[4 * i + 3] = 0.f;
  }
  for (int i = tid; i < 3 * H; i += BT) sW4[i] = W[OFF_W4 + i];
  if (tid < 3) sB4[tid] = W[OFF_B4 + tid];
  const unsigned lt_mask = (1u << lane) - 1u;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = atomicAdd(a.ticket, 1);
      sWarp[BW] = 0;   // invalid-input flag
    }
    __syncthreads();
    const int item = s_item;
    if (item >= a.num_items) break;
    const int pad = a.item_pad[item];
    const int env = pad / a.P;
    const int ty = a.pad_type[pad];
    const int o = a.type_off[ty];
    const int n = a.type_off[ty + 1] - o;
    const long long base = a.pad_off[pad];
    const float* tpos = a.type_pos + 3 * (size_t)o;
    const float* tnrm = a.type_nrm + 3 * (size_t)o;
    if (!ETAC_IN(a.status, base + n - 1, a.num_nodes)) continue;   // block-uniform

    const bool given = a.mask_in != nullptr;   // mode B: contact supplied by the caller
    if (tid < a.K && !given) {
      const int ob = env * a.K + tid;
      const float* op = a.obj_pose + 7 * (size_t)ob;
      const float* pp = a.pad_pose + 7 * (size_t)pad;
      const float* od = a.obj_dims + 3 * (size_t)ob;
      int type = a.obj_type[ob];
      if (type < OBJ_NONE || type > OBJ_MESH) type = OBJ_NONE;
      const MeshDev* mesh = nullptr;
      if (type == OBJ_MESH && !(mesh = object_mesh(od, a.meshes, a.num_meshes))) type = OBJ_NONE;
      bool ok = finite7(op) && finite7(pp) && isfinite(od[0]) && isfinite(od[1]) &&
                isfinite(od[2]);
      if (!ok && type != OBJ_NONE) {
        sWarp[BW] = 1;
        type = OBJ_NONE;
      }
      setup_pad_obj(op, type, od, pp, a.type_pmax[ty], &spo[tid], mesh);
    }
    __syncthreads();
    if (sWarp[BW]) {
      if (tid == 0) latch_status(a.status, STATUS_NONFINITE);
      for (int i = tid; i < n; i += BT) {
        float* d = a.disp + 3 * (base + i);
        d[0] = d[1] = d[2] = 0.f;
        if (a.mask) a.mask[base + i] = 0;
        if (a.pen) a.pen[base + i] = 0.f;
      }
      if (tid == 0 && a.count) a.count[pad] = 0;
      continue;
    }

    // ---- 1. contact; active set in node order
    int m = 0;
    for (int r0 = 0; r0 < n; r0 += BT) {
      const int i = r0 + tid;
      NodeContact c;
      c.active = false;
      c.phi = 0.f;
      if (i < n) {
        float3 p = make_float3(tpos[3 * i], tpos[3 * i + 1], tpos[3 * i + 2]);
        float3 nr = make_float3(tnrm[3 * i], tnrm[3 * i + 1], tnrm[3 * i + 2]);
        c = given ? contact_given(a.mask_in, a.uhat_in, base + i)
                  : contact_node<MESH>(spo, a.K, p, nr);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, c.active);
      if (lane == 0) sWarp[warp] = __popc(bal);
      __syncthreads();
      int woff = 0, tot = 0;
#pragma unroll
      for (int w = 0; w < BW; ++w) {
        const int v = sWarp[w];
        woff += w < warp ? v : 0;
        tot += v;
      }
      if (i < n) {
        sMask[i] = c.active ? 1 : 0;
        if (a.mask) a.mask[base + i] = c.active ? 1 : 0;
        if (a.pen) a.pen[base + i] = c.active ? -c.phi : 0.f;
        if (c.active) {
          const int slot = m + woff + __popc(bal & lt_mask);
          sActIdx[slot] = (int16_t)i;
          sActU[slot] = make_float4(c.u[0], c.u[1], c.u[2], OTF ? tpos[3 * i] : 0.f);
          if (OTF) sActP[slot] = make_float2(tpos[3 * i + 1], tpos[3 * i + 2]);
          float* d = a.disp + 3 * (base + i);
          d[0] = c.u[0];
          d[1] = c.u[1];
          d[2] = c.u[2];
        }
      }
      m += tot;
      __syncthreads();
    }
    if (tid == 0 && a.count) a.count[pad] = m;
    if (m == 0) {   // no contact: the whole pad is at rest
      for (int i = tid; i < n; i += BT) {
        float* d = a.disp + 3 * (base + i);
        d[0] = d[1] = d[2] = 0.f;
      }
      continue;
    }

    // ---- 2. residual network (factored)
    if (uses_residual(a.mode)) {
    float fm0 = 0.f, fm1 = 0.f;   // running max of channels lane and lane + 32
    int fi0 = 0x7fffffff, fi1 = 0x7fffffff;   // their lowest-index maximiser (node)
    for (int a0 = 0; a0 < m; a0 += BT) {
      const int aa = a0 + tid;
      const bool live = aa < m;
      float z1[H];
      if (live) {
        const int i = sActIdx[aa];
        const float4 u = sActU[aa];
        const float4* crow = reinterpret_cast<const float4*>(a.ctab + (size_t)(o + i) * H);
#pragma unroll
        for (int c4 = 0; c4 < H / 4; ++c4) {
          const float4 cv = __ldg(crow + c4);
          const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * c4 + q;
            const float4 w = *reinterpret_cast<const float4*>(sW1u + 4 * c);
            z1[c] = fmaxf(fmaf(w.x, u.x, fmaf(w.y, u.y, fmaf(w.z, u.z, cc[q]))), 0.f);
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < H; ++c) z1[c] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < H; ++c) {
        float acc = sB2[c];
        const float4* wr = reinterpret_cast<const float4*>(sW2 + c * H);
#pragma unroll
        for (int k4 = 0; k4 < H / 4; ++k4) {
          const float4 w = wr[k4];
          acc = fmaf(w.x, z1[4 * k4 + 0], acc);
          acc = fmaf(w.y, z1[4 * k4 + 1], acc);
          acc = fmaf(w.z, z1[4 * k4 + 2], acc);
          acc = fmaf(w.w, z1[4 * k4 + 3], acc);
        }
        const float f = live ? fmaxf(acc, 0.f) : 0.f;
        // f >= 0, so unsigned order of the bit patterns is the float order
        const float mx = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(f)));
        if (a.g0arg) {
          // the lowest active slot holding the maximum: slots are in node order
          const unsigned hold = __ballot_sync(0xffffffffu, live && f == mx);
          const int node = hold ? (int)sActIdx[a0 + 32 * warp + __ffs(hold) - 1] : 0x7fffffff;
          if (lane == (c & 31)) {
            float& fm = c < 32 ? fm0 : fm1;
            int& fi = c < 32 ? fi0 : fi1;
            if (mx > fm || (mx == fm && node < fi)) {
              fm = mx;
              fi = node;
            }
          }
        } else if (c < 32) {
          if (lane == c) fm0 = fmaxf(fm0, mx);
        } else {
          if (lane == c - 32) fm1 = fmaxf(fm1, mx);
        }
      }
    }
    sRed[warp * H + lane] = fm0;
    sRed[warp * H + 32 + lane] = fm1;
    if (a.g0arg) {
      sRedI[warp * H + lane] = fi0;
      sRedI[warp * H + 32 + lane] = fi1;
    }
    __syncthreads();
    

      if (tid < H) {
        float g0 = 0.f;
        int gi = 0x7fffffff;
#pragma unroll
        for (int w = 0; w < BW; ++w) {
          const float v = sRed[w * H + tid];
          if (a.g0arg) {
            const int id = sRedI[w * H + tid];
            if (v > g0 || (v == g0 && id < gi)) {
              g0 = v;
              gi = id;
            }
          } else {
            g0 = fmaxf(g0, v);
          }
        }
        // passive maximum: first passive node in this channel's descending order of f0
        const int16_t* ord = a.order + (size_t)H * o + (size_t)tid * n;
        for (int r = 0; r < n; ++r) {
          const int idx = ord[r];
          if (!sMask[idx]) {
            const float v = __ldg(a.f0tab + (size_t)(o + idx) * H + tid);
            if (v > g0 || (v == g0 && idx < gi)) {
              g0 = v;
              gi = idx;
            }
            break;
          }
        }
        sG[tid] = g0;
        if (a.g0arg) {   // the forward state the reverse mode differentiates
          a.g0rec[(size_t)pad * H + tid] = g0;
          a.g0arg[(size_t)pad * H + tid] = gi;
        }
      }
      __syncthreads();
      {
        // global MLP and the decoder's global half, 4 partial sums per output on 256 threads
        const int u = tid & (H - 1), part = tid >> 6;
        float acc = 0.f;
        const float* wr = W + OFF_WG + u * H + part * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(__ldg(wr + k), sG[part * 16 + k], acc);
        sRed[part * H + u] = acc;
        __syncthreads();
        if (tid < H) {
          const float gsum = W[OFF_BG + tid] + sRed[tid] + sRed[H + tid] + sRed[2 * H + tid] +
                             sRed[3 * H + tid];
          sG[tid] = fmaxf(gsum, 0.f);
        }
        __syncthreads();
        acc = 0.f;
        const float* wd = W + OFF_WD + u * 2 * H + H + part * 16;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(__ldg(wd + k), sG[part * 16 + k], acc);
        sRed[part * H + u] = acc;
        __syncthreads();
        if (tid < H) sBeta[tid] = sRed[tid] + sRed[H + tid] + sRed[2 * H + tid] + sRed[3 * H + tid];
        __syncthreads();
      }
    }


    // ---- 3. passive nodes: Eq. 4
    // residual of passive node i and the store (l: its propagated term)
    auto finish = [&](int i, float l0, float l1, float l2) {
      if (uses_residual(a.mode)) {
        float r0 = sB4[0], r1 = sB4[1], r2 = sB4[2];
        const float4* hrow = reinterpret_cast<const float4*>(a.h0tab + (size_t)(o + i) * H);
#pragma unroll
        for (int c4 = 0; c4 < H / 4; ++c4) {
          const float4 hv = __ldg(hrow + c4);
          const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * c4 + q;
            const float z = fmaxf(hh[q] + sBeta[c], 0.f);
            r0 = fmaf(sW4[c], z, r0);
            r1 = fmaf(sW4[H + c], z, r1);
            r2 = fmaf(sW4[2 * H + c], z, r2);
          }
        }
        l0 += r0;
        l1 += r1;
        l2 += r2;
      }
      float* d = a.disp + 3 * (base + i);
      d[0] = l0;
      d[1] = l1;
      d[2] = l2;
    };
    if constexpr (OTF) {
      // Omega_ji = exp(-alpha |p_j - p_i|), the per-type table's expression (bit for bit),
      // with the active node's position staged in shared memory beside its u_hat.  Each thread
      // takes two passive nodes at a time (two independent chains; each node still sums its
      // active nodes in order)
      const float alpha = W[OFF_ALPHA];
      for (int i = tid; i < n; i += 2 * BT) {
        const int i2 = i + BT;
        const bool pa = !sMask[i], pb = i2 < n && !sMask[i2];
        if (!pa && !pb) continue;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f;
        if (uses_propagation(a.mode)) {
          const int ib = pb ? i2 : i;
          const float pax = tpos[3 * i], pay = tpos[3 * i + 1], paz = tpos[3 * i + 2];
          const float pbx = tpos[3 * ib], pby = tpos[3 * ib + 1], pbz = tpos[3 * ib + 2];
#pragma unroll 2
          for (int aa = 0; aa < m; ++aa) {
            const float4 u = sActU[aa];
            const float2 pyz = sActP[aa];
            const float dxa = u.w - pax, dya = pyz.x - pay, dza = pyz.y - paz;
            const float dxb = u.w - pbx, dyb = pyz.x - pby, dzb = pyz.y - pbz;
            const float wa = expf(-alpha * sqrtf(fmaf(dza, dza, fmaf(dya, dya, dxa * dxa))));
            const float wb = expf(-alpha * sqrtf(fmaf(dzb, dzb, fmaf(dyb, dyb, dxb * dxb))));
            a0 = fmaf(wa, u.x, a0);
            a1 = fmaf(wa, u.y, a1);
            a2 = fmaf(wa, u.z, a2);
            b0 = fmaf(wb, u.x, b0);
            b1 = fmaf(wb, u.y, b1);
            b2 = fmaf(wb, u.z, b2);
          }
        }
        if (pa) finish(i, a0, a1, a2);
        if (pb) finish(i2, b0, b1, b2);
      }
    } else {
      const float* Om = a.omega + a.omega_off[ty];
      for (int i = tid; i < n; i += BT) {
        if (sMask[i]) continue;
        float l0 = 0.f, l1 = 0.f, l2 = 0.f;
        if (uses_propagation(a.mode)) {
          const float* col = Om + i;
#pragma unroll 4
          for (int aa = 0; aa < m; ++aa) {
            const int j = sActIdx[aa];
            const float4 u = sActU[aa];
            const float w = __ldg(col + (size_t)j * n);
            l0 = fmaf(w, u.x, l0);
            l1 = fmaf(w, u.y, l1);
            l2 = fmaf(w, u.z, l2);
          }
        }
        finish(i, l0, l1, l2);
      }
    }
  }
}

size_t batched_smem_bytes(int nmax, int K, bool otf) { return BatchedSmem(nmax, K, otf).total; }
int batched_threads() { return BT; }

template <bool MESH, bool OTF>
static cudaError_t configure_one(int nmax, int K) {
  static size_t configured = 0;
  const size_t smem = BatchedSmem(nmax, K, OTF).total;
  if (smem <= configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(batched_forward_kernel<MESH, OTF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) configured = smem;
  return e;
}

template <bool OTF>
static cudaError_t occupancy_pair(int nmax, int K, int* per_sm) {
  const size_t smem = BatchedSmem(nmax, K, OTF).total;
  cudaError_t e = configure_one<false, OTF>(nmax, K);
  if (e == cudaSuccess) e = configure_one<true, OTF>(nmax, K);
  int x = 0, y = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, batched_forward_kernel<false, OTF>, BT, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&y, batched_forward_kernel<true, OTF>, BT, smem);
  *per_sm = x < y ? x : y;   // the grid suits the mesh and the primitive instantiation
  return e;
}

cudaError_t batched_occupancy(int nmax, int K, bool otf, int* blocks_per_sm) {
  return otf ? occupancy_pair<true>(nmax, K, blocks_per_sm)
             : occupancy_pair<false>(nmax, K, blocks_per_sm);
}

cudaError_t launch_batched_forward(const BatchedArgs& a, int grid, cudaStream_t s) {
  const bool otf = a.omega == nullptr;
  const size_t smem = BatchedSmem(a.nmax, a.K, otf).total;
  cudaError_t e = cudaSuccess;
  if (a.num_meshes > 0) {
    if (otf) {
      if ((e = configure_one<true, true>(a.nmax, a.K)) == cudaSuccess)
        batched_forward_kernel<true, true><<<grid, BT, smem, s>>>(a);
    } else {
      if ((e = configure_one<true, false>(a.nmax, a.K)) == cudaSuccess)
        batched_forward_kernel<true, false><<<grid, BT, smem, s>>>(a);
    }
  } else {
    if (otf) {
      if ((e = configure_one<false, true>(a.nmax, a.K)) == cudaSuccess)
        batched_forward_kernel<false, true><<<grid, BT, smem, s>>>(a);
    } else {
      if ((e = configure_one<false, false>(a.nmax, a.K)) == cudaSuccess)
        batched_forward_kernel<false, false><<<grid, BT, smem, s>>>(a);
    }
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace etac
