// etac_kernels.h -- launch interfaces between the C-ABI host code and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace etac {

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
};
cudaError_t launch_batched_forward(const BatchedArgs& a, int grid, cudaStream_t s);
size_t batched_smem_bytes(int nmax, int K);
int batched_threads();
cudaError_t batched_occupancy(int nmax, int K, int* blocks_per_sm);

}  // namespace etac
