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
