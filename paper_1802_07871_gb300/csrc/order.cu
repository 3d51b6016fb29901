// order.cu — storage order of the atoms. The caller may give its atoms in
// any order and name a storage order (ctbop_set_order): storage slot k holds
// the caller's atom order[k]. Per-atom inputs are gathered into storage
// order on the device and outputs scattered back, so every kernel works on
// storage order, where neighbouring slots are neighbouring atoms (the block
// preconditioner's blocks and the gathers of the list passes profit).
#include "internal.cuh"
#include "kernels.h"

namespace ct {

// dst[k] = src[order[k]] (to storage order) or dst[order[k]] = src[k] (back),
// elements of W words of type T.
template <class T, int W>
__global__ void k_permute(int N, const int* __restrict__ order, const T* __restrict__ src, T* __restrict__ dst,
                          int to_storage) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  size_t a = (size_t)k * W, b = (size_t)order[k] * W;
  if (to_storage) {
#pragma unroll
    for (int w = 0; w < W; ++w) dst[a + w] = src[b + w];
  } else {
#pragma unroll
    for (int w = 0; w < W; ++w) dst[b + w] = src[a + w];
  }
}

cudaError_t launch_permute(int N, const int* order, const void* src, void* dst, int elem_bytes, bool to_storage,
                           cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  dim3 g((N + 255) / 256), b(256);
  int ts = to_storage ? 1 : 0;
  switch (elem_bytes) {
    case 1: k_permute<uint8_t, 1><<<g, b, 0, st>>>(N, order, (const uint8_t*)src, (uint8_t*)dst, ts); break;
    case 4: k_permute<int, 1><<<g, b, 0, st>>>(N, order, (const int*)src, (int*)dst, ts); break;
    case 8: k_permute<double, 1><<<g, b, 0, st>>>(N, order, (const double*)src, (double*)dst, ts); break;
    case 24: k_permute<double, 3><<<g, b, 0, st>>>(N, order, (const double*)src, (double*)dst, ts); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ct
