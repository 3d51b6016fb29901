// Accuracy probe of the library's FP32 reciprocal cube root (rcbrt_newton)
// against CUDA's rcbrtf, both measured against an FP64 reference, over
// log-spaced inputs. Prints: n, max relative error of rcbrt_newton, of
// rcbrtf.
#include <cstdio>
#include <cmath>
#include <vector>
#include "internal.cuh"

__global__ void k_probe(int n, const float* x, float* a, float* b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a[i] = ct::rcbrt_newton(x[i]);
    b[i] = rcbrtf(x[i]);
  }
}

int main() {
  const int n = 1 << 20;
  std::vector<float> x(n), a(n), b(n);
  for (int i = 0; i < n; ++i) x[i] = (float)std::pow(10.0, -2.0 + 6.0 * i / (n - 1));   // 1e-2 .. 1e4
  float *dx, *da, *db;
  cudaMalloc(&dx, n * 4);
  cudaMalloc(&da, n * 4);
  cudaMalloc(&db, n * 4);
  cudaMemcpy(dx, x.data(), n * 4, cudaMemcpyHostToDevice);
  k_probe<<<(n + 255) / 256, 256>>>(n, dx, da, db);
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  cudaMemcpy(a.data(), da, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(b.data(), db, n * 4, cudaMemcpyDeviceToHost);
  double ea = 0, eb = 0;
  for (int i = 0; i < n; ++i) {
    double ref = 1.0 / std::cbrt((double)x[i]);
    ea = std::fmax(ea, std::fabs(a[i] - ref) / ref);
    eb = std::fmax(eb, std::fabs(b[i] - ref) / ref);
  }
  printf("%d %.3e %.3e\n", n, ea, eb);
  return 0;
}
