// peaks.cu — arithmetic-pipe peaks of the GPU, for the roofline of the
// kernels bound by arithmetic rather than by memory (the bond pass, the
// covalent force pass, the charge-force gather, the gradient passes).
//
// Each microkernel runs CH independent dependent chains per thread of one
// instruction kind (FP32 fused multiply-add, the two special-function
// instructions the path issues most, base-2 exponential and reciprocal
// square root, and FP64 fused multiply-add), on every SM at full occupancy,
// so the pipe, not the chain latency, limits the rate. The count of
// operations is exact (threads x iterations x chains); the time is CUDA
// events on the caller's stream around one launch after a warm-up launch
// sized the iteration count to about 40 ms. The SM clock during the FP32
// run is read on the device (clock64 ticks over globaltimer nanoseconds of
// each block), so a reported peak comes with the clock it was taken at.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "kernels.h"

namespace ct {

#define PK_CH 8
#define PK_THREADS 256

enum PeakOp { PK_FFMA = 0, PK_EX2 = 1, PK_RSQ = 2, PK_DFMA = 3 };

__device__ inline float pk_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ inline float pk_rsq(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void __launch_bounds__(PK_THREADS)
    k_peak(long long iters, float a, float b, float* __restrict__ sink, long long* __restrict__ ticks) {
  long long c0 = clock64();
  unsigned long long g0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  float x[PK_CH];
  double y[PK_CH];
#pragma unroll
  for (int k = 0; k < PK_CH; ++k) {
    x[k] = 1.0f + 1e-3f * (float)(threadIdx.x + k);
    y[k] = (double)x[k];
  }
  const double ad = (double)a, bd = (double)b;
  // unrolled so that the loop counter costs a few issue slots per 128
  // operations (FP32 FMA issues at one warp instruction per clock per
  // scheduler, the same rate as any instruction)
#pragma unroll 16
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PK_CH; ++k) {
      if (OP == PK_FFMA) x[k] = fmaf(x[k], a, b);
      if (OP == PK_EX2) x[k] = pk_ex2(x[k]);
      if (OP == PK_RSQ) x[k] = pk_rsq(x[k]);
      if (OP == PK_DFMA) y[k] = fma(y[k], ad, bd);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < PK_CH; ++k) s += x[k] + (float)y[k];
  if (s == 1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    ticks[2 * blockIdx.x] = clock64() - c0;
    ticks[2 * blockIdx.x + 1] = (long long)(g1 - g0);
  }
}

template <int OP>
static cudaError_t run_peak(int grid, long long iters, cudaStream_t st, float* sink, long long* ticks,
                            cudaEvent_t e0, cudaEvent_t e1, float& ms) {
  // a = 1 - 2^-20, b = 2^-20 keep the FMA chains finite; rsqrt chains settle
  // at 1, ex2 chains saturate: the special-function pipe rate does not
  // depend on the operand
  k_peak<OP><<<grid, PK_THREADS, 0, st>>>(iters, 0.99999905f, 9.5367432e-7f, sink, ticks);
  cudaEventRecord(e0, st);
  k_peak<OP><<<grid, PK_THREADS, 0, st>>>(iters, 0.99999905f, 9.5367432e-7f, sink, ticks);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return e;
  return cudaEventElapsedTime(&ms, e0, e1);
}

// Runs the four microkernels; ops_per_s[op] is operations per second
// (FMA counted as one operation), mhz the SM clock during the FP32 run.
int measure_peaks(int device, cudaStream_t st, double ops_per_s[4], double ms_out[4], double& mhz, int& sms,
                  std::string& why) {
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peak<PK_FFMA>, PK_THREADS, 0);
  if (e != cudaSuccess) {
    why = std::string("measure_peaks: ") + cudaGetErrorString(e);
    return -6;
  }
  int grid = sms * std::max(occ, 1);
  float* sink = nullptr;
  long long* ticks = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(float) * (size_t)grid * PK_THREADS);
  if (e == cudaSuccess) e = cudaMalloc(&ticks, sizeof(long long) * 2 * (size_t)grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double target_ms = 40.0;
  for (int op = 0; op < 4 && e == cudaSuccess; ++op) {
    long long iters = op == PK_DFMA ? 256 : 4096;
    float ms = 0.0f;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      switch (op) {
        case PK_FFMA: e = run_peak<PK_FFMA>(grid, iters, st, sink, ticks, e0, e1, ms); break;
        case PK_EX2: e = run_peak<PK_EX2>(grid, iters, st, sink, ticks, e0, e1, ms); break;
        case PK_RSQ: e = run_peak<PK_RSQ>(grid, iters, st, sink, ticks, e0, e1, ms); break;
        default: e = run_peak<PK_DFMA>(grid, iters, st, sink, ticks, e0, e1, ms); break;
      }
      if (pass == 0 && e == cudaSuccess) {
        double scale = target_ms / std::max((double)ms, 1e-3);
        iters = std::max(1LL, std::min((long long)(iters * scale), 1LL << 30));
      }
    }
    if (e != cudaSuccess) break;
    ms_out[op] = ms;
    ops_per_s[op] = (double)grid * PK_THREADS * (double)iters * PK_CH / (ms * 1e-3);
    if (op == PK_FFMA) {
      std::vector<long long> h(2 * (size_t)grid);
      e = cudaMemcpy(h.data(), ticks, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost);
      std::vector<double> f;
      for (int b = 0; b < grid; ++b)
        if (h[2 * b + 1] > 0) f.push_back((double)h[2 * b] / (double)h[2 * b + 1] * 1e3);   // MHz
      std::sort(f.begin(), f.end());
      mhz = f.empty() ? 0.0 : f[f.size() / 2];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (ticks) cudaFree(ticks);
  if (e != cudaSuccess) {
    why = std::string("measure_peaks: ") + cudaGetErrorString(e);
    return -6;
  }
  return 0;
}

}  // namespace ct

extern "C" int ctbop_measure_peaks(int32_t device, void* cuda_stream, ctbop_peaks* out) {
  if (!out) return CTBOP_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  double ops[4] = {0, 0, 0, 0}, ms[4] = {0, 0, 0, 0}, mhz = 0.0;
  int sms = 0;
  std::string why;
  int rc = ct::measure_peaks(device, static_cast<cudaStream_t>(cuda_stream), ops, ms, mhz, sms, why);
  if (rc) return CTBOP_ERR_CUDA;
  out->fp32_tflops = 2.0 * ops[ct::PK_FFMA] / 1e12;
  out->mufu_ex2_tops = ops[ct::PK_EX2] / 1e12;
  out->mufu_rsq_tops = ops[ct::PK_RSQ] / 1e12;
  out->fp64_tflops = 2.0 * ops[ct::PK_DFMA] / 1e12;
  for (int k = 0; k < 4; ++k) out->ms[k] = ms[k];
  out->sm_mhz = mhz;
  out->sms = sms;
  return CTBOP_OK;
}
