// noalloc.cu — per-replica energy reduction that allocates nothing.
//
// A variant of the per-replica energy sum the force gather accumulates
// (the sum over each replica of the per-atom energies), computed here from
// the per-atom energies with all of its scratch in one file-scope device
// array: no cudaMalloc/cudaFree and no allocating library call, ever. It
// serves callers that cannot allocate device memory while they read
// energies: programs whose GPU memory belongs to another framework's caching
// allocator (a cudaMalloc could fail or make that allocator release memory),
// monitoring between steps (a cudaFree synchronises the whole device), long
// runs that must not run out of memory after they start. The array (about
// 156 KB) stays resident on every GPU that loads the library until exit.
//
// Scratch layout (NA_BLOCKS x NA_REPS doubles of block partials, then one
// row of results, then the last-block counter):
//   * the block partials are overwritten in full by every launch, so
//     nothing there has to start at zero;
//   * the counter must be zero when a launch starts: it is zero from static
//     initialisation and the last block of every launch resets it.
// Limits: at most NA_REPS replicas per system (larger systems are rejected
// with an error, never truncated); any atom count (the grid strides).
//
// The symbol's address is looked up when a system is created
// (noalloc_setup, called by ctbop_create with the system's device current),
// kept with that system and passed to the kernel; device code could name the
// array directly, host code only through this address. The lookup also loads
// this file's kernels if the runtime loads modules lazily, so that an
// energy_noalloc call neither loads a module nor looks anything up. A device
// reset destroys every system of that device, and the next system created
// looks the address up again, so a kept address never outlives its module.
// Concurrent calls share the one scratch array and race; callers must not
// overlap them, on any stream.
#include <string>

#include "internal.cuh"
#include "kernels.h"

namespace ct {

#define NA_BLOCKS 304   // 2 blocks per SM on 152 SMs
#define NA_REPS 64
#define NA_THREADS 256

struct NoallocScratch {
  double part[NA_BLOCKS][NA_REPS];
  double result[NA_REPS];
  unsigned counter;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__global__ void __launch_bounds__(NA_THREADS)
    k_energy_noalloc(int N, int R, const double* __restrict__ e_atom, const int* __restrict__ rep,
                     NoallocScratch* __restrict__ sc) {
  __shared__ double s_sum[NA_REPS];
  __shared__ bool am_last;
  for (int r = threadIdx.x; r < NA_REPS; r += blockDim.x) s_sum[r] = 0.0;
  __syncthreads();
  // per-thread run over consecutive atoms of one replica, flushed to
  // shared memory when the replica changes
  int cur = -1;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    int r = rep[i];
    if (r != cur) {
      if (cur >= 0) atomicAdd(&s_sum[cur], acc);
      cur = r;
      acc = 0.0;
    }
    acc += e_atom[i];
  }
  if (cur >= 0) atomicAdd(&s_sum[cur], acc);
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) sc->part[blockIdx.x][r] = s_sum[r];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&sc->counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // the last block sums the partials in block order and resets the counter
  // for the next launch (inside a block the shared-memory atomics add in a
  // varying order, so results agree to rounding, not bit for bit)
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&sc->part[b][r]);
    sc->result[r] = t;
  }
  if (threadIdx.x == 0) sc->counter = 0u;
}

// Address of the scratch array on the current device (a system's set-up).
// Also loads this file's kernel, so the first energy_noalloc call has nothing
// left to load. Status 0 or a negative ctbop status with the reason in why.
int noalloc_setup(void** addr, std::string& why) {
  *addr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(addr, g_noalloc_scratch);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_energy_noalloc);
  if (e != cudaSuccess) {
    *addr = nullptr;
    why = std::string("energy_noalloc set-up: ") + cudaGetErrorString(e);
    return -6;
  }
  return 0;
}

// Per-replica sums of e_atom[0..N) into host_out[0..R), with the scratch at
// `scratch` (noalloc_setup's address for the system's device). Status 0 or a
// negative ctbop status with the reason in why.
int energy_noalloc(const double* e_atom, const int* rep, int N, int R, void* scratch, cudaStream_t st,
                   double* host_out, std::string& why) {
  if (R < 1 || R > NA_REPS) {
    why = "energy_noalloc: at most " + std::to_string(NA_REPS) + " replicas (its scratch is a fixed device array)";
    return -1;
  }
  if (!scratch) {
    why = "energy_noalloc: the scratch array's address was not set up";
    return -6;
  }
  NoallocScratch* sc = static_cast<NoallocScratch*>(scratch);
  int grid = (N + NA_THREADS - 1) / NA_THREADS;
  if (grid > NA_BLOCKS) grid = NA_BLOCKS;
  if (grid < 1) grid = 1;
  k_energy_noalloc<<<grid, NA_THREADS, 0, st>>>(N, R, e_atom, rep, sc);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, sc->result, sizeof(double) * R, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    why = std::string("energy_noalloc: ") + cudaGetErrorString(e);
    return -6;
  }
  return 0;
}

}  // namespace ct
