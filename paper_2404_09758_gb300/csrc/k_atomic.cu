// Global float atomic throughput, the ceiling of the per-contribution AtomicAdd of Algorithm 2
// (the plain path's scatter, the transparent estimator, the fused kernels' flush).  Each thread
// issues `per_thread` fire-and-forget reductions (red.global.add.f32: the sum's result is not
// read); thread i of the grid targets address (i mod n_addr) on every round, so n_addr = the grid
// size gives one address per thread and small n_addr gives 1-of-K hot addresses.
#include <cuda_runtime.h>

#include "sge_internal.h"

namespace sge {

namespace {

__global__ void k_red_f32(float* buf, long long n_addr, int per_thread, float v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float* p = buf + (i % n_addr);
#pragma unroll 4
  for (int r = 0; r < per_thread; ++r) atomicAdd(p, v);  // result unused: compiles to RED
}

}  // namespace

cudaError_t launch_red_bench(float* buf, long long n_addr, long long n_threads, int per_thread, cudaStream_t st) {
  const long long blocks = (n_threads + 255) / 256;
  k_red_f32<<<(unsigned)blocks, 256, 0, st>>>(buf, n_addr, per_thread, 1.0f);
  return cudaGetLastError();
}

}  // namespace sge
