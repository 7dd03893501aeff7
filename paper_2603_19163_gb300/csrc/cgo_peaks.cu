// Gather-rate microbenchmarks: the denominators of the gather view of the
// roofline.  The search reads its instance data by random gathers (tour
// positions and distance-matrix entries), so the relevant peak is the rate of
// random element gathers a kernel can sustain from shared memory (instance
// staged per CTA) or from an L2-resident global buffer, not a streaming copy.
// Every thread runs eight independent chains of linear-congruential indices
// (one multiply-add per gather), so the loads, not the index arithmetic, set
// the pace.
#include <cstdint>
#include <cuda_runtime.h>

#include "cgo.h"
#include "cgo_internal.h"

namespace cgo {

namespace {

constexpr int kChains = 8;
constexpr uint32_t kLcgA = 1664525u, kLcgC = 1013904223u;  // Numerical Recipes LCG

// Random 16-bit gathers from a shared buffer of 2^log2n elements.
__global__ void __launch_bounds__(1024, 1)
    smem_gather_kernel(int log2n, int iters, uint32_t seed, uint32_t *out) {
  extern __shared__ int16_t buf[];
  const int n = 1 << log2n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = (int16_t)(i * 7 + 3);
  __syncthreads();
  const uint32_t mask = (uint32_t)n - 1u;
  uint32_t x[kChains];
  int acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    x[c] = seed ^ (blockIdx.x * 0x9E3779B9u) ^ (threadIdx.x * 0x85EBCA6Bu) ^ (c * 0xC2B2AE35u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      x[c] = x[c] * kLcgA + kLcgC;
      acc += buf[(x[c] >> 8) & mask];
    }
  }
  if (acc == 0x7FFFFFFF) out[0] = (uint32_t)acc;  // keeps the loads; never true in practice
}

// Random 32-bit gathers from a global buffer of 2^log2n elements (L2-resident
// when the buffer fits the L2).
__global__ void __launch_bounds__(256)
    global_gather_kernel(const int32_t *__restrict__ buf, int log2n, int iters, uint32_t seed,
                         uint32_t *out) {
  const uint32_t mask = (1u << log2n) - 1u;
  uint32_t x[kChains];
  int acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    x[c] = seed ^ (blockIdx.x * 0x9E3779B9u) ^ (threadIdx.x * 0x85EBCA6Bu) ^ (c * 0xC2B2AE35u);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      x[c] = x[c] * kLcgA + kLcgC;
      acc += __ldcg(buf + ((x[c] >> 6) & mask));
    }
  }
  if (acc == 0x7FFFFFFF) out[0] = (uint32_t)acc;
}

__global__ void fill_kernel(int32_t *buf, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = (int32_t)(i * 2654435761u);
}

}  // namespace

cudaError_t measure_gather_peak(int kind, int log2n, double *per_s, double *ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t *d_out = nullptr;
  int32_t *d_buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  double gathers = 0.0;
  float ms = 0.f;
  auto done = [&](cudaError_t r) {
    if (d_out) cudaFree(d_out);
    if (d_buf) cudaFree(d_buf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return r;
  };
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return done(e);
  if ((e = cudaMalloc(&d_out, 16)) != cudaSuccess) return done(e);
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    return done(e);
  const int iters = 4096;
  if (kind == 0) {
    const size_t smem = (size_t)2 << log2n;
    if ((e = cudaFuncSetAttribute(smem_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return done(e);
    const int grid = sms, block = 1024;
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, st);
      smem_gather_kernel<<<grid, block, smem, st>>>(log2n, iters, 12345u + rep, d_out);
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return done(e);
    }
    note_launches(2);
    gathers = (double)grid * block * iters * kChains;
  } else {
    const int64_t n = (int64_t)1 << log2n;
    if ((e = cudaMalloc(&d_buf, (size_t)n * 4)) != cudaSuccess) return done(e);
    fill_kernel<<<2 * sms, 256, 0, st>>>(d_buf, n);
    const int grid = 8 * sms, block = 256;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      global_gather_kernel<<<grid, block, 0, st>>>(d_buf, log2n, iters / 4, 777u + rep, d_out);
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return done(e);
    }
    note_launches(3);
    gathers = (double)grid * block * (iters / 4) * kChains;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
  if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return done(e);
  *per_s = gathers / ((double)ms / 1000.0);
  if (ms_out) *ms_out = ms;
  return done(cudaSuccess);
}

}  // namespace cgo
