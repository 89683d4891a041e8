// Arithmetic peak probes: the FP32 and FP64 fused multiply-add rates this GPU
// sustains, measured by a kernel that does nothing else.  The path's kernels
// are bound by the FP32 pipe (distance tests) or, where decisions are taken in
// double precision, by the FP64 pipe; their roofline fractions divide by
// these measured rates instead of a rate derived from unit counts and a
// nominal clock.
#include <cuda_runtime.h>

#include <cstdint>

#include "gfs.h"

namespace {

constexpr int kChains = 16;   // independent accumulators per thread (hides the FMA latency)
constexpr int kUnroll = 8;    // FMAs per chain per loop trip (loop overhead < 3% of the issue slots)
constexpr int kThreads = 256;

// Each thread runs kChains independent chains x <- x * a + b.  With a just
// below 1 and b small the values stay bounded; the final sum is stored so the
// chains cannot be removed.
template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(T* __restrict__ sink, int64_t iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" int gfs_fma_probe(int fp64, int64_t iters, int blocks_per_sm, void* sink, int64_t sink_bytes,
                             void* cuda_stream, double* flops_host) {
  if ((fp64 != 0 && fp64 != 1) || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !sink || !flops_host)
    return GFS_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return GFS_ERR_CUDA;
  }
  const int64_t blocks = int64_t(sms) * blocks_per_sm;
  const int64_t threads = blocks * kThreads;
  if (sink_bytes < threads * int64_t(fp64 ? sizeof(double) : sizeof(float))) return GFS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (fp64)
    k_fma_probe<double><<<unsigned(blocks), kThreads, 0, st>>>(static_cast<double*>(sink), iters, 0.999999, 1e-7);
  else
    k_fma_probe<float><<<unsigned(blocks), kThreads, 0, st>>>(static_cast<float*>(sink), iters, 0.9999f, 1e-5f);
  if (cudaGetLastError() != cudaSuccess) return GFS_ERR_CUDA;
  *flops_host = 2.0 * double(threads) * double(iters) * kUnroll * kChains;
  return GFS_OK;
}
