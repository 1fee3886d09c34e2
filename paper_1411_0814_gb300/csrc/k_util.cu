// Small copy kernels that keep the per-call plan upload and workspace zeroing
// off the DMA engines, and gather the per-problem results for one small copy
// back.  Host buffers are pinned (cudaMallocHost) and therefore directly
// addressable from the device under unified addressing, so a kernel reads the
// plan from them: a caller's large asynchronous host-to-device copy on another
// stream (queued on a copy engine) then does not hold back a decomposition's
// first launch.
#include "common.cuh"
#include "kernels.h"

namespace rsm {

// dst[0 .. n16) = src[0 .. n16) in 16-byte words (either side may be pinned host memory).
__global__ void __launch_bounds__(256) k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void __launch_bounds__(256) k_zero16(uint4* __restrict__ dst, int64_t n16) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Per problem: counters (16 x u64) then stats (64 x f64) at stride `stride` bytes (device staging area).
__global__ void __launch_bounds__(128) k_readback(const ProbDesc* __restrict__ descs, int nprob,
                                                 unsigned char* __restrict__ host, int stride) {
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  unsigned long long* c = reinterpret_cast<unsigned long long*>(host + (size_t)p * stride);
  double* st = reinterpret_cast<double*>(host + (size_t)p * stride + 128);
  if (threadIdx.x < 16) c[threadIdx.x] = d.counters[threadIdx.x];
  if (threadIdx.x < 64) st[threadIdx.x] = d.stats[threadIdx.x];
}

// The library's FP64 reciprocal, inverse square root and square root
// (common.cuh) on an array, for tests that bound their error.
__global__ void __launch_bounds__(256) k_fp64_math(const double* __restrict__ x, int64_t count,
                                                  double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[i] = rcp64(v);
    out[count + i] = v > 0.0 ? rsqrt64(v) : 0.0;
    out[2 * count + i] = v >= 0.0 ? sqrt64(v) : 0.0;
  }
}

cudaError_t launch_fp64_math(const double* x, int64_t count, double* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = (count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096;
  k_fp64_math<<<(unsigned)blocks, 256, 0, s>>>(x, count, out);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_copy16(const void* src, void* dst, size_t bytes, cudaStream_t s) {
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 <= 0) return cudaSuccess;
  const int64_t blocks = (n16 + 255) / 256 < 1024 ? (n16 + 255) / 256 : 1024;
  k_copy16<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_zero16(void* dst, size_t bytes, cudaStream_t s) {
  const int64_t n16 = (int64_t)(bytes / 16);
  if (n16 <= 0) return cudaSuccess;
  const int64_t blocks = (n16 + 255) / 256 < 4096 ? (n16 + 255) / 256 : 4096;
  k_zero16<<<(unsigned)blocks, 256, 0, s>>>(static_cast<uint4*>(dst), n16);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_readback(const ProbDesc* descs, int nprob, void* host, int stride, cudaStream_t s) {
  k_readback<<<nprob, 128, 0, s>>>(descs, nprob, static_cast<unsigned char*>(host), stride);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
