// Gather-rate probe: the ceiling of the row-slab Gram's memory pattern.
//
// The slab Gram reads 4-byte elements of rows chosen by data from a 32 MiB
// slab of Y that stays in L2; almost every such read is a separate 32-byte L2
// sector.  This kernel measures how many such reads the GPU serves per second:
// every thread issues `per_thread` 4-byte loads at pseudo-random positions of
// an L2-resident buffer (a multiplicative hash of the thread and load index,
// so no index array competes for bandwidth), kGather loads in flight per
// thread, and adds them up so nothing is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rsm.h"
#include "kernels.h"

namespace rsm {

namespace {
constexpr int kGather = 8;  // independent loads in flight per thread
}

__global__ void __launch_bounds__(256) k_probe_gather(const float* __restrict__ buf, uint32_t mask, int per_thread,
                                                     float* __restrict__ out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t h = tid * 0x9E3779B1u + 0x7F4A7C15u;
  float acc = 0.f;
  for (int k = 0; k < per_thread; k += kGather) {
    float v[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      h = h * 1664525u + 1013904223u;
      v[q] = __ldg(buf + ((h >> 3) & mask));
    }
#pragma unroll
    for (int q = 0; q < kGather; ++q) acc += v[q];
  }
  if (acc == 1.2345f) out[tid] = acc;  // practically never: keeps the loads alive
}

}  // namespace rsm

extern "C" int32_t rsm_probe_gather(const float* buf, int64_t elems, int64_t blocks, int32_t per_thread, float* out,
                                    void* stream) {
  if (!buf || !out || elems < 1024 || (elems & (elems - 1)) != 0 || elems > ((int64_t)1 << 31) || blocks < 1 ||
      blocks > (1 << 20) || per_thread < 8 || per_thread % 8 != 0)
    return RSM_ERR_INVALID_ARG;
  rsm::k_probe_gather<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(buf, (uint32_t)(elems - 1),
                                                                                       per_thread, out);
  return cudaGetLastError() == cudaSuccess ? RSM_OK : RSM_ERR_CUDA;
}
