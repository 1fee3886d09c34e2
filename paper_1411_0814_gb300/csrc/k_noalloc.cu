// rsm_residual_noalloc: the RMS residual e over the known entries for a given
// U and V, computed without allocating any device memory.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// the error - a process whose device memory belongs to its own fixed pool and
// forbids the runtime allocator, or a latency-bound loop that must not pay the
// device synchronisation an allocation or a free can cause.  The regular path
// keeps its per-block partial sums in workspace that rsm_decompose allocates;
// this variant keeps them in a fixed array that lives in the library image.
//
// The scratch is the file-scope array g_residual_scratch below: kMaxBlocks
// partial sums (one per 256 rows), 256 KiB, which caps m at kMaxBlocks * 256
// = 4,194,304 rows.  Every GPU that loads the library holds that array until the
// process exits.  Every call uses the same array and leaves its contents behind;
// each call overwrites every slot it reads, so nothing has to start at zero, but
// two calls that run at the same time on the GPU (different streams, or
// different host threads) race on the array and produce wrong results.
//
// Host code must not pass &g_residual_scratch to a kernel: on the host that name
// is only a stand-in, not the device address.  The first call on each device
// (with that device current) resolves the address once with
// cudaGetSymbolAddress and caches it; make that first call before any stream
// capture begins, since the lookup itself is not enqueued work.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/rsm.h"

namespace rsm {
void set_last_error(const std::string& msg);  // defined with the rest of the C ABI
}

namespace {

constexpr int kThreads = 256;           // rows per block
constexpr int64_t kMaxBlocks = 16384;   // partial sums the scratch array holds
constexpr int kMaxRank = 32;
constexpr int kMaxDevices = 64;

struct Partial {
  double sum;               // sum over the block's known entries of (y - u.v)^2
  unsigned long long known;  // known entries of the block
};

static __device__ __align__(256) Partial g_residual_scratch[kMaxBlocks];

// One thread per row: squared residuals over the known entries of the row.
// V is staged in shared memory 32 columns at a time; the mask is read as bytes.
__global__ void __launch_bounds__(kThreads) k_residual_rows_noalloc(const void* __restrict__ Y, int64_t ldy,
                                                                    int y_dtype, const uint8_t* __restrict__ W,
                                                                    int64_t ldw, const double* __restrict__ U,
                                                                    int64_t ldu, const double* __restrict__ V,
                                                                    int64_t ldv, int64_t m, int64_t n, int r,
                                                                    Partial* __restrict__ scratch) {
  __shared__ double vs[32][kMaxRank + 1];
  __shared__ double red[kThreads];
  __shared__ unsigned long long cnt[kThreads];
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double u[kMaxRank];
  for (int a = 0; a < kMaxRank; ++a) u[a] = 0.0;
  if (i < m)
    for (int a = 0; a < r; ++a) u[a] = U[(int64_t)a * ldu + i];
  double acc = 0.0;
  unsigned long long known = 0;
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * r; e += kThreads) {
      const int jj = e / r, a = e % r;
      const int64_t j = j0 + jj;
      vs[jj][a] = j < n ? V[(int64_t)a * ldv + j] : 0.0;
    }
    __syncthreads();
    if (i < m) {
      const int64_t jn = n - j0 < 32 ? n - j0 : 32;
      for (int jj = 0; jj < jn; ++jj) {
        const int64_t j = j0 + jj;
        if (!W[j * ldw + i]) continue;
        double pred = 0.0;
        for (int a = 0; a < r; ++a) pred = fma(u[a], vs[jj][a], pred);
        const double y = y_dtype == RSM_F64 ? static_cast<const double*>(Y)[j * ldy + i]
                                            : (double)static_cast<const float*>(Y)[j * ldy + i];
        const double diff = y - pred;
        acc += diff * diff;
        ++known;
      }
    }
  }
  red[threadIdx.x] = acc;
  cnt[threadIdx.x] = known;
  __syncthreads();
  for (int o = kThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      cnt[threadIdx.x] += cnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[blockIdx.x].sum = red[0];
    scratch[blockIdx.x].known = cnt[0];
  }
}

// One block: sum the partials in a fixed order and write e.
__global__ void __launch_bounds__(kThreads) k_residual_total_noalloc(const Partial* __restrict__ scratch,
                                                                     int64_t blocks, double* __restrict__ e_out) {
  __shared__ double red[kThreads];
  __shared__ unsigned long long cnt[kThreads];
  double s = 0.0;
  unsigned long long k = 0;
  for (int64_t b = threadIdx.x; b < blocks; b += kThreads) {
    s += scratch[b].sum;
    k += scratch[b].known;
  }
  red[threadIdx.x] = s;
  cnt[threadIdx.x] = k;
  __syncthreads();
  for (int o = kThreads / 2; o; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      cnt[threadIdx.x] += cnt[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *e_out = cnt[0] ? sqrt(red[0] / (double)cnt[0]) : 0.0;
}

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (resolved once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int32_t rsm_residual_noalloc(const void* Y, int64_t ldy, int32_t y_dtype, const uint8_t* W, int64_t ldw,
                                        const double* U, int64_t ldu, const double* V, int64_t ldv, int64_t m,
                                        int64_t n, int32_t r, double* e, void* stream) {
  if (!Y || !W || !U || !V || !e) {
    rsm::set_last_error("rsm_residual_noalloc: Y, W, U, V and e must be device pointers");
    return RSM_ERR_INVALID_ARG;
  }
  if (m < 1 || n < 1 || r < 1 || r > kMaxRank || ldy < m || ldw < m || ldu < m || ldv < n ||
      (y_dtype != RSM_F64 && y_dtype != RSM_F32)) {
    rsm::set_last_error("rsm_residual_noalloc: need m, n >= 1, 1 <= r <= 32, ldy, ldw, ldu >= m, ldv >= n "
                        "and y_dtype RSM_F64 or RSM_F32");
    return RSM_ERR_INVALID_ARG;
  }
  const int64_t blocks = (m + kThreads - 1) / kThreads;
  if (blocks > kMaxBlocks) {
    rsm::set_last_error("rsm_residual_noalloc: m = " + std::to_string(m) + " exceeds the " +
                        std::to_string(kMaxBlocks * kThreads) + "-row limit of its fixed scratch array");
    return RSM_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  cudaError_t err = scratch_address(&scratch);
  if (err != cudaSuccess) {
    rsm::set_last_error(std::string("rsm_residual_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(err));
    return RSM_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Partial* part = static_cast<Partial*>(scratch);
  k_residual_rows_noalloc<<<(unsigned)blocks, kThreads, 0, s>>>(Y, ldy, y_dtype, W, ldw, U, ldu, V, ldv, m, n, r,
                                                                 part);
  k_residual_total_noalloc<<<1, kThreads, 0, s>>>(part, blocks, e);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    rsm::set_last_error(std::string("rsm_residual_noalloc: launch: ") + cudaGetErrorString(err));
    return RSM_ERR_CUDA;
  }
  return RSM_OK;
}
