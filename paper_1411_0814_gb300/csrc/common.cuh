// Shared device-side definitions of the RSM library: the per-problem
// descriptor every batched kernel reads, the Philox4x32-10 generator and a few
// block-level helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace rsm {

constexpr int kMaxL = 32;  // columns per submatrix supported by the kernels
constexpr int kStatTrace = 46;  // stats slot of trace(M) when M is supplied by the caller
constexpr int kMaxR = 32;  // rank supported by the kernels (r < l <= 32)

// Everything a kernel needs to know about one problem of a batch.  Lives in
// device memory (an array with one entry per problem).
struct ProbDesc {
  int64_t m, n, trials;
  int32_t r, l, n_minor, variant;
  uint64_t seed;
  uint32_t pid;
  int32_t y_dtype;  // 0 = FP64, 1 = FP32
  // caller inputs
  const void* Y;
  int64_t ldy;
  const uint8_t* W;
  int64_t ldw;
  // library workspace
  uint32_t* bits;  // packed mask, n columns of ldb words
  int64_t ldb;
  int32_t* cols;        // trials x l
  int32_t* row_counts;  // trials
  double* gram;         // trials x l(l+1)/2, packed upper triangle (a <= b), row-major by a
  unsigned long long* macc;  // n x n fixed-point accumulator of M
  double* M;                 // n x n
  float2* Mdf;               // n x n, M as FP32 pairs (hi, lo) for the products M X
  void* F1;                  // npad x npad work (Cholesky factor, then A^-1), FP32 or FP64
  void* F2;                  // npad x npad work (inverse factor)
  void* Dinv;                // nblk diagonal-block inverses, 32 x 32 each
  double* X;                 // n x kx  subspace
  double* MX;                // n x kx
  double* R;                 // n x kx
  double* small;             // per-problem small matrices (k x k blocks)
  double* Kmat;              // n x q_pad products of V for the normal equations
  double* NB;                // m x q_pad normal-equation data (N_i packed, b_i)
  float* Lf;                 // FP32 normal equations only: m x r(r+1)/2 packed Cholesky factors of the N_i
                             // (row-major lower, a(a+1)/2 + b), entry 0 = -1 for rows on the minimum-norm path
  unsigned long long* counters;  // [0] accepted trials, [1] known entries, [2] max column count, [3] chol fail,
                                 // [4] underdetermined rows, [5] selected rows, [6] device waits that ran out,
                                 // [7] trace(M) in units of one minor vector (rows variant), [8] visited known
                                 // entries (coverage); 16 slots are read back
  uint32_t* visited;             // coverage: n columns of ldb words (zeroed), or NULL
  // method M2 (variant 2): row-packed mask (m rows of ldr words) and per trial B_t (k x r, FP64)
  uint32_t* rbits;
  int64_t ldr;
  double* Bt;
  // L1 forms: each trial's minor vectors (trials x l x n_minor, zero for rejected trials), the
  // reweighting parameters; the eigen stage then reads trace(M) from stats[kStatTrace]
  double* Zst;
  int32_t l1;
  int32_t irls_iters;
  double delta_v, delta_u;
  unsigned* tflag;               // 3 nblk^2 tile states of the factor launch (zeroed before it)
  int32_t* colcount;             // n: how many trials drew each column
  double* stats;                 // [0..31] eigenvalues, [32] residual num, [33] e, [34] eig residual
  // outputs
  double* U;
  int64_t ldu;
  double* V;
  int64_t ldv;
  double* debug_Z;
  double* debug_M;
  int32_t* debug_cols;
  int32_t* debug_row_counts;
  // sizes of the eigen stage
  int32_t kx;    // subspace dimension (r + extra, <= n)
  int32_t nblk;  // ceil(n / 32)
  int32_t q;     // number of normal-equation columns: r(r+1)/2 + r
  int32_t q_pad;
  int32_t status;  // device-written status of this problem
  int32_t m_given;  // 1: M was supplied by the caller (eigen stage alone); trace(M) is in stats[kStatTrace]
  int64_t slab_rows;  // rows per slab of the row-slab Gram schedule (a function of n and the Y type only)
  // normal equations on the tensor cores (FP32 form): padded N of the W x Kw product, V columns per row of
  // the FP32 V copy; V in FP32 for the FP32 residual (row j at vf32 + j * vf_ld)
  int32_t tc;  // 1: this problem's normal equations run on the tensor cores
  const void* tmap;  // TMA descriptors (128 B each) of Y and of the packed mask, or NULL
  int32_t gram_fp32;  // 1: the Gram is accumulated in plain FP32
  int32_t resv;       // 1: the FP32 residual pass of r <= 8 with 16-byte aligned columns of Y (even m)
  int32_t tc_npad;
  int32_t tc_rb;
  int32_t vf_ld;
  const float* vf32;
};

// ------------------------------------------------------------------ FP64 reciprocal and square root
// FP64 instructions issue at a small fraction of the FP32 rate on this part,
// and the correctly rounded FP64 divide and square root expand into long FP64
// sequences.  Where a last-ulp difference is harmless (pivots, rotations,
// substitutions), seed from the FP32 hardware approximation and refine with
// Newton-Raphson steps in FP64: each step squares the relative error
// (2^-22 -> 2^-44 -> below 2^-53), so two steps give about one ulp.
// Reciprocal: y <- y + y (1 - x y).  Inverse square root: y <- y + y (1/2 - x y^2 / 2).
// Arguments whose FP32 conversion would overflow or underflow take the IEEE path.
__device__ __forceinline__ double rcp64(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double y = (double)__frcp_rn((float)x);
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt64(double x) {  // x > 0
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  double e = fma(-h * y, y, 0.5);
  y = fma(y, e, y);
  e = fma(-h * y, y, 0.5);
  return fma(y, e, y);
}

__device__ __forceinline__ double sqrt64(double x) {  // x >= 0
  if (!(x > 1e-30 && x < 1e30)) return sqrt(x);
  const double y = rsqrt64(x);
  const double s = x * y;
  return fma(0.5 * y, fma(-s, s, x), s);  // one correction of s = sqrt(x) with the residual x - s^2
}

// Type-generic forms for code templated on float / double.
// FP32: the hardware approximations (a few ulp), enough for rotations and pivots
// whose result is refined or rounded to FP32 anyway.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) { return rcp64(x); }
__device__ __forceinline__ float fast_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double fast_sqrt(double x) { return sqrt64(x); }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt64(x); }

// ------------------------------------------------------------------ asynchronous copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Global -> shared copies without register staging, grouped and waited on per stage.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {  // 0: zero fill
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {  // 0: zero fill
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialisation attribute may be scheduled as soon as every CTA of its
// predecessor on the stream has exited, before that grid's completion and
// memory flush; pdl_enter() (griddepcontrol.wait; a no-op for a normal launch)
// blocks until the predecessor has completed and its memory is visible.  It is
// the first statement of every kernel launched that way, before any access to
// memory.  No kernel signals its dependents early (launch_dependents): measured
// on the eigen stage's chain of small launches, the early-scheduled CTAs of the
// next launch made the chain slower, not faster.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Host side: launch `kernel` with programmatic stream serialisation (see
// pdl_enter, which the kernel must call first).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), unsigned blocks, unsigned threads, size_t smem,
                                  cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ------------------------------------------------------------------ division by a small runtime divisor
// q = floor(e / d) as a high multiply with m = ceil(2^32 / d) (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994),
// exact for e d < 2^32 (here e < 2^16, d <= 32768).  The plain integer division
// by a runtime divisor is a long instruction sequence.
struct SmallDiv {
  uint32_t d, m;
  __device__ __forceinline__ explicit SmallDiv(uint32_t dd) : d(dd), m(dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t e) const { return d > 1 ? __umulhi(e, m) : e; }
  __device__ __forceinline__ void divmod(uint32_t e, uint32_t& q, uint32_t& r) const {
    q = div(e);
    r = e - q * d;
  }
  __device__ __forceinline__ int q(int e) const { return (int)div((uint32_t)e); }
  __device__ __forceinline__ int r(int e) const { return e - (int)div((uint32_t)e) * (int)d; }
};

// ------------------------------------------------------------------ Philox4x32-10
// J. K. Salmon et al., "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
// ten rounds of the Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and
// Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox_round(uint4 x, uint32_t k0, uint32_t k1) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(m0, x.x), lo0 = m0 * x.x;
  uint32_t hi1 = __umulhi(m1, x.z), lo1 = m1 * x.z;
  return make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    if (i) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    ctr = philox_round(ctr, k0, k1);
  }
  return ctr;
}

// Index of the problem owning flat item g, given exclusive prefix sums
// offsets[0..nprob] (offsets[nprob] = total).  Binary search.
__device__ __forceinline__ int find_problem(const int64_t* offsets, int nprob, int64_t g) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Exclusive prefix sum of one int per thread over a block of NT threads.
// Returns the exclusive prefix; *total receives the block total.  Needs
// NT/32 ints of shared memory in warp_sums.  Contains __syncthreads().
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = (lane < NT / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  int base = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[NT / 32 - 1];
  return base + x - v;
}

// Fixed-point scale of the M accumulator: the largest f with
// (max column count + 1) * 2^f <= 2^61, so no sum of rounded contributions of
// magnitude <= 1 can overflow a signed 64-bit word.
__device__ __forceinline__ int macc_frac_bits(unsigned long long max_count) {
  int bits = 64 - __clzll((long long)(max_count + 1));  // ceil(log2(count + 2))
  int f = 61 - bits;
  return f > 52 ? 52 : f;
}

}  // namespace rsm
