// Stage a7: V-hat = eigenvectors of M for its r smallest eigenvalues (eq.
// solve.barV_L2_norm: only M = Xi Xi^T is stored, and V-hat takes the vectors of
// the r smallest singular values of Xi).
//
// Method (preconditioned inverse iteration with Rayleigh-Ritz, PINVIT):
//   * A = M + tau I with a small shift tau = c * trace(M) / n is factored
//     A = L L^T (blocked right-looking Cholesky, 32 x 32 blocks), then
//     T = A^-1 = L^-T L^-1 is formed.  T is only a preconditioner.  The fast
//     form factors in FP32 with c = 1e-3 (enough when lambda_{r+1} >> tau);
//     the robust form factors in FP64 with c = 1e-11, which makes the step an
//     exact shift-invert iteration and resolves clustered small eigenvalues.
//   * A block X of kx >= r + 1 vectors is iterated in FP64:
//       Rayleigh-Ritz on span(X):  S = X^T X, H = X^T M X, S = C C^T,
//         eig(C^-1 H C^-T) = Q' diag(theta), X <- X C^-T Q'  (orthonormal Ritz basis)
//       residual R = M X - X diag(theta)
//       X <- X - T R
//     Components of X along an eigenvector with eigenvalue lambda shrink by
//     about (tau + theta) / (lambda + tau) per step, so the r smallest Ritz
//     pairs converge quickly when lambda_{r+1} >> tau.  M X and all reductions
//     are FP64, so the limiting accuracy is that of FP64 arithmetic on M.
// Every kernel is batched over the problems of the launch.
#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace rsm {

constexpr int BS = 32;  // block size of the FP32 factorisation
constexpr int kConvFlag = 40;   // stats[40] != 0: the block iteration of this problem has converged
constexpr double kConvTol = 1e-12;  // converged when max ||R_j|| <= kConvTol * (theta_{r+1} - theta_r)
constexpr double kStallTol = 1e-10;  // ... or when it stops falling (rounding floor) below kStallTol * gap
constexpr int kPrevRes = 41;         // stats[41]: max ||R_j|| at the previous check
constexpr int kIterCount = 43;       // stats[43]: block iterations run so far

// Index arithmetic of the eigen stage is 32-bit (n <= 32768 is validated on the host): 64-bit
// integer multiplies and adds are slow on this part.
__device__ __forceinline__ int npad_of(const ProbDesc& d) { return d.nblk * BS; }

template <typename T>
__device__ __forceinline__ T* F1of(const ProbDesc& d) { return static_cast<T*>(d.F1); }
template <typename T>
__device__ __forceinline__ T* F2of(const ProbDesc& d) { return static_cast<T*>(d.F2); }
template <typename T>
__device__ __forceinline__ T* Dinvof(const ProbDesc& d) { return static_cast<T*>(d.Dinv); }

// ------------------------------------------------------------------ A = M + tau I (padded with I)
template <typename T>
__global__ void __launch_bounds__(256) k_eig_prep(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                 int nprob, double shift_rel, int iter0) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - off[p];
  if (e == 0) {
    d.stats[kConvFlag] = 0.0;
    d.stats[kPrevRes] = 0.0;
    d.stats[kIterCount] = (double)iter0;  // the unchecked leading steps
  }
  const int np = npad_of(d);
  const int64_t i = e / np, j = e % np;
  const double mean = (double)d.counters[0] * d.n_minor / (double)d.n;
  const double tau = mean > 0.0 ? shift_rel * mean : 1.0;
  T v;
  if (i < d.n && j < d.n) {
    const double mij = d.M[i * d.n + j];
    v = (T)(mij + (i == j ? tau : 0.0));
    const float hi = __double2float_rn(mij);  // M as an FP32 pair for the products M X
    d.Mdf[i * d.n + j] = make_float2(hi, __double2float_rn(mij - (double)hi));
  } else {
    v = (i == j) ? (T)1 : (T)0;
  }
  F1of<T>(d)[e] = v;
}

// ------------------------------------------------------------------ Cholesky, step k
// Factor the 32 x 32 diagonal block and invert the factor with one warp, all in
// registers: lane i holds row i.  Step j takes the pivot from lane j, scales
// column j, and updates the trailing columns with L[c][j] fetched by shuffle
// from lane c (fully unrolled, so every register index is a constant).  The
// inverse X = L^-1 is formed row by row: once row t is final on lane t it is
// broadcast and every later row adds L[i][t] X[t][.] (forward substitution).
// Factor and invert one diagonal block held as a[c] = A_kk[lane][c] (row per
// lane); writes L_kk (lower, zeros above) at A and its inverse at Dinv[k].
template <typename T>
__device__ __forceinline__ void warp_potrf_block(T (&a)[BS], const ProbDesc& d, int k, int np, bool write_global,
                                                 T (*dinv_smem)[BS + 1]) {
  const int lane = threadIdx.x & 31;
  T* A = F1of<T>(d) + (int64_t)k * BS * np + (int64_t)k * BS;
  bool bad = false;
  T rinv = (T)1;  // 1 / L[lane][lane]
#pragma unroll
  for (int j = 0; j < BS; ++j) {
    T piv = __shfl_sync(0xffffffffu, a[j], j);
    if (!(piv > (T)0)) {  // not positive definite at this precision: flag, continue with a tiny pivot
      bad = true;
      piv = (T)1e-30;
    }
    const T ij = fast_rsqrt(piv);  // the FP32 factor is a preconditioner: the hardware approximation suffices
    const T dj = piv * ij;
    if (lane == j) rinv = ij;
    a[j] = lane > j ? a[j] * ij : (lane == j ? dj : (T)0);
#pragma unroll
    for (int c = j + 1; c < BS; ++c) a[c] = fma(-a[j], __shfl_sync(0xffffffffu, a[j], c), a[c]);
  }
  if (bad && lane == 0) atomicAdd(&d.counters[3], 1ull);
  T x[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) x[c] = (T)0;
#pragma unroll
  for (int t = 0; t < BS; ++t) {
    const bool me = lane == t;
#pragma unroll
    for (int c = 0; c < t; ++c) x[c] = me ? -x[c] * rinv : x[c];
    x[t] = me ? rinv : x[t];
    const T lit = lane > t ? a[t] : (T)0;  // L[lane][t] for the rows still open
#pragma unroll
    for (int c = 0; c <= t; ++c) x[c] = fma(lit, __shfl_sync(0xffffffffu, x[c], t), x[c]);
  }
  if (write_global) {
    T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      A[lane * np + c] = c <= lane ? a[c] : (T)0;
      D[lane * BS + c] = c <= lane ? x[c] : (T)0;  // entry (lane, c) of inv(L_kk)
    }
  }
  if (dinv_smem)
#pragma unroll
    for (int c = 0; c < BS; ++c) dinv_smem[lane][c] = c <= lane ? x[c] : (T)0;
}


// 32 x 32 x 32 product helper: each of 256 threads owns 4 outputs (row ty + 8s, column tx).
// out[r][c] = sum_t X[r][t] * Y(t, c) with Y accessed through the functor.

// Panel: L_ik = A_ik * inv(L_kk)^T for i > k.
// Step k of the factorisation: block column k.  CTA 0 of a problem factors
// and inverts the diagonal block A_kk and writes L_kk and inv(L_kk); CTA
// q >= 1 factors A_kk as well (the same arithmetic, so the same result, in
// parallel with CTA 0) and forms L_{k+q,k} = A_{k+q,k} inv(L_kk)^T.  One
// launch per step replaces a factorisation launch followed by a panel launch.
template <typename T>
__global__ void __launch_bounds__(256) k_panel(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                              int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  const int q = (int)(blockIdx.x - off[p]);
  if (threadIdx.x < 32) {
    const T* Akk = F1of<T>(d) + (int64_t)k * BS * np + (int64_t)k * BS;
    T a[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) a[c] = Akk[threadIdx.x * np + c];
    __syncwarp();
    warp_potrf_block<T>(a, d, k, np, q == 0, q == 0 ? nullptr : y);
  }
  if (q == 0) return;
  const int i = k + q;
  T* Aik = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)k * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) x[e / BS][e % BS] = Aik[(e / BS) * np + (e % BS)];
  __syncthreads();
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int t = 0; t < BS; ++t) {
    const T yv = y[tx][t];  // inv(L_kk)[tx][t]
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][t], yv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Aik[(ty + 8 * s) * np + tx] = acc[s];
}

__device__ __forceinline__ void tri_index(int64_t u, int& i, int& j) {
  // u -> (i, j) with 0 <= j <= i, u = i (i + 1) / 2 + j
  int r = (int)((sqrt(8.0 * (double)u + 1.0) - 1.0) * 0.5);
  while ((int64_t)(r + 1) * (r + 2) / 2 <= u) ++r;
  while ((int64_t)r * (r + 1) / 2 > u) --r;
  i = r;
  j = (int)(u - (int64_t)r * (r + 1) / 2);
}

// Trailing update: A_ij -= L_ik L_jk^T for k < j <= i.
template <typename T>
__global__ void __launch_bounds__(256) k_trail(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                              int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  int ii, jj;
  tri_index(blockIdx.x - off[p], ii, jj);
  const int i = k + 1 + ii, j = k + 1 + jj;
  const T* Lik = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)k * BS;
  const T* Ljk = F1of<T>(d) + (int64_t)j * BS * np + (int64_t)k * BS;
  T* Aij = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = Lik[(e / BS) * np + (e % BS)];
    y[e / BS][e % BS] = Ljk[(e / BS) * np + (e % BS)];
  }
  __syncthreads();
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int t = 0; t < BS; ++t) {
    const T yv = y[tx][t];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][t], yv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Aij[(ty + 8 * s) * np + tx] -= acc[s];
}

// ------------------------------------------------------------------ L^-1 (into F2)
// Right-looking block forward substitution of L X = I: X starts as I on the
// diagonal blocks and 0 below; at step k block row k is final after
// X_kj <- inv(L_kk) X_kj (j <= k), and every block X_ij (i > k, j <= k) then
// subtracts L_ik X_kj.  Each CTA does one 32 x 32 x 32 product per launch.
template <typename T>
__global__ void __launch_bounds__(256) k_linv_init(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob) {
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  int i, j;
  tri_index(blockIdx.x - off[p], i, j);
  T* out = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    const int r = e / BS, c = e % BS;
    out[r * np + c] = (i == j && r == c) ? (T)1 : (T)0;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_linv_scale(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                   int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  const int j = (int)(blockIdx.x - off[p]);  // j <= k
  T* Xkj = F2of<T>(d) + (int64_t)k * BS * np + (int64_t)j * BS;
  const T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = D[e];
    y[e / BS][e % BS] = Xkj[(e / BS) * np + (e % BS)];
  }
  __syncthreads();
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int u = 0; u < BS; ++u) {
    const T yv = y[u][tx];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][u], yv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Xkj[(ty + 8 * s) * np + tx] = acc[s];
}

template <typename T>
__global__ void __launch_bounds__(256) k_linv_update(const ProbDesc* __restrict__ descs,
                                                    const int64_t* __restrict__ off, int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  const int64_t local = blockIdx.x - off[p];
  const int i = k + 1 + (int)(local / (k + 1)), j = (int)(local % (k + 1));
  const T* Lik = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)k * BS;
  const T* Xkj = F2of<T>(d) + (int64_t)k * BS * np + (int64_t)j * BS;
  T* Xij = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = Lik[(e / BS) * np + (e % BS)];
    y[e / BS][e % BS] = Xkj[(e / BS) * np + (e % BS)];
  }
  __syncthreads();
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int u = 0; u < BS; ++u) {
    const T yv = y[u][tx];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][u], yv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Xij[(ty + 8 * s) * np + tx] -= acc[s];
}

// T = A^-1 = L^-T L^-1:  T_ij = sum_{t >= max(i, j)} Linv_ti^T Linv_tj  (into F1, both triangles)
template <typename T>
__global__ void __launch_bounds__(256) k_ainv(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                             int nprob) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int np = npad_of(d);
  int i, j;
  tri_index(blockIdx.x - off[p], i, j);  // j <= i
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int t = i; t < d.nblk; ++t) {
    const T* Lti = F2of<T>(d) + (int64_t)t * BS * np + (int64_t)i * BS;
    const T* Ltj = F2of<T>(d) + (int64_t)t * BS * np + (int64_t)j * BS;
    __syncthreads();
    for (int e = threadIdx.x; e < BS * BS; e += 256) {
      x[e / BS][e % BS] = Lti[(e / BS) * np + (e % BS)];
      y[e / BS][e % BS] = Ltj[(e / BS) * np + (e % BS)];
    }
    __syncthreads();
    for (int u = 0; u < BS; ++u) {
      const T yv = y[u][tx];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s] = fma(x[u][ty + 8 * s], yv, acc[s]);
    }
  }
  T* Tij = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  T* Tji = F1of<T>(d) + (int64_t)j * BS * np + (int64_t)i * BS;
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    Tij[(ty + 8 * s) * np + tx] = acc[s];
    x[ty + 8 * s][tx] = acc[s];
  }
  __syncthreads();
  if (i != j)
    for (int e = threadIdx.x; e < BS * BS; e += 256) Tji[(e / BS) * np + (e % BS)] = x[e % BS][e / BS];
}

// ------------------------------------------------------------------ block iteration (FP64)
// X (n x kx, row-major) starts from deterministic Philox noise in [-1, 1).
__global__ void __launch_bounds__(256) k_init_X(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - off[p];
  const uint4 w = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)(e >> 32), d.pid, 0x52534d31u), 0x9E3779B9u,
                                (uint32_t)d.seed);
  d.X[e] = ((double)w.x + 0.5) * (2.0 / 4294967296.0) - 1.0;
}

constexpr int kSplit = 32;   // split of the inner dimension of the product M X (R slots)
constexpr int kPSplit = 4;   // split of the inner dimension of the preconditioner product
constexpr int kMxRows = 128;  // rows per CTA of M X (one per thread)
constexpr int kMxSub = 64;    // columns of X staged per pass

// out = M X to about FP64 accuracy on the FP32 pipes (FP64 instructions issue
// far slower than FP32 ones here).  M is held as FP32 pairs (hi + lo, 48
// significant bits, written by k_eig_prep); X is split the same way when it is
// staged.  Per term: the head product hi*hi is split exactly (TwoProduct by
// FMA), the cross terms hi*lo + lo*hi are single FP32 products, and the running
// sum is a float pair updated by TwoSum (Knuth), so the accumulation carries
// about 2^-44 relative accuracy; the lo*lo term (2^-48) is dropped.
// Thread = row i (M is symmetric, so M[j][i] is read: consecutive threads read
// consecutive addresses); split s covers columns j in [s n / kSplit, (s+1) n / kSplit);
// the parts go to R slots and k_split_sum adds them in FP64 in a fixed order.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int KXB>
__global__ void __launch_bounds__(kMxRows) k_gemm_MX(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                    int nprob) {
  __shared__ float2 xs[kMxSub][KXB];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int local = (int)(blockIdx.x - off[p]);
  const int n = (int)d.n;
  const int kx = d.kx;
  const int ntile = (n + kMxRows - 1) / kMxRows;
  const int split = local / ntile;
  const int i = (local % ntile) * kMxRows + threadIdx.x;
  const int j_begin = split * n / kSplit, j_end = (split + 1) * n / kSplit;
  float sh[KXB], sl[KXB];
#pragma unroll
  for (int c = 0; c < KXB; ++c) sh[c] = sl[c] = 0.f;
  const float2* __restrict__ Mdf = d.Mdf;
  for (int j0 = j_begin; j0 < j_end; j0 += kMxSub) {
    const int jn = j_end - j0 < kMxSub ? j_end - j0 : kMxSub;
    __syncthreads();
    for (int e = threadIdx.x; e < jn * KXB; e += kMxRows) {
      const int jj = e / KXB, c = e % KXB;
      const double x = c < kx ? d.X[(j0 + jj) * kx + c] : 0.0;
      const float xh = __double2float_rn(x);
      xs[jj][c] = make_float2(xh, __double2float_rn(x - (double)xh));
    }
    __syncthreads();
    if (i < n) {
      for (int jj = 0; jj < jn; ++jj) {
        const float2 m = __ldg(Mdf + (j0 + jj) * n + i);
#pragma unroll
        for (int c = 0; c < KXB; ++c) {
          const float2 x = xs[jj][c];
          const float ph = __fmul_rn(m.x, x.x);
          const float pe = __fmaf_rn(m.x, x.x, -ph);
          const float cross = __fmaf_rn(m.x, x.y, __fmul_rn(m.y, x.x));
          float s, er;
          two_sum(sh[c], ph, s, er);
          sh[c] = s;
          sl[c] = __fadd_rn(sl[c], __fadd_rn(er, __fadd_rn(pe, cross)));
        }
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < KXB; ++c)
      if (c < kx) d.R[(split * n + i) * kx + c] = (double)sh[c] + (double)sl[c];
}

__global__ void __launch_bounds__(256) k_split_sum(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int e = (int)(g - off[p]);
  const int nk = (int)d.n * d.kx;
  double s = d.R[e];
  for (int q = 1; q < kSplit; ++q) s += d.R[q * nk + e];
  d.MX[e] = s;
}

// Partial Gram sums over chunks of kChunk rows: part[chunk] = [X^T X | X^T MX]
// (2 kx^2 values; the second half only when WITH_H).
constexpr int kChunk = 64;
template <bool WITH_H>
__global__ void __launch_bounds__(256) k_xtx(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                            int nprob, double* __restrict__ part_base, const int64_t* __restrict__ part_off) {
  extern __shared__ double xtx_smem[];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int chunk = (int)(blockIdx.x - off[p]);
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  double* xs = xtx_smem;                  // kChunk x kx
  double* ys = xtx_smem + kChunk * kx;    // kChunk x kx
  const int i0 = chunk * kChunk;
  for (int e = threadIdx.x; e < kChunk * kx; e += 256) {
    const int i = i0 + dkx.q(e);
    xs[e] = i < d.n ? d.X[i0 * kx + e] : 0.0;
    if (WITH_H) ys[e] = i < d.n ? d.MX[i0 * kx + e] : 0.0;
  }
  __syncthreads();
  double* part = part_base + part_off[p] + chunk * 2 * kx * kx;
  const int outs = (WITH_H ? 2 : 1) * kx * kx;
  for (int e = threadIdx.x; e < outs; e += 256) {
    const int which = e / (kx * kx), ab = e % (kx * kx), a = dkx.q(ab), b = dkx.r(ab);
    const double* y = which == 0 ? xs : ys;
    double s0 = 0.0, s1 = 0.0;
    for (int r = 0; r < kChunk; r += 2) {
      s0 = fma(xs[r * kx + a], y[r * kx + b], s0);
      s1 = fma(xs[(r + 1) * kx + a], y[(r + 1) * kx + b], s1);
    }
    part[e] = s0 + s1;
  }
}

// ------------------------------------------------------------------ small dense algebra (one CTA per problem)
constexpr int kLs = kMaxL + 1;
constexpr int kSmallThreads = 128;  // four warps: the FP64 products use all four schedulers
typedef double DRow[kLs];
typedef float FRow[kLs];

// Sum the per-chunk partials in a fixed order: S = X^T X (and H = X^T M X).
__device__ inline void reduce_partials(const ProbDesc& d, const double* part, DRow* S, DRow* H, int kx) {
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  const int nchunk = (int)((d.n + kChunk - 1) / kChunk);
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) {
    double s = 0.0, h = 0.0;
#pragma unroll 4
    for (int c = 0; c < nchunk; ++c) {
      s += part[c * 2 * kx * kx + e];
      if (H) h += part[c * 2 * kx * kx + kx * kx + e];
    }
    S[dkx.q(e)][dkx.r(e)] = s;
    if (H) H[dkx.q(e)][dkx.r(e)] = h;
  }
}

// C = op(A) B for kx x kx blocks in shared memory, all threads of the CTA.
__device__ inline void small_prod(DRow* C, const DRow* A, bool transA, const DRow* B, int kx) {
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    double s = 0.0;
    for (int t = 0; t < kx; ++t) s = fma(transA ? A[t][a] : A[a][t], B[t][b], s);
    C[a][b] = s;
  }
}

// Shifted Cholesky S + s I = C C^T in place (lower triangle), s = shift_rel
// trace(S): keeps the factor defined when the block is numerically rank
// deficient (shifted CholeskyQR).  One warp, lane i owns row i; rdiag[j] = 1 / C_jj.
template <typename CT>
__device__ inline void warp_chol_shifted(CT (*S)[kLs], CT* rdiag, int kx, CT shift_rel) {
  const int lane = threadIdx.x & 31;
  CT trS = 0;
  for (int j = 0; j < kx; ++j) trS += S[j][j];
  __syncwarp();
  if (lane < kx) S[lane][lane] += shift_rel * trS;
  __syncwarp();
  for (int j = 0; j < kx; ++j) {
    CT v = S[j][j];
    v = v > (CT)0 ? fast_sqrt(v) : (CT)1e-30;
    const CT rv = fast_rcp(v);
    __syncwarp();
    if (lane == j) {
      S[j][j] = v;
      rdiag[j] = rv;
    }
    if (lane > j && lane < kx) S[lane][j] *= rv;
    __syncwarp();
    if (lane > j && lane < kx) {
      const CT lij = S[lane][j];
      for (int c = j + 1; c <= lane; ++c) S[lane][c] -= lij * S[c][j];
    }
    __syncwarp();
  }
}

// Q = C^-T (upper triangular) by back substitution, column c per thread.
template <typename CT>
__device__ inline void inv_transpose_factor(const CT (*C)[kLs], const CT* rdiag, CT (*Q)[kLs], int kx) {
  for (int c = threadIdx.x; c < kx; c += kSmallThreads)
    for (int i = kx - 1; i >= 0; --i) {
      CT v = (i == c) ? (CT)1 : (CT)0;
      for (int t = i + 1; t < kx; ++t) v -= C[t][i] * Q[t][c];
      Q[i][c] = (i > c) ? (CT)0 : v * rdiag[i];
    }
}

// Orthonormalisation step of the subspace iteration: S = X^T X (FP64 partial
// sums), S + s I = C C^T in precision CT, small[0 .. kx^2) = Q = C^-T so that
// X Q has orthonormal columns.
template <typename CT>
__global__ void __launch_bounds__(kSmallThreads) k_orth(const ProbDesc* __restrict__ descs, int nprob,
                                                      const double* __restrict__ part_base,
                                                      const int64_t* __restrict__ part_off) {
  __shared__ CT S[kMaxL][kLs], Q[kMaxL][kLs];
  __shared__ DRow Sd[kMaxL];
  __shared__ CT rdiag[kMaxL];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  reduce_partials(d, part_base + part_off[p], Sd, nullptr, kx);
  __syncthreads();
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) S[dkx.q(e)][dkx.r(e)] = (CT)Sd[dkx.q(e)][dkx.r(e)];
  __syncthreads();
  if (threadIdx.x < 32) warp_chol_shifted<CT>(S, rdiag, kx, (CT)(sizeof(CT) == 8 ? 1e-15 : 1e-6));
  __syncthreads();
  inv_transpose_factor<CT>(S, rdiag, Q, kx);
  __syncthreads();
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) d.small[e] = (double)Q[dkx.q(e)][dkx.r(e)];
}

// Rayleigh-Ritz step of the FP64 block iteration, one CTA per problem.
// Reduce S = X^T X and H = X^T M X, factor S + s I = C C^T (FP64), Q1 = C^-T,
// H1 = Q1^T H Q1.  Then, with FP64 work kept to a few kx^3 products (FP64
// issues far slower than FP32 here, and an FP64 Jacobi sweep costs tens of
// microseconds on one warp):
//  - FP32 Jacobi on H1 gives eigenvectors to FP32 accuracy, sorted by Ritz value;
//  - two Lowdin steps Q2 <- Q2 (3I - Q2^T Q2) / 2 make them orthogonal in FP64;
//  - B = Q2^T H1 Q2 is diagonal up to the FP32 error; what matters is the
//    coupling B12 between the r wanted and the kx - r other columns, which a
//    first-order rotation removes: G = I + A with A_pq = B_pq / (B_qq - B_pp)
//    (p < r <= q, A_qp = -A_pq; the gap theta_{r+1} - theta_r keeps it
//    defined), made orthogonal by one Lowdin step.  The coupling left is
//    second order, ||B12||^2 / gap.  Mixing inside the wanted (or the other)
//    block is harmless: only the two subspaces matter.
// Writes small = [Q | H' | theta] with Q = Q1 Q2 G, H' = Q^T H Q (FP64) and
// theta = diag(H') in ascending order of the FP32 Ritz values.
constexpr size_t kRRSmem = sizeof(DRow) * kMaxL * 7 + sizeof(FRow) * kMaxL * 2;

__device__ inline void lowdin_step(DRow* Q, DRow* W1, DRow* W2, int kx) {  // Q <- Q (3I - Q^T Q) / 2
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  small_prod(W1, Q, true, Q, kx);
  __syncthreads();
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    double s = 0.0;
    for (int t = 0; t < kx; ++t) s = fma(Q[a][t], ((t == b) ? 3.0 : 0.0) - W1[t][b], s);
    W2[a][b] = 0.5 * s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) Q[dkx.q(e)][dkx.r(e)] = W2[dkx.q(e)][dkx.r(e)];
  __syncthreads();
}

__device__ inline void sym_congruence(DRow* out, const DRow* Q, const DRow* A, DRow* W, int kx) {  // out = Q^T A Q
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  small_prod(W, A, false, Q, kx);
  __syncthreads();
  for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    double s = 0.0;
    for (int t = 0; t < kx; ++t) s = fma(Q[t][lo], W[t][hi], s);
    out[a][b] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSmallThreads) k_rr64(const ProbDesc* __restrict__ descs, int nprob,
                                                      const double* __restrict__ part_base,
                                                      const int64_t* __restrict__ part_off) {
  extern __shared__ __align__(16) unsigned char rr_smem[];
  DRow* S = reinterpret_cast<DRow*>(rr_smem);
  DRow* H = S + kMaxL;
  DRow* Q1 = H + kMaxL;
  DRow* W1 = Q1 + kMaxL;
  DRow* H1 = W1 + kMaxL;
  DRow* Q2 = H1 + kMaxL;
  DRow* W2 = Q2 + kMaxL;
  FRow* Sf = reinterpret_cast<FRow*>(W2 + kMaxL);
  FRow* Vf = Sf + kMaxL;
  __shared__ JacobiScratchT<float> jsf;
  __shared__ int order[kMaxL];
  __shared__ double rdiag[kMaxL];
  __shared__ int rotated, coupled;
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int kx = d.kx, r = d.r, tid = threadIdx.x;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  reduce_partials(d, part_base + part_off[p], S, H, kx);
  __syncthreads();
  // S = X^T X is close to I here (X was orthonormalised before its last small
  // update), so: FP32 Cholesky S + s I = C C^T and Q0 = C^-T, then one
  // Newton-Schulz step in FP64, Q1 = Q0 (3I - Q0^T S Q0) / 2, which squares the
  // FP32 error: X Q1 is orthonormal to FP64 accuracy.
  for (int e = tid; e < kx * kx; e += kSmallThreads) Sf[dkx.q(e)][dkx.r(e)] = (float)S[dkx.q(e)][dkx.r(e)];
  __syncthreads();
  if (tid < 32) warp_chol_shifted<float>(Sf, reinterpret_cast<float*>(rdiag), kx, 1e-7f);
  __syncthreads();
  inv_transpose_factor<float>(Sf, reinterpret_cast<const float*>(rdiag), Vf, kx);
  __syncthreads();
  for (int e = tid; e < kx * kx; e += kSmallThreads) Q2[dkx.q(e)][dkx.r(e)] = (double)Vf[dkx.q(e)][dkx.r(e)];
  __syncthreads();
  sym_congruence(W2, Q2, S, W1, kx);  // Z = Q0^T S Q0
  for (int e = tid; e < kx * kx; e += kSmallThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    double s = 0.0;
    for (int t = 0; t < kx; ++t) s = fma(Q2[a][t], ((t == b) ? 3.0 : 0.0) - W2[t][b], s);
    Q1[a][b] = 0.5 * s;
  }
  __syncthreads();
  sym_congruence(H1, Q1, H, W1, kx);  // H1 = Q1^T H Q1
  // FP32 Jacobi of H1 when it has off-diagonal entries FP32 can resolve; then
  // the eigenvector columns in ascending order of the Ritz values
  for (int e = tid; e < kx * kx; e += kSmallThreads) Sf[dkx.q(e)][dkx.r(e)] = (float)H1[dkx.q(e)][dkx.r(e)];
  __syncthreads();
  if (tid < 32) {
    float f = 0.f, o = 0.f;
    for (int e = tid; e < kx * kx; e += 32) {
      const float v = Sf[dkx.q(e)][dkx.r(e)];
      f += v * v;
      if (dkx.q(e) != dkx.r(e)) o = fmaxf(o, fabsf(v));
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) {
      f += __shfl_xor_sync(0xffffffffu, f, s);
      o = fmaxf(o, __shfl_xor_sync(0xffffffffu, o, s));
    }
    const float tol = 4.f * FLT_EPSILON * sqrtf(f);
    int sweeps = 0;
    if (o > tol) {
      sweeps = warp_jacobi<float>(&Sf[0][0], &Vf[0][0], kx, kLs, jsf, tol);
    }
    if (tid == 0) {
      rotated = sweeps;
      coupled = 0;
      for (int i = 0; i < kx; ++i) order[i] = i;
      for (int a = 1; a < kx; ++a) {
        const int v = order[a];
        int b = a - 1;
        while (b >= 0 && Sf[order[b]][order[b]] > Sf[v][v]) {
          order[b + 1] = order[b];
          --b;
        }
        order[b + 1] = v;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < kx * kx; e += kSmallThreads)
    Q2[dkx.q(e)][dkx.r(e)] = rotated ? (double)Vf[dkx.q(e)][order[dkx.r(e)]] : (dkx.q(e) == order[dkx.r(e)] ? 1.0 : 0.0);
  __syncthreads();
  if (rotated) {  // FP32 rotations: make them orthogonal in FP64, then B = Q2^T H1 Q2
    lowdin_step(Q2, W1, W2, kx);
    lowdin_step(Q2, W1, W2, kx);
    sym_congruence(S, Q2, H1, W1, kx);  // into S: the factor is no longer needed
  } else {  // H1 was already diagonal to FP32 accuracy: Q2 is a permutation, B a reordering of H1
    for (int e = tid; e < kx * kx; e += kSmallThreads) S[dkx.q(e)][dkx.r(e)] = H1[order[dkx.q(e)]][order[dkx.r(e)]];
    __syncthreads();
  }
  // first-order decoupling of the wanted block: G = I + A (into W2), then one Lowdin step
  for (int e = tid; e < kx * kx; e += kSmallThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    double g = (a == b) ? 1.0 : 0.0;
    if (a < r && b >= r) {
      g = S[a][b] * rcp64(S[b][b] - S[a][a]);
    } else if (a >= r && b < r) {
      g = -S[b][a] * rcp64(S[a][a] - S[b][b]);
    }
    if (a != b && fabs(g) > 1e-9) atomicOr(&coupled, 1);
    W2[a][b] = g;
  }
  __syncthreads();
  for (int e = tid; e < kx * kx; e += kSmallThreads) H1[dkx.q(e)][dkx.r(e)] = W2[dkx.q(e)][dkx.r(e)];  // G in H1
  __syncthreads();
  // I + A is orthogonal up to ||A||^2: below 1e-18 it needs no Lowdin step
  if (coupled) lowdin_step(H1, W1, W2, kx);
  if (rotated) {
    small_prod(W1, Q2, false, H1, kx);  // W1 = Q2 G
  } else {
    for (int e = tid; e < kx * kx; e += kSmallThreads) W1[dkx.q(e)][dkx.r(e)] = H1[dkx.q(e)][dkx.r(e)];
    __syncthreads();
    for (int e = tid; e < kx * kx; e += kSmallThreads) {  // W1 = P G (P the permutation Q2): rows by order
      const int a = dkx.q(e), b = dkx.r(e);
      W2[order[a]][b] = W1[a][b];
    }
    __syncthreads();
    for (int e = tid; e < kx * kx; e += kSmallThreads) W1[dkx.q(e)][dkx.r(e)] = W2[dkx.q(e)][dkx.r(e)];
  }
  __syncthreads();
  small_prod(Q2, Q1, false, W1, kx);  // Q = Q1 Q2 G (into Q2)
  __syncthreads();
  sym_congruence(W2, Q2, H, W1, kx);  // H' = Q^T H Q
  double* out = d.small;
  for (int e = tid; e < kx * kx; e += kSmallThreads) {
    out[e] = Q2[dkx.q(e)][dkx.r(e)];
    out[kx * kx + e] = W2[dkx.q(e)][dkx.r(e)];
  }
  for (int c = tid; c < kx; c += kSmallThreads) out[2 * kx * kx + c] = W2[c][c];
}

// X <- X Q (FULL: also MX <- MX Q and R = MX - X H').  A CTA takes 8 rows;
// thread (row, column) computes one entry of each product from rows staged in
// shared memory.
constexpr int kRotRows = 8;
constexpr int kResSlot = 7;  // R slot of the per-tile residual sums of squares (slots 1..kPSplit: preconditioner parts)
template <bool FULL>
__global__ void __launch_bounds__(256) k_rotate(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  __shared__ double q[2 * kMaxL * kMaxL];
  __shared__ double xs[kRotRows][kMaxL], ms[kRotRows][kMaxL], nxs[kRotRows][kMaxL];
  __shared__ double rsq[FULL ? kRotRows : 1][kMaxL];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  const int i0 = (int)(blockIdx.x - off[p]) * kRotRows;
  for (int e = threadIdx.x; e < (FULL ? 2 : 1) * kx * kx; e += blockDim.x) q[e] = d.small[e];
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = dkx.q(e), c = dkx.r(e);
    const int i = i0 + r;
    xs[r][c] = i < d.n ? d.X[i * kx + c] : 0.0;
    if (FULL) ms[r][c] = i < d.n ? d.MX[i * kx + c] : 0.0;
  }
  __syncthreads();
  const double* H = q + kx * kx;
  double nmx[kMaxL * kRotRows / 256 + 1];
  int cnt = 0;
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = dkx.q(e), c = dkx.r(e);
    double a = 0.0, b = 0.0;
    for (int t = 0; t < kx; ++t) {
      a = fma(xs[r][t], q[t * kx + c], a);
      if (FULL) b = fma(ms[r][t], q[t * kx + c], b);
    }
    nxs[r][c] = a;
    nmx[cnt++] = b;
  }
  __syncthreads();
  cnt = 0;
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = dkx.q(e), c = dkx.r(e);
    const int i = i0 + r;
    const double b = nmx[cnt++];
    double s = 0.0;
    if (i < d.n) {
      d.X[i * kx + c] = nxs[r][c];
      if (FULL) {
        s = b;
        for (int t = 0; t < kx; ++t) s = fma(-nxs[r][t], H[t * kx + c], s);
        d.MX[i * kx + c] = b;
        d.R[i * kx + c] = s;
      }
    }
    if (FULL) rsq[r][c] = s * s;
  }
  if (FULL) {  // this tile's sum of squares per column, for the residual norms (fixed order later)
    __syncthreads();
    if (threadIdx.x < kx) {
      double t = 0.0;
      for (int r = 0; r < kRotRows; ++r) t += rsq[r][threadIdx.x];
      d.R[(int64_t)kResSlot * d.n * kx + (blockIdx.x - off[p]) * kx + threadIdx.x] = t;
    }
  }
}

// Product with the preconditioner A^-1 = (M + tau I)^-1 at precision T.  SRC 0:
// of the residual R (block iteration); SRC 1: of X itself (subspace iteration).
// Split over the inner dimension: CTA (row tile of 16, part s) writes its
// partial product to R slot 1 + s; k_precond_apply sums the parts in a fixed order.
constexpr int kPRows = 16;
template <typename T, int SRC>
__global__ void __launch_bounds__(256) k_precond(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  __shared__ T ts[kPRows][65];
  __shared__ T rs[64][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int n = (int)d.n, np = npad_of(d);
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  const double* src = SRC == 0 ? d.R : d.X;
  const int local = (int)(blockIdx.x - off[p]);
  const int ntile = (n + kPRows - 1) / kPRows;
  const int split = local / ntile;
  const int i0 = (local % ntile) * kPRows;
  const int j_begin = split * n / kPSplit, j_end = (split + 1) * n / kPSplit;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  T acc[2] = {(T)0, (T)0};
  for (int j0 = j_begin; j0 < j_end; j0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < kPRows * 64; e += 256) {
      const int r = e / 64, c = e % 64;
      const int i = i0 + r, j = j0 + c;
      ts[r][c] = (i < n && j < j_end) ? F1of<T>(d)[i * np + j] : (T)0;
    }
    for (int e = threadIdx.x; e < 64 * kx; e += 256) {
      const int r = dkx.q(e), c = dkx.r(e);
      const int j = j0 + r;
      rs[r][c] = (j < j_end) ? (T)src[j * kx + c] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int u = 0; u < 64; ++u) {
      const T tv = ts[tr][u];
      acc[0] = fma(tv, rs[u][tc], acc[0]);
      acc[1] = fma(tv, rs[u][tc + 16 < kx ? tc + 16 : tc], acc[1]);
    }
  }
  const int i = i0 + tr;
  double* part = d.R + (1 + split) * n * kx;
  if (i < n) {
    if (tc < kx) part[i * kx + tc] = (double)acc[0];
    if (tc + 16 < kx) part[i * kx + tc + 16] = (double)acc[1];
  }
}

// MODE 0: X <- X - sum of the parts (block iteration); MODE 1: X <- sum of the parts.
template <int MODE>
__global__ void __launch_bounds__(256) k_precond_apply(const ProbDesc* __restrict__ descs,
                                                      const int64_t* __restrict__ off, int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int e = (int)(g - off[p]);
  const int nk = (int)d.n * d.kx;
  double s = 0.0;
  for (int q = 0; q < kPSplit; ++q) s += d.R[(1 + q) * nk + e];
  d.X[e] = MODE == 0 ? d.X[e] - s : s;
}

// Largest residual column norm ||R_j|| over the r wanted columns, from the
// per-tile sums of squares of k_rotate (summed in a fixed order).  256 threads:
// 8 groups split the tiles, lane = column.
__device__ inline double wanted_residual_norm(const ProbDesc& d) {
  __shared__ double red[8][32];
  const int kx = d.kx, r = d.r;
  const int ntile = (int)((d.n + kRotRows - 1) / kRotRows);
  const double* pr = d.R + (int64_t)kResSlot * d.n * kx;
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  double s = 0.0;
  if (c < r)
    for (int t = g; t < ntile; t += 8) s += pr[t * kx + c];
  red[g][c] = s;
  __syncthreads();
  double mx = 0.0;
  if (threadIdx.x < 32) {
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += red[k][c];
    mx = c < r ? sqrt64(tot) : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  return mx;  // valid in thread 0
}

// After a Rayleigh-Ritz step: the largest wanted residual norm against the gap
// theta_{r+1} - theta_r; sets the flag that skips the remaining iterations.
__global__ void __launch_bounds__(256) k_conv_check(const ProbDesc* __restrict__ descs, int nprob) {
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int kx = d.kx, r = d.r;
  const double mx = wanted_residual_norm(d);
  if (threadIdx.x == 0) {
    const double* th = d.small + 2 * kx * kx;
    const double gap = r < kx ? th[r] - th[r - 1] : 0.0;
    const double prev = d.stats[kPrevRes];
    // converged: below the target, or no longer falling (at the FP64 rounding
    // floor of M X - X Theta) while already below kStallTol * gap
    const bool stalled = prev > 0.0 && mx > 0.5 * prev && mx <= kStallTol * gap;
    if (gap > 0.0 && (mx <= kConvTol * gap || stalled)) d.stats[kConvFlag] = 1.0;
    d.stats[kPrevRes] = mx;
    d.stats[kIterCount] += 1.0;
  }
}

// V = first r columns of X (n x r column-major, ldv); Ritz values; residual norm.
__global__ void __launch_bounds__(256) k_eig_finish(const ProbDesc* __restrict__ descs, int nprob) {
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx, r = d.r;
  for (int c = 0; c < r; ++c)
    for (int64_t i = threadIdx.x; i < d.n; i += 256) d.V[(int64_t)c * d.ldv + i] = d.X[i * kx + c];
  const double mx = wanted_residual_norm(d);
  if (threadIdx.x < kx && threadIdx.x < 32) d.stats[threadIdx.x] = d.small[2 * kx * kx + threadIdx.x];
  if (threadIdx.x == 0) d.stats[34] = mx;
}

// ------------------------------------------------------------------ launchers
#define RSM_LAUNCH_SMEM(kernel, blocks, threads, smem, ...)            \
  do {                                                                \
    if ((blocks) > 0) {                                               \
      kernel<<<(unsigned)(blocks), threads, smem, s>>>(__VA_ARGS__);  \
      ++g_kernel_launches;                                            \
      cudaError_t e_ = cudaGetLastError();                            \
      if (e_ != cudaSuccess) return e_;                               \
    }                                                                 \
  } while (0)
#define RSM_LAUNCH(kernel, blocks, threads, ...) RSM_LAUNCH_SMEM(kernel, blocks, threads, 0, __VA_ARGS__)

template <typename T>
static cudaError_t launch_eig_t(const EigPlan& P, double shift_rel, int iters, cudaStream_t s) {
  const int xtx_smem = (int)(2 * kChunk * kMaxL * sizeof(double));
  cudaError_t ea = cudaFuncSetAttribute(k_xtx<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, xtx_smem);
  if (ea == cudaSuccess) ea = cudaFuncSetAttribute(k_xtx<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, xtx_smem);
  if (ea == cudaSuccess) ea = cudaFuncSetAttribute(k_rr64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRRSmem);
  if (ea != cudaSuccess) return ea;
  const ProbDesc* D = P.descs;
  const int np = P.nprob;
  auto dev = [&](size_t pos) { return P.dT + pos; };
  auto total = [&](size_t pos) { return P.hT[pos + np]; };
  // Phase A: subspace iteration X <- orth(A^-1 X) with the factor alone (no
  // product with M), until span(X) holds the wanted eigenvectors to about the
  // factor's precision.  The FP64 factor is an almost exact shift-invert whose
  // steps amplify the wanted directions by up to ~1/tau: two steps, each
  // orthonormalised twice (shifted CholeskyQR2); three single-pass steps with
  // the FP32 factor.
  const int a_iters = sizeof(T) == 8 ? 2 : 3, a_passes = sizeof(T) == 8 ? 2 : 1;
  auto* precond_x = k_precond<T, 1>;  // A^-1 X
  auto* precond_r = k_precond<T, 0>;  // A^-1 R
  RSM_LAUNCH(k_eig_prep<T>, (total(P.pad2) + 255) / 256, 256, D, dev(P.pad2), np, shift_rel, a_iters);
  // Blocked Cholesky on the stream; the inverse factor X = L^-1 on the second
  // stream, step k of it as soon as block column k of L is final (after the
  // panel of step k), so the two sequential chains overlap.
  cudaError_t ee;
  if ((ee = cudaEventRecord(P.fork, s)) != cudaSuccess || (ee = cudaStreamWaitEvent(P.aux, P.fork, 0)) != cudaSuccess)
    return ee;
  {
    cudaStream_t s = P.aux;
    RSM_LAUNCH(k_linv_init<T>, total(P.tri), 256, D, dev(P.tri), np);
  }
  for (int k = 0; k < P.max_nblk; ++k) {
    const size_t o1 = P.step + (size_t)k * 3 * (np + 1), o3 = o1 + 2 * (np + 1);
    RSM_LAUNCH(k_panel<T>, total(o1), 256, D, dev(o1), np, k);  // diagonal block + block column k
    if ((ee = cudaEventRecord(P.fork, s)) != cudaSuccess || (ee = cudaStreamWaitEvent(P.aux, P.fork, 0)) != cudaSuccess)
      return ee;
    {
      cudaStream_t s = P.aux;
      const size_t l1 = P.linv + (size_t)k * 2 * (np + 1), l2 = l1 + (np + 1);
      RSM_LAUNCH(k_linv_scale<T>, total(l1), 256, D, dev(l1), np, k);
      RSM_LAUNCH(k_linv_update<T>, total(l2), 256, D, dev(l2), np, k);
    }
    RSM_LAUNCH(k_trail<T>, total(o3), 256, D, dev(o3), np, k);
  }
  if ((ee = cudaEventRecord(P.join, P.aux)) != cudaSuccess || (ee = cudaStreamWaitEvent(s, P.join, 0)) != cudaSuccess)
    return ee;
  RSM_LAUNCH(k_ainv<T>, total(P.tri), 256, D, dev(P.tri), np);
  RSM_LAUNCH(k_init_X, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
  auto orthonormalise = [&]() -> cudaError_t {
    RSM_LAUNCH_SMEM(k_xtx<false>, total(P.chunk), 256, xtx_smem, D, dev(P.chunk), np, P.part, dev(P.part_off));
    RSM_LAUNCH(k_orth<T>, np, kSmallThreads, D, np, P.part, dev(P.part_off));
    RSM_LAUNCH(k_rotate<false>, total(P.rot), 256, D, dev(P.rot), np);
    return cudaSuccess;
  };
  cudaError_t e;
  for (int it = 0; it < a_iters; ++it) {
    RSM_LAUNCH(precond_x, total(P.row_tile), 256, D, dev(P.row_tile), np);
    RSM_LAUNCH(k_precond_apply<1>, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    for (int pass = 0; pass < a_passes; ++pass)
      if ((e = orthonormalise()) != cudaSuccess) return e;
  }
  // Phase B: preconditioned block iteration X <- X - A^-1 (M X - X Theta) with
  // FP64 products with M and an FP64 Rayleigh-Ritz step each time; every step
  // ends with a convergence check, and a converged problem skips everything
  // after it.  With the FP64 factor a step can again collapse the block, so X is
  // re-orthonormalised before each product.  The last step never preconditions.
  for (int it = 0; it <= iters; ++it) {
    if (sizeof(T) == 8 && it > 0)
      if ((e = orthonormalise()) != cudaSuccess) return e;
    if (P.kx_max <= 16)
      RSM_LAUNCH(k_gemm_MX<16>, total(P.mx), kMxRows, D, dev(P.mx), np);
    else
      RSM_LAUNCH(k_gemm_MX<32>, total(P.mx), kMxRows, D, dev(P.mx), np);
    RSM_LAUNCH(k_split_sum, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    RSM_LAUNCH_SMEM(k_xtx<true>, total(P.chunk), 256, xtx_smem, D, dev(P.chunk), np, P.part, dev(P.part_off));
    RSM_LAUNCH_SMEM(k_rr64, np, kSmallThreads, kRRSmem, D, np, P.part, dev(P.part_off));
    RSM_LAUNCH(k_rotate<true>, total(P.rot), 256, D, dev(P.rot), np);
    RSM_LAUNCH(k_conv_check, np, 256, D, np);
    if (it < iters) {
      RSM_LAUNCH(precond_r, total(P.row_tile), 256, D, dev(P.row_tile), np);
      RSM_LAUNCH(k_precond_apply<0>, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    }
  }
  RSM_LAUNCH(k_eig_finish, np, 256, D, np);
  return cudaSuccess;
}

cudaError_t launch_eig(const EigPlan& P, bool fp64_factor, double shift_rel, int iters, cudaStream_t s) {
  return fp64_factor ? launch_eig_t<double>(P, shift_rel, iters, s) : launch_eig_t<float>(P, shift_rel, iters, s);
}

}  // namespace rsm
