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

__device__ __forceinline__ int64_t npad_of(const ProbDesc& d) { return (int64_t)d.nblk * BS; }

template <typename T>
__device__ __forceinline__ T* F1of(const ProbDesc& d) { return static_cast<T*>(d.F1); }
template <typename T>
__device__ __forceinline__ T* F2of(const ProbDesc& d) { return static_cast<T*>(d.F2); }
template <typename T>
__device__ __forceinline__ T* Dinvof(const ProbDesc& d) { return static_cast<T*>(d.Dinv); }

// ------------------------------------------------------------------ A = M + tau I (padded with I)
template <typename T>
__global__ void __launch_bounds__(256) k_eig_prep(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                 int nprob, double shift_rel) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - off[p];
  if (e == 0) d.stats[kConvFlag] = 0.0;
  const int64_t np = npad_of(d);
  const int64_t i = e / np, j = e % np;
  const double mean = (double)d.counters[0] * d.n_minor / (double)d.n;
  const double tau = mean > 0.0 ? shift_rel * mean : 1.0;
  T v;
  if (i < d.n && j < d.n)
    v = (T)(d.M[i * d.n + j] + (i == j ? tau : 0.0));
  else
    v = (i == j) ? (T)1 : (T)0;
  F1of<T>(d)[e] = v;
}

// ------------------------------------------------------------------ Cholesky, step k
// Factor the diagonal block and invert the factor; one thread per entry (32 x 32).
// Step j: one thread takes the square root and reciprocal of the pivot, the
// column-j threads scale, and the trailing threads update.  The inverse is
// formed one column per warp by forward substitution with warp reductions.
template <typename T>
__global__ void __launch_bounds__(1024) k_potrf(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob, int k) {
  __shared__ T a[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int i = threadIdx.x / BS, c = threadIdx.x % BS;  // row, column
  T* A = F1of<T>(d) + (int64_t)k * BS * np + (int64_t)k * BS;
  a[i][c] = A[(int64_t)i * np + c];
  __syncthreads();
  __shared__ T piv;
  for (int j = 0; j < BS; ++j) {
    if (threadIdx.x == 0) {
      T dj = a[j][j];
      if (!(dj > (T)0)) {  // not positive definite at this precision: flag and continue with a tiny pivot
        atomicAdd(&d.counters[3], 1ull);
        dj = (T)1e-30;
      }
      const T s = sqrt(dj);
      a[j][j] = s;
      piv = (T)1 / s;
    }
    __syncthreads();
    if (c == j && i > j) a[i][j] *= piv;
    __syncthreads();
    if (c > j && c <= i) a[i][c] -= a[i][j] * a[c][j];
    __syncthreads();
  }
  // inverse of the lower-triangular factor: warp w computes column w (lane t holds entry t)
  const int col = threadIdx.x / 32, lane = threadIdx.x % 32;
  T mine = (T)0;
  for (int r = 0; r < BS; ++r) {
    T term = (lane >= col && lane < r) ? a[r][lane] * mine : (T)0;
#pragma unroll
    for (int o = 16; o; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    if (lane == r) mine = (r < col) ? (T)0 : (((r == col) ? (T)1 : (T)0) - term) / a[r][r];
  }
  T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
  D[lane * BS + col] = mine;  // entry (lane, col) of inv(L_kk)
  A[(int64_t)i * np + c] = (c <= i) ? a[i][c] : (T)0;
}

// 32 x 32 x 32 product helper: each of 256 threads owns 4 outputs (row ty + 8s, column tx).
// out[r][c] = sum_t X[r][t] * Y(t, c) with Y accessed through the functor.

// Panel: L_ik = A_ik * inv(L_kk)^T for i > k.
template <typename T>
__global__ void __launch_bounds__(256) k_panel(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                              int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int i = k + 1 + (int)(blockIdx.x - off[p]);
  T* Aik = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)k * BS;
  const T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = Aik[(e / BS) * np + (e % BS)];
    y[e / BS][e % BS] = D[e];
  }
  __syncthreads();
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int t = 0; t < BS; ++t) {
    const T yv = y[tx][t];  // (inv L_kk)^T [t][tx]
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][t], yv, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Aik[(int64_t)(ty + 8 * s) * np + tx] = acc[s];
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
  const int64_t np = npad_of(d);
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
  for (int s = 0; s < 4; ++s) Aij[(int64_t)(ty + 8 * s) * np + tx] -= acc[s];
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
  const int64_t np = npad_of(d);
  int i, j;
  tri_index(blockIdx.x - off[p], i, j);
  T* out = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    const int r = e / BS, c = e % BS;
    out[(int64_t)r * np + c] = (i == j && r == c) ? (T)1 : (T)0;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_linv_scale(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                   int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int j = (int)(blockIdx.x - off[p]);  // j <= k
  T* Xkj = F2of<T>(d) + (int64_t)k * BS * np + (int64_t)j * BS;
  const T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = D[e];
    y[e / BS][e % BS] = Xkj[(int64_t)(e / BS) * np + (e % BS)];
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
  for (int s = 0; s < 4; ++s) Xkj[(int64_t)(ty + 8 * s) * np + tx] = acc[s];
}

template <typename T>
__global__ void __launch_bounds__(256) k_linv_update(const ProbDesc* __restrict__ descs,
                                                    const int64_t* __restrict__ off, int nprob, int k) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int64_t local = blockIdx.x - off[p];
  const int i = k + 1 + (int)(local / (k + 1)), j = (int)(local % (k + 1));
  const T* Lik = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)k * BS;
  const T* Xkj = F2of<T>(d) + (int64_t)k * BS * np + (int64_t)j * BS;
  T* Xij = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    x[e / BS][e % BS] = Lik[(int64_t)(e / BS) * np + (e % BS)];
    y[e / BS][e % BS] = Xkj[(int64_t)(e / BS) * np + (e % BS)];
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
  for (int s = 0; s < 4; ++s) Xij[(int64_t)(ty + 8 * s) * np + tx] -= acc[s];
}

// T = A^-1 = L^-T L^-1:  T_ij = sum_{t >= max(i, j)} Linv_ti^T Linv_tj  (into F1, both triangles)
template <typename T>
__global__ void __launch_bounds__(256) k_ainv(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                             int nprob) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
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
    Tij[(int64_t)(ty + 8 * s) * np + tx] = acc[s];
    x[ty + 8 * s][tx] = acc[s];
  }
  __syncthreads();
  if (i != j)
    for (int e = threadIdx.x; e < BS * BS; e += 256) Tji[(int64_t)(e / BS) * np + (e % BS)] = x[e % BS][e / BS];
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

constexpr int kSplit = 8;    // split of the inner dimension of the FP64 product M X
constexpr int kPSplit = 4;   // split of the inner dimension of the preconditioner product
constexpr int kRowTile = 32;  // rows per CTA of the n x kx products

// out = M X (FP64), split over the inner dimension: part s covers j in [s n / kSplit, (s+1) n / kSplit).
// Partial results go to d.R (kSplit x n x kx) and are summed in fixed order by k_split_sum.
__global__ void __launch_bounds__(256) k_gemm_MX(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  __shared__ double ms[kRowTile][33];
  __shared__ double xs[32][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int64_t local = blockIdx.x - off[p];
  const int64_t n = d.n;
  const int kx = d.kx;
  const int64_t ntile = (n + kRowTile - 1) / kRowTile;
  const int split = (int)(local / ntile);
  const int64_t i0 = (local % ntile) * kRowTile;
  const int64_t j_begin = split * n / kSplit, j_end = (split + 1) * n / kSplit;
  const int tr = threadIdx.x % kRowTile, tc = threadIdx.x / kRowTile;  // 8 column groups
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t j0 = j_begin; j0 < j_end; j0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < kRowTile * 32; e += 256) {
      const int r = e / 32, c = e % 32;
      const int64_t i = i0 + r, j = j0 + c;
      ms[r][c] = (i < n && j < j_end) ? d.M[i * n + j] : 0.0;
    }
    for (int e = threadIdx.x; e < 32 * kx; e += 256) {
      const int r = e / kx, c = e % kx;
      const int64_t j = j0 + r;
      xs[r][c] = (j < j_end) ? d.X[j * kx + c] : 0.0;
    }
    __syncthreads();
    for (int u = 0; u < 32; ++u) {
      const double mv = ms[tr][u];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int c = tc + 8 * s;
        if (c < kx) acc[s] = fma(mv, xs[u][c], acc[s]);
      }
    }
  }
  const int64_t i = i0 + tr;
  if (i < n)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int c = tc + 8 * s;
      if (c < kx) d.R[((int64_t)split * n + i) * kx + c] = acc[s];
    }
}

__global__ void __launch_bounds__(256) k_split_sum(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int64_t e = g - off[p];
  const int64_t nk = d.n * d.kx;
  double s = d.R[e];
  for (int q = 1; q < kSplit; ++q) s += d.R[q * nk + e];
  d.MX[e] = s;
}

// Partial Gram sums over chunks of kChunk rows: part[chunk] = [X^T X | X^T MX] (2 kx^2 values).
constexpr int kChunk = 64;
__global__ void __launch_bounds__(256) k_xtx(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                            int nprob, double* __restrict__ part_base, const int64_t* __restrict__ part_off) {
  extern __shared__ double xtx_smem[];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int64_t chunk = blockIdx.x - off[p];
  const int kx = d.kx;
  double* xs = xtx_smem;                  // kChunk x kx
  double* ys = xtx_smem + kChunk * kx;    // kChunk x kx
  const int64_t i0 = chunk * kChunk;
  for (int e = threadIdx.x; e < kChunk * kx; e += 256) {
    const int64_t i = i0 + e / kx;
    xs[e] = i < d.n ? d.X[i0 * kx + e] : 0.0;
    ys[e] = i < d.n ? d.MX[i0 * kx + e] : 0.0;
  }
  __syncthreads();
  double* part = part_base + part_off[p] + chunk * 2 * kx * kx;
  for (int e = threadIdx.x; e < 2 * kx * kx; e += 256) {
    const int which = e / (kx * kx), ab = e % (kx * kx), a = ab / kx, b = ab % kx;
    const double* y = which == 0 ? xs : ys;
    double s0 = 0.0, s1 = 0.0;
    for (int r = 0; r < kChunk; r += 2) {
      s0 = fma(xs[r * kx + a], y[r * kx + b], s0);
      s1 = fma(xs[(r + 1) * kx + a], y[(r + 1) * kx + b], s1);
    }
    part[e] = s0 + s1;
  }
}

// Lane-parallel shifted Cholesky S + s I = C C^T in place (lower triangle),
// s = 1e-15 trace(S): keeps the factor defined when the block is numerically
// rank deficient (shifted CholeskyQR).  kx <= 32, lane i owns row i.
__device__ inline void warp_chol_shifted(double (*S)[kMaxL + 1], int kx) {
  const int lane = threadIdx.x & 31;
  double trS = 0.0;
  for (int j = 0; j < kx; ++j) trS += S[j][j];
  __syncwarp();
  if (lane < kx) S[lane][lane] += 1e-15 * trS;
  __syncwarp();
  for (int j = 0; j < kx; ++j) {
    double v = S[j][j];
    v = v > 0.0 ? sqrt(v) : 1e-300;
    const double rv = 1.0 / v;
    __syncwarp();
    if (lane == j) S[j][j] = v;
    if (lane > j && lane < kx) S[lane][j] *= rv;
    __syncwarp();
    if (lane > j && lane < kx) {
      const double lij = S[lane][j];
      for (int c = j + 1; c <= lane; ++c) S[lane][c] -= lij * S[c][j];
    }
    __syncwarp();
  }
  for (int e = lane; e < kx * kx; e += 32)
    if (e / kx < e % kx) S[e / kx][e % kx] = 0.0;
  __syncwarp();
}

// One warp per problem.  Reduce the partials (fixed order) into S = X^T X and
// H = X^T M X, factor S + s I = C C^T (shifted CholeskyQR), and write
// small = [Q | H' | theta] with X Q orthonormal and H' = Q^T H Q.
// Intermediate steps (FINAL = false) stop there (Q = C^-T): the block
// iteration X <- X - T (M X - X H') only needs the subspace to converge, and
// any basis of it gives the same fixed point.  With the FP32 factor they run
// in FP32, enough for an orthonormalisation that the next step repeats.
// The final step (FINAL = true) also diagonalises H' (FP32 Jacobi + FP64
// polish): Q = C^-T Q', H' = diag(theta), columns by ascending Ritz value.
constexpr int kLs = kMaxL + 1;
constexpr size_t kRRSmem = sizeof(double) * 4 * kMaxL * kLs + sizeof(float) * 4 * kMaxL * kLs;

template <bool FINAL, typename CT>
__global__ void __launch_bounds__(32) k_rayleigh_ritz(const ProbDesc* __restrict__ descs, int nprob,
                                                     const double* __restrict__ part_base,
                                                     const int64_t* __restrict__ part_off) {
  extern __shared__ __align__(16) unsigned char rr_smem[];
  typedef double DRow[kLs];
  typedef float FRow[kLs];
  DRow* S = reinterpret_cast<DRow*>(rr_smem);
  DRow* H = S + kMaxL;
  DRow* Vq = H + kMaxL;
  DRow* T = Vq + kMaxL;
  FRow* Sf = reinterpret_cast<FRow*>(T + kMaxL);
  FRow* Vf = Sf + kMaxL;
  FRow* Sj = Vf + kMaxL;
  FRow* Vj = Sj + kMaxL;
  __shared__ JacobiScratchT<float> jsf;
  __shared__ JacobiScratchT<double> jsd;
  __shared__ int order[kMaxL];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int kx = d.kx, lane = threadIdx.x;
  const int64_t nchunk = (d.n + kChunk - 1) / kChunk;
  const double* part = part_base + part_off[p];
  for (int e = lane; e < kx * kx; e += 32) {
    double s = 0.0, h = 0.0;
#pragma unroll 8
    for (int64_t c = 0; c < nchunk; ++c) {
      s += part[c * 2 * kx * kx + e];
      h += part[c * 2 * kx * kx + kx * kx + e];
    }
    S[e / kx][e % kx] = s;
    H[e / kx][e % kx] = h;
  }
  __syncwarp();
  double* out = d.small;
  if (!FINAL) {
    // (1) shifted Cholesky of S in precision CT (lane i owns row i); CT is the
    // precision of the preconditioner's factor: FP64 when a step may amplify
    // the wanted directions by ~1/tau ~ 1e11, FP32 otherwise
    CT (*Sc)[kLs];
    CT (*Vc)[kLs];
    if constexpr (sizeof(CT) == 8) {
      Sc = S;
      Vc = Vq;
    } else {
      Sc = Sf;
      Vc = Vf;
    }
    CT trS = 0;
    for (int j = 0; j < kx; ++j) trS += (CT)S[j][j];
    if constexpr (sizeof(CT) != 8)
      for (int e = lane; e < kx * kx; e += 32) Sc[e / kx][e % kx] = (CT)S[e / kx][e % kx];
    __syncwarp();
    if (lane < kx) Sc[lane][lane] += (CT)(sizeof(CT) == 8 ? 1e-15 : 1e-6) * trS;
    __syncwarp();
    for (int j = 0; j < kx; ++j) {
      CT v = Sc[j][j];
      v = v > (CT)0 ? sqrt(v) : (CT)1e-30;
      const CT rv = (CT)1 / v;
      __syncwarp();
      if (lane == j) Sc[j][j] = v;
      if (lane > j && lane < kx) Sc[lane][j] *= rv;
      __syncwarp();
      if (lane > j && lane < kx) {
        const CT lij = Sc[lane][j];
        for (int c = j + 1; c <= lane; ++c) Sc[lane][c] -= lij * Sc[c][j];
      }
      __syncwarp();
    }
    // (2) Q1 = C^-T (upper triangular): column c solves C^T q = e_c
    for (int c = lane; c < kx; c += 32)
      for (int i = kx - 1; i >= 0; --i) {
        CT v = (i == c) ? (CT)1 : (CT)0;
        for (int t = i + 1; t < kx; ++t) v -= Sc[t][i] * Vc[t][c];
        Vc[i][c] = (i > c) ? (CT)0 : v / Sc[i][i];
      }
    __syncwarp();
    if constexpr (sizeof(CT) != 8) {
      // FP32 factor: the Ritz rotation of an intermediate step is all FP32.
      // (3) H1 = Q1^T H Q1 (into Sj)
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        float s = 0.f;
        for (int t = 0; t < kx; ++t) s = fmaf((float)H[a][t], Vc[t][b], s);
        T[a][b] = s;
      }
      __syncwarp();
      float fro2 = 0.f;
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        float s = 0.f;
        for (int t = 0; t < kx; ++t) s = fmaf(Vc[t][a], (float)T[t][b], s);
        Sj[a][b] = s;
        fro2 += s * s;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) fro2 += __shfl_xor_sync(0xffffffffu, fro2, o);
      __syncwarp();
      // (4) Ritz rotation Q2 from Jacobi; Q = Q1 Q2, H_out = Q2^T H1 Q2 (the rotated Sj)
      warp_jacobi<float>(&Sj[0][0], &Vj[0][0], kx, kLs, jsf, 4.f * FLT_EPSILON * sqrtf(fro2));
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        float q = 0.f;
        for (int t = 0; t < kx; ++t) q = fmaf(Vc[a][t], Vj[t][b], q);
        out[e] = (double)q;
        out[kx * kx + e] = (double)Sj[a][b];
      }
      return;
    } else {
      // FP64 factor: steps may amplify the wanted directions by ~1e11, keep the
      // rotation in FP64 products of the FP64 basis.
      // (3) H1 = Q1^T H Q1 in FP64 (into S, free now)
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        double s = 0.0;
        for (int t = 0; t < kx; ++t) s = fma(H[a][t], (double)Vc[t][b], s);
        T[a][b] = s;
      }
      __syncwarp();
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        double s = 0.0;
        for (int t = 0; t < kx; ++t) s = fma((double)Vc[t][a], T[t][b], s);
        Sj[a][b] = (float)s;
        S[a][b] = s;
      }
      __syncwarp();
      // (4) Ritz rotation from FP32 Jacobi of H1; Q = Q1 Q2 and H_out = Q2^T H1 Q2 in FP64
      const double fro = warp_frobenius(&S[0][0], kx, kLs);
      warp_jacobi<float>(&Sj[0][0], &Vj[0][0], kx, kLs, jsf, (float)(4.0 * FLT_EPSILON * fro));
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        double q = 0.0, h = 0.0;
        for (int t = 0; t < kx; ++t) {
          q = fma((double)Vc[a][t], (double)Vj[t][b], q);
          h = fma(S[a][t], (double)Vj[t][b], h);
        }
        T[a][b] = q;
        H[a][b] = h;
      }
      __syncwarp();
      for (int e = lane; e < kx * kx; e += 32) {
        const int a = e / kx, b = e % kx;
        double s = 0.0;
        for (int t = 0; t < kx; ++t) s = fma((double)Vj[t][a], H[t][b], s);
        out[e] = T[a][b];
        out[kx * kx + e] = s;
      }
      return;
    }
  }
  warp_chol_shifted(S, kx);
  // T = C^-1 H  (forward substitution, one column per lane)
  for (int c = lane; c < kx; c += 32)
    for (int i = 0; i < kx; ++i) {
      double v = 0.5 * (H[i][c] + H[c][i]);
      for (int t = 0; t < i; ++t) v -= S[i][t] * T[t][c];
      T[i][c] = v / S[i][i];
    }
  __syncwarp();
  // H' = T C^-T: row c of H' solves C z = (row c of T)
  for (int c = lane; c < kx; c += 32)
    for (int i = 0; i < kx; ++i) {
      double v = T[c][i];
      for (int t = 0; t < i; ++t) v -= S[i][t] * Vq[c][t];
      Vq[c][i] = v / S[i][i];
    }
  __syncwarp();
  for (int e = lane; e < kx * kx; e += 32) {
    const int a = e / kx, b = e % kx;
    H[a][b] = 0.5 * (Vq[a][b] + Vq[b][a]);
  }
  __syncwarp();
  warp_eig_mixed(&H[0][0], &Vq[0][0], &Sf[0][0], &Vf[0][0], &T[0][0], kx, kLs, jsf, jsd);
  if (lane == 0) {  // ascending order of the Ritz values
    for (int i = 0; i < kx; ++i) order[i] = i;
    for (int a = 1; a < kx; ++a) {
      const int v = order[a];
      int b = a - 1;
      while (b >= 0 && H[order[b]][order[b]] > H[v][v]) {
        order[b + 1] = order[b];
        --b;
      }
      order[b + 1] = v;
    }
  }
  __syncwarp();
  // Q = C^-T Q'  (back substitution, one column per lane)
  for (int c = lane; c < kx; c += 32) {
    const int oc = order[c];
    for (int i = kx - 1; i >= 0; --i) {
      double v = Vq[i][oc];
      for (int t = i + 1; t < kx; ++t) v -= S[t][i] * T[t][c];
      T[i][c] = v / S[i][i];
    }
  }
  __syncwarp();
  for (int e = lane; e < kx * kx; e += 32) {
    const int a = e / kx, b = e % kx;
    out[e] = T[a][b];
    out[kx * kx + e] = (a == b) ? H[order[a]][order[a]] : 0.0;
  }
  for (int c = lane; c < kx; c += 32) out[2 * kx * kx + c] = H[order[c]][order[c]];
}

// X <- X Q, MX <- MX Q, R = MX - X H'.  A CTA takes 8 rows; thread (row, column)
// computes one entry of each product from rows staged in shared memory.
constexpr int kRotRows = 8;
__global__ void __launch_bounds__(256) k_rotate(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  __shared__ double q[2 * kMaxL * kMaxL];
  __shared__ double xs[kRotRows][kMaxL], ms[kRotRows][kMaxL], nxs[kRotRows][kMaxL];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int kx = d.kx;
  const int64_t i0 = (blockIdx.x - off[p]) * kRotRows;
  for (int e = threadIdx.x; e < 2 * kx * kx; e += blockDim.x) q[e] = d.small[e];
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = e / kx, c = e % kx;
    const int64_t i = i0 + r;
    xs[r][c] = i < d.n ? d.X[i * kx + c] : 0.0;
    ms[r][c] = i < d.n ? d.MX[i * kx + c] : 0.0;
  }
  __syncthreads();
  const double* H = q + kx * kx;
  double nmx[kMaxL * kRotRows / 256 + 1];
  int cnt = 0;
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = e / kx, c = e % kx;
    double a = 0.0, b = 0.0;
    for (int t = 0; t < kx; ++t) {
      a = fma(xs[r][t], q[t * kx + c], a);
      b = fma(ms[r][t], q[t * kx + c], b);
    }
    nxs[r][c] = a;
    nmx[cnt++] = b;
  }
  __syncthreads();
  cnt = 0;
  for (int e = threadIdx.x; e < kRotRows * kx; e += blockDim.x) {
    const int r = e / kx, c = e % kx;
    const int64_t i = i0 + r;
    const double b = nmx[cnt++];
    double s = b;
    for (int t = 0; t < kx; ++t) s = fma(-nxs[r][t], H[t * kx + c], s);
    if (i < d.n) {
      d.X[i * kx + c] = nxs[r][c];
      d.MX[i * kx + c] = b;
      d.R[i * kx + c] = s;
    }
  }
}

// X <- X - A^-1 R with A^-1 at precision T (the preconditioner).  Split over the
// inner dimension: CTA (row tile of 16, part s) writes its partial product to
// R slot 1 + s; k_precond_apply sums the parts in a fixed order.
constexpr int kPRows = 16;
template <typename T>
__global__ void __launch_bounds__(256) k_precond(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  __shared__ T ts[kPRows][65];
  __shared__ T rs[64][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int64_t n = d.n, np = npad_of(d);
  const int kx = d.kx;
  const int64_t local = blockIdx.x - off[p];
  const int64_t ntile = (n + kPRows - 1) / kPRows;
  const int split = (int)(local / ntile);
  const int64_t i0 = (local % ntile) * kPRows;
  const int64_t j_begin = split * n / kPSplit, j_end = (split + 1) * n / kPSplit;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  T acc[2] = {(T)0, (T)0};
  for (int64_t j0 = j_begin; j0 < j_end; j0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < kPRows * 64; e += 256) {
      const int r = e / 64, c = e % 64;
      const int64_t i = i0 + r, j = j0 + c;
      ts[r][c] = (i < n && j < j_end) ? F1of<T>(d)[i * np + j] : (T)0;
    }
    for (int e = threadIdx.x; e < 64 * kx; e += 256) {
      const int r = e / kx, c = e % kx;
      const int64_t j = j0 + r;
      rs[r][c] = (j < j_end) ? (T)d.R[j * kx + c] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int u = 0; u < 64; ++u) {
      const T tv = ts[tr][u];
      acc[0] = fma(tv, rs[u][tc], acc[0]);
      acc[1] = fma(tv, rs[u][tc + 16 < kx ? tc + 16 : tc], acc[1]);
    }
  }
  const int64_t i = i0 + tr;
  double* part = d.R + (int64_t)(1 + split) * n * kx;
  if (i < n) {
    if (tc < kx) part[i * kx + tc] = (double)acc[0];
    if (tc + 16 < kx) part[i * kx + tc + 16] = (double)acc[1];
  }
}

__global__ void __launch_bounds__(256) k_precond_apply(const ProbDesc* __restrict__ descs,
                                                      const int64_t* __restrict__ off, int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int64_t e = g - off[p];
  const int64_t nk = d.n * d.kx;
  double s = 0.0;
  for (int q = 0; q < kPSplit; ++q) s += d.R[(int64_t)(1 + q) * nk + e];
  d.X[e] -= s;
}

// After a polished Rayleigh-Ritz step: largest residual column norm over the r
// wanted Ritz pairs against the gap theta_{r+1} - theta_r; sets the flag that
// skips the remaining iterations of the problem.
__global__ void __launch_bounds__(256) k_conv_check(const ProbDesc* __restrict__ descs, int nprob) {
  __shared__ double red[256];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int kx = d.kx, r = d.r;
  double mx = 0.0;
  for (int c = 0; c < r; ++c) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < d.n; i += 256) {
      const double v = d.R[i * kx + c];
      s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    mx = fmax(mx, sqrt(red[0]));
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double* th = d.small + 2 * kx * kx;
    const double gap = r < kx ? th[r] - th[r - 1] : 0.0;
    if (gap > 0.0 && mx <= kConvTol * gap) d.stats[kConvFlag] = 1.0;
  }
}

// V = first r columns of X (n x r column-major, ldv); eigenvalue estimates; residual norm.
__global__ void __launch_bounds__(256) k_eig_finish(const ProbDesc* __restrict__ descs, int nprob) {
  __shared__ double red[256];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx, r = d.r;
  double mx = 0.0;
  for (int64_t e = threadIdx.x; e < d.n * r; e += 256) {
    const int64_t i = e / r;
    const int c = (int)(e % r);
    d.V[(int64_t)c * d.ldv + i] = d.X[i * kx + c];
  }
  // largest residual column norm among the r wanted Ritz pairs
  for (int c = 0; c < r; ++c) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < d.n; i += 256) {
      const double v = d.R[i * kx + c];
      s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) mx = fmax(mx, sqrt(red[0]));
    __syncthreads();
  }
  if (threadIdx.x < kx && threadIdx.x < 32) d.stats[threadIdx.x] = d.small[2 * kx * kx + threadIdx.x];
  if (threadIdx.x == 0) d.stats[34] = mx;
}

// ------------------------------------------------------------------ launchers
#define RSM_LAUNCH(kernel, blocks, threads, ...)                   \
  do {                                                             \
    if ((blocks) > 0) {                                            \
      kernel<<<(unsigned)(blocks), threads, 0, s>>>(__VA_ARGS__);  \
      ++g_kernel_launches;                                         \
      cudaError_t e_ = cudaGetLastError();                         \
      if (e_ != cudaSuccess) return e_;                            \
    }                                                              \
  } while (0)

template <typename T>
static cudaError_t launch_eig_t(const EigPlan& P, double shift_rel, int iters, cudaStream_t s) {
  cudaError_t ea = cudaFuncSetAttribute(k_xtx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(2 * kChunk * kMaxL * sizeof(double)));
  if (ea == cudaSuccess)
    ea = cudaFuncSetAttribute(k_rayleigh_ritz<true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRRSmem);
  if (ea == cudaSuccess)
    ea = cudaFuncSetAttribute(k_rayleigh_ritz<false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRRSmem);
  if (ea != cudaSuccess) return ea;
  const ProbDesc* D = P.descs;
  const int np = P.nprob;
  auto dev = [&](size_t pos) { return P.dT + pos; };
  auto total = [&](size_t pos) { return P.hT[pos + np]; };
  RSM_LAUNCH(k_eig_prep<T>, (total(P.pad2) + 255) / 256, 256, D, dev(P.pad2), np, shift_rel);
  for (int k = 0; k < P.max_nblk; ++k) {
    const size_t o1 = P.step + (size_t)k * 3 * (np + 1), o2 = o1 + (np + 1), o3 = o2 + (np + 1);
    RSM_LAUNCH(k_potrf<T>, total(o1), 1024, D, dev(o1), np, k);
    RSM_LAUNCH(k_panel<T>, total(o2), 256, D, dev(o2), np, k);
    RSM_LAUNCH(k_trail<T>, total(o3), 256, D, dev(o3), np, k);
  }
  RSM_LAUNCH(k_linv_init<T>, total(P.tri), 256, D, dev(P.tri), np);
  for (int k = 0; k < P.max_nblk; ++k) {
    const size_t o1 = P.linv + (size_t)k * 2 * (np + 1), o2 = o1 + (np + 1);
    RSM_LAUNCH(k_linv_scale<T>, total(o1), 256, D, dev(o1), np, k);
    RSM_LAUNCH(k_linv_update<T>, total(o2), 256, D, dev(o2), np, k);
  }
  RSM_LAUNCH(k_ainv<T>, total(P.tri), 256, D, dev(P.tri), np);
  RSM_LAUNCH(k_init_X, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
  // The FP64 factor is an almost exact shift-invert: a step can amplify the
  // wanted directions by ~1/tau, so each step runs the Rayleigh-Ritz pass twice
  // (the first re-orthonormalises a nearly rank-deficient block).  The closing
  // pass diagonalises in FP64 (polished); the steps before it in FP32.
  const int passes = sizeof(T) == 8 ? 2 : 1;
  // Adaptive: steps before min_iters diagonalise in FP32; from min_iters on every
  // step ends with the polished FP64 Rayleigh-Ritz and a convergence check, and a
  // converged problem skips everything after it.  The last step never preconditions.
  const int min_iters = sizeof(T) == 8 ? 2 : 5;
  for (int it = 0; it <= iters; ++it) {
    const bool final_rr = it >= min_iters || it == iters;
    RSM_LAUNCH(k_gemm_MX, total(P.mx), 256, D, dev(P.mx), np);
    RSM_LAUNCH(k_split_sum, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    for (int pass = 0; pass < passes; ++pass) {
      if (total(P.chunk) > 0) {
        k_xtx<<<(unsigned)total(P.chunk), 256, 2 * kChunk * kMaxL * sizeof(double), s>>>(D, dev(P.chunk), np, P.part,
                                                                                        dev(P.part_off));
        ++g_kernel_launches;
        if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
      }
      if (final_rr && pass == passes - 1) {
        k_rayleigh_ritz<true, T><<<np, 32, kRRSmem, s>>>(D, np, P.part, dev(P.part_off));
      } else {
        k_rayleigh_ritz<false, T><<<np, 32, kRRSmem, s>>>(D, np, P.part, dev(P.part_off));
      }
      ++g_kernel_launches;
      if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
      RSM_LAUNCH(k_rotate, total(P.rot), 256, D, dev(P.rot), np);
    }
    if (final_rr) RSM_LAUNCH(k_conv_check, np, 256, D, np);
    if (it < iters) {
      RSM_LAUNCH(k_precond<T>, total(P.row_tile), 256, D, dev(P.row_tile), np);
      RSM_LAUNCH(k_precond_apply, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    }
  }
  RSM_LAUNCH(k_eig_finish, np, 256, D, np);
  return cudaSuccess;
}

cudaError_t launch_eig(const EigPlan& P, bool fp64_factor, double shift_rel, int iters, cudaStream_t s) {
  return fp64_factor ? launch_eig_t<double>(P, shift_rel, iters, s) : launch_eig_t<float>(P, shift_rel, iters, s);
}

}  // namespace rsm
