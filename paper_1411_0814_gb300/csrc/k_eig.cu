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
// Factor the diagonal block in shared memory and invert the factor.
template <typename T>
__global__ void __launch_bounds__(256) k_potrf(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                              int nprob, int k) {
  __shared__ T a[BS][BS + 1];
  __shared__ T inv[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  T* A = F1of<T>(d) + (int64_t)k * BS * np + (int64_t)k * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) a[e / BS][e % BS] = A[(e / BS) * np + (e % BS)];
  __syncthreads();
  for (int j = 0; j < BS; ++j) {
    if (threadIdx.x == 0) {
      T dj = a[j][j];
      if (!(dj > (T)0)) {  // not positive definite at this precision: flag and continue with a tiny pivot
        atomicAdd(&d.counters[3], 1ull);
        dj = (T)1e-30;
      }
      a[j][j] = sqrt(dj);
    }
    __syncthreads();
    const T djj = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < BS; i += 256) a[i][j] /= djj;
    __syncthreads();
    for (int e = threadIdx.x; e < BS * BS; e += 256) {
      const int i = e / BS, c = e % BS;
      if (c > j && c <= i) a[i][c] -= a[i][j] * a[c][j];
    }
    __syncthreads();
  }
  // inverse of the lower-triangular factor: one column per thread, forward substitution
  if (threadIdx.x < BS) {
    const int c = threadIdx.x;
    for (int i = 0; i < BS; ++i) {
      T s = (i == c) ? (T)1 : (T)0;
      for (int t = c; t < i; ++t) s -= a[i][t] * inv[t][c];
      inv[i][c] = (i < c) ? (T)0 : s / a[i][i];
    }
  }
  __syncthreads();
  T* D = Dinvof<T>(d) + (int64_t)k * BS * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) {
    const int i = e / BS, c = e % BS;
    A[i * np + c] = (c <= i) ? a[i][c] : (T)0;
    D[e] = inv[i][c];
  }
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
template <typename T>
__global__ void __launch_bounds__(256) k_linv_diag(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob) {
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int i = (int)(blockIdx.x - off[p]);
  const T* D = Dinvof<T>(d) + (int64_t)i * BS * BS;
  T* out = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)i * BS;
  for (int e = threadIdx.x; e < BS * BS; e += 256) out[(e / BS) * np + (e % BS)] = D[e];
}

// Block row i of L^-1: Linv_ij = -inv(L_ii) * sum_{t=j}^{i-1} L_it Linv_tj, for j < i.
template <typename T>
__global__ void __launch_bounds__(256) k_linv_step(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob, int i) {
  __shared__ T x[BS][BS + 1], y[BS][BS + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t np = npad_of(d);
  const int j = (int)(blockIdx.x - off[p]);
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int t = j; t < i; ++t) {
    const T* Lit = F1of<T>(d) + (int64_t)i * BS * np + (int64_t)t * BS;
    const T* Ltj = F2of<T>(d) + (int64_t)t * BS * np + (int64_t)j * BS;
    __syncthreads();
    for (int e = threadIdx.x; e < BS * BS; e += 256) {
      x[e / BS][e % BS] = Lit[(e / BS) * np + (e % BS)];
      y[e / BS][e % BS] = Ltj[(e / BS) * np + (e % BS)];
    }
    __syncthreads();
    for (int u = 0; u < BS; ++u) {
      const T yv = y[u][tx];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][u], yv, acc[s]);
    }
  }
  __syncthreads();
  const T* D = Dinvof<T>(d) + (int64_t)i * BS * BS;
  for (int s = 0; s < 4; ++s) x[ty + 8 * s][tx] = acc[s];
  for (int e = threadIdx.x; e < BS * BS; e += 256) y[e / BS][e % BS] = D[e];
  __syncthreads();
  T* out = F2of<T>(d) + (int64_t)i * BS * np + (int64_t)j * BS;
  for (int s = 0; s < 4; ++s) {
    const int r = ty + 8 * s;
    T v = (T)0;
    for (int u = 0; u <= r; ++u) v = fma(y[r][u], x[u][tx], v);
    out[(int64_t)r * np + tx] = -v;
  }
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

constexpr int kSplit = 4;    // split of the inner dimension of the FP64 product
constexpr int kRowTile = 32;  // rows per CTA of the n x kx products

// out = M X (FP64), split over the inner dimension: part s covers j in [s n / kSplit, (s+1) n / kSplit).
// Partial results go to d.R (kSplit x n x kx) and are summed in fixed order by k_split_sum.
__global__ void __launch_bounds__(256) k_gemm_MX(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  __shared__ double ms[kRowTile][33];
  __shared__ double xs[32][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
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
  const int64_t e = g - off[p];
  const int64_t nk = d.n * d.kx;
  double s = d.R[e];
  for (int q = 1; q < kSplit; ++q) s += d.R[q * nk + e];
  d.MX[e] = s;
}

// Partial Gram sums over chunks of 64 rows: part[chunk] = [X^T X | X^T MX] (2 kx^2 values).
constexpr int kChunk = 64;
__global__ void __launch_bounds__(256) k_xtx(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                            int nprob, double* __restrict__ part_base, const int64_t* __restrict__ part_off) {
  __shared__ double xs[kChunk][kMaxL + 1], ys[kChunk][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t chunk = blockIdx.x - off[p];
  const int kx = d.kx;
  const int64_t i0 = chunk * kChunk;
  for (int e = threadIdx.x; e < kChunk * kx; e += 256) {
    const int r = e / kx, c = e % kx;
    const int64_t i = i0 + r;
    xs[r][c] = i < d.n ? d.X[i * kx + c] : 0.0;
    ys[r][c] = i < d.n ? d.MX[i * kx + c] : 0.0;
  }
  __syncthreads();
  double* part = part_base + part_off[p] + chunk * 2 * kx * kx;
  for (int e = threadIdx.x; e < 2 * kx * kx; e += 256) {
    const int which = e / (kx * kx), ab = e % (kx * kx), a = ab / kx, b = ab % kx;
    double s = 0.0;
    if (which == 0)
      for (int r = 0; r < kChunk; ++r) s = fma(xs[r][a], xs[r][b], s);
    else
      for (int r = 0; r < kChunk; ++r) s = fma(xs[r][a], ys[r][b], s);
    part[e] = s;
  }
}

// One warp per problem: reduce the partials (fixed order), S = C C^T, H' = C^-1 H C^-T,
// eig(H') by Jacobi, Q = C^-T Q' (columns sorted by ascending Ritz value).
// small layout: [0, kx^2) = Q, [kx^2, kx^2 + kx) = theta.
__global__ void __launch_bounds__(32) k_rayleigh_ritz(const ProbDesc* __restrict__ descs, int nprob,
                                                     const double* __restrict__ part_base,
                                                     const int64_t* __restrict__ part_off) {
  __shared__ double S[kMaxL][kMaxL + 1], H[kMaxL][kMaxL + 1], Vq[kMaxL][kMaxL + 1], T[kMaxL][kMaxL + 1];
  __shared__ JacobiScratch js;
  __shared__ int order[kMaxL];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx, lane = threadIdx.x;
  const int64_t nchunk = (d.n + kChunk - 1) / kChunk;
  const double* part = part_base + part_off[p];
  for (int e = lane; e < kx * kx; e += 32) {
    double s = 0.0, h = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) {
      s += part[c * 2 * kx * kx + e];
      h += part[c * 2 * kx * kx + kx * kx + e];
    }
    S[e / kx][e % kx] = s;
    H[e / kx][e % kx] = h;
  }
  __syncwarp();
  // symmetrise H (X^T M X is symmetric up to rounding)
  for (int e = lane; e < kx * kx; e += 32) {
    const int a = e / kx, b = e % kx;
    if (a < b) {
      const double v = 0.5 * (H[a][b] + H[b][a]);
      H[a][b] = v;
      H[b][a] = v;
    }
  }
  __syncwarp();
  // Cholesky of S + s I (lane 0; kx <= 32).  The tiny shift s = 1e-15 trace(S)
  // keeps the factorisation defined when the block is numerically rank
  // deficient (shifted CholeskyQR); a second pass restores orthonormality.
  if (lane == 0) {
    double trS = 0.0;
    for (int j = 0; j < kx; ++j) trS += S[j][j];
    const double shift = 1e-15 * trS;
    for (int j = 0; j < kx; ++j) S[j][j] += shift;
    for (int j = 0; j < kx; ++j) {
      double v = S[j][j];
      for (int t = 0; t < j; ++t) v -= S[j][t] * S[j][t];
      v = v > 0.0 ? sqrt(v) : 1e-300;
      S[j][j] = v;
      for (int i = j + 1; i < kx; ++i) {
        double w = S[i][j];
        for (int t = 0; t < j; ++t) w -= S[i][t] * S[j][t];
        S[i][j] = w / v;
      }
      for (int i = 0; i < j; ++i) S[i][j] = 0.0;
    }
  }
  __syncwarp();
  // T = C^-1 H  (forward substitution, one column per lane)
  for (int c = lane; c < kx; c += 32)
    for (int i = 0; i < kx; ++i) {
      double v = H[i][c];
      for (int t = 0; t < i; ++t) v -= S[i][t] * T[t][c];
      T[i][c] = v / S[i][i];
    }
  __syncwarp();
  // H' = T C^-T = (C^-1 T^T)^T : solve C Z = T^T column by column, H'[a][b] = Z[b][a]
  for (int c = lane; c < kx; c += 32)
    for (int i = 0; i < kx; ++i) {
      double v = T[c][i];
      for (int t = 0; t < i; ++t) v -= S[i][t] * H[c][t];
      H[c][i] = v / S[i][i];
    }
  __syncwarp();
  for (int e = lane; e < kx * kx; e += 32) {
    const int a = e / kx, b = e % kx;
    if (a < b) {
      const double v = 0.5 * (H[a][b] + H[b][a]);
      H[a][b] = v;
      H[b][a] = v;
    }
  }
  __syncwarp();
  warp_jacobi(&H[0][0], &Vq[0][0], kx, kMaxL + 1, js);
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
  double* Q = d.small;
  for (int c = lane; c < kx; c += 32) {
    const int oc = order[c];
    for (int i = kx - 1; i >= 0; --i) {
      double v = Vq[i][oc];
      for (int t = i + 1; t < kx; ++t) v -= S[t][i] * T[t][c];
      T[i][c] = v / S[i][i];
    }
  }
  __syncwarp();
  for (int e = lane; e < kx * kx; e += 32) Q[e] = T[e / kx][e % kx];
  for (int c = lane; c < kx; c += 32) Q[kx * kx + c] = H[order[c]][order[c]];
}

// X <- X Q, MX <- MX Q, R = MX - X diag(theta); one thread per row.
__global__ void __launch_bounds__(128) k_rotate(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  __shared__ double q[kMaxL * kMaxL + kMaxL];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int kx = d.kx;
  for (int e = threadIdx.x; e < kx * kx + kx; e += 128) q[e] = d.small[e];
  __syncthreads();
  const int64_t i = (blockIdx.x - off[p]) * 128 + threadIdx.x;
  if (i >= d.n) return;
  double x[kMaxL], mx[kMaxL];
  for (int c = 0; c < kx; ++c) {
    x[c] = d.X[i * kx + c];
    mx[c] = d.MX[i * kx + c];
  }
  for (int c = 0; c < kx; ++c) {
    double a = 0.0, b = 0.0;
    for (int t = 0; t < kx; ++t) {
      a = fma(x[t], q[t * kx + c], a);
      b = fma(mx[t], q[t * kx + c], b);
    }
    d.X[i * kx + c] = a;
    d.MX[i * kx + c] = b;
    d.R[i * kx + c] = b - q[kx * kx + c] * a;
  }
}

// X <- X - A^-1 R with A^-1 at precision T (the preconditioner).
template <typename T>
__global__ void __launch_bounds__(256) k_precond(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  __shared__ T ts[kRowTile][33];
  __shared__ T rs[32][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int64_t n = d.n, np = npad_of(d);
  const int kx = d.kx;
  const int64_t i0 = (blockIdx.x - off[p]) * kRowTile;
  const int tr = threadIdx.x % kRowTile, tc = threadIdx.x / kRowTile;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  for (int64_t j0 = 0; j0 < n; j0 += 32) {
    __syncthreads();
    for (int e = threadIdx.x; e < kRowTile * 32; e += 256) {
      const int r = e / 32, c = e % 32;
      const int64_t i = i0 + r, j = j0 + c;
      ts[r][c] = (i < n && j < n) ? F1of<T>(d)[i * np + j] : (T)0;
    }
    for (int e = threadIdx.x; e < 32 * kx; e += 256) {
      const int r = e / kx, c = e % kx;
      const int64_t j = j0 + r;
      rs[r][c] = (j < n) ? (T)d.R[j * kx + c] : (T)0;
    }
    __syncthreads();
    for (int u = 0; u < 32; ++u) {
      const T tv = ts[tr][u];
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[s] = fma(tv, rs[u][tc + 8 * s < kx ? tc + 8 * s : 0], acc[s]);
    }
  }
  const int64_t i = i0 + tr;
  if (i < n)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int c = tc + 8 * s;
      if (c < kx) d.X[i * kx + c] -= (double)acc[s];
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
  if (threadIdx.x < kx && threadIdx.x < 32) d.stats[threadIdx.x] = d.small[kx * kx + threadIdx.x];
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
  const ProbDesc* D = P.descs;
  const int np = P.nprob;
  auto dev = [&](size_t pos) { return P.dT + pos; };
  auto total = [&](size_t pos) { return P.hT[pos + np]; };
  RSM_LAUNCH(k_eig_prep<T>, (total(P.pad2) + 255) / 256, 256, D, dev(P.pad2), np, shift_rel);
  for (int k = 0; k < P.max_nblk; ++k) {
    const size_t o1 = P.step + (size_t)k * 3 * (np + 1), o2 = o1 + (np + 1), o3 = o2 + (np + 1);
    RSM_LAUNCH(k_potrf<T>, total(o1), 256, D, dev(o1), np, k);
    RSM_LAUNCH(k_panel<T>, total(o2), 256, D, dev(o2), np, k);
    RSM_LAUNCH(k_trail<T>, total(o3), 256, D, dev(o3), np, k);
  }
  RSM_LAUNCH(k_linv_diag<T>, total(P.blk), 256, D, dev(P.blk), np);
  for (int i = 1; i < P.max_nblk; ++i) {
    const size_t o = P.linv + (size_t)i * (np + 1);
    RSM_LAUNCH(k_linv_step<T>, total(o), 256, D, dev(o), np, i);
  }
  RSM_LAUNCH(k_ainv<T>, total(P.tri), 256, D, dev(P.tri), np);
  RSM_LAUNCH(k_init_X, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
  // The FP64 factor is an almost exact shift-invert: a step can amplify the
  // wanted directions by ~1/tau, so each step runs the Rayleigh-Ritz pass twice
  // (the first re-orthonormalises a nearly rank-deficient block).
  const int passes = sizeof(T) == 8 ? 2 : 1;
  for (int it = 0; it <= iters; ++it) {
    RSM_LAUNCH(k_gemm_MX, total(P.mx), 256, D, dev(P.mx), np);
    RSM_LAUNCH(k_split_sum, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
    for (int pass = 0; pass < passes; ++pass) {
      RSM_LAUNCH(k_xtx, total(P.chunk), 256, D, dev(P.chunk), np, P.part, dev(P.part_off));
      RSM_LAUNCH(k_rayleigh_ritz, np, 32, D, np, P.part, dev(P.part_off));
      RSM_LAUNCH(k_rotate, total(P.rot), 128, D, dev(P.rot), np);
    }
    if (it < iters) RSM_LAUNCH(k_precond<T>, total(P.row_tile), 256, D, dev(P.row_tile), np);
  }
  RSM_LAUNCH(k_eig_finish, np, 256, D, np);
  return cudaSuccess;
}

cudaError_t launch_eig(const EigPlan& P, bool fp64_factor, double shift_rel, int iters, cudaStream_t s) {
  return fp64_factor ? launch_eig_t<double>(P, shift_rel, iters, s) : launch_eig_t<float>(P, shift_rel, iters, s);
}

}  // namespace rsm
