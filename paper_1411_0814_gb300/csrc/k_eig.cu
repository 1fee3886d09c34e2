// Stage a7: V-hat = eigenvectors of M for its r smallest eigenvalues (eq.
// solve.barV_L2_norm: only M = Xi Xi^T is stored, and V-hat takes the vectors of
// the r smallest singular values of Xi).
//
// Method (preconditioned inverse iteration with Rayleigh-Ritz, PINVIT):
//   * A = M + tau I with a small shift tau = c * trace(M) / n is factored
//     A = L L^T (blocked right-looking Cholesky, 32 x 32 blocks), then
//     T = A^-1 = L^-T L^-1 is formed, all in one dataflow launch (k_factor).
//     T is only a preconditioner.  The fast form factors in FP32 with
//     c = 3e-4 (enough when lambda_{r+1} >> tau); the robust form factors in
//     FP64 with c = 1e-11, which makes the step an exact shift-invert
//     iteration and resolves clustered small eigenvalues.
//   * Phase A: X <- orth(T X) a few times (subspace iteration, no product
//     with M).
//   * Phase B: a block X of kx >= r + 1 vectors is iterated:
//       Rayleigh-Ritz on span(X):  S = X^T X, H = X^T M X, S = C C^T,
//         eig(C^-1 H C^-T) = Q' diag(theta), X <- X C^-T Q'  (orthonormal Ritz basis)
//       residual R = M X - X diag(theta)
//       X <- X - T R
//     Components of X along an eigenvector with eigenvalue lambda shrink by
//     about (tau + theta) / (lambda + tau) per step, so the r smallest Ritz
//     pairs converge quickly when lambda_{r+1} >> tau.  M X, the reductions and
//     the Rayleigh-Ritz step run in FP32-pair arithmetic (about 2^-44
//     relative; FP64 reductions with the FP64 factor).  The iteration stops
//     at a residual target, or after the correction of a step that is
//     predicted to reach it.
//   * FP64 refinement: a final pass with M X in IEEE FP64 (k_gemm_MX64), a
//     Rayleigh-Ritz step whose FP64 residual M v - theta v is what the host
//     checks against the eigen-gap (with the FP64 factor a residual and
//     correction pass first).
// Every kernel is batched over the problems of the launch.
#include <atomic>
#include <utility>

#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"
#include "small_df.cuh"

namespace rsm {

constexpr int BS = 32;  // block size of the FP32 factorisation
// stats[40]: 0 while the block iteration of this problem runs; 1 once it has
// converged (every later kernel of the iteration returns at once); 2 when it
// stops after one more correction X <- X - A^-1 R (the preconditioner kernels of
// that step still run; the next convergence check sets 1)
constexpr int kConvFlag = 40;
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
// T = A^-1 (npad x npad) follows the factor in the F1 region.
template <typename T>
__device__ __forceinline__ T* Tof(const ProbDesc& d) {
  return static_cast<T*>(d.F1) + d.nblk * BS * d.nblk * BS;
}

// ------------------------------------------------------------------ A = M + tau I (padded with I)
// Four consecutive entries of one padded row per thread; npad is a multiple of
// 32, so the 1024 entries of a CTA belong to one problem.  Also writes M as
// FP32 (hi, lo) pairs for the products M X and L^-1 = I on the lower blocks.
template <typename T>
__global__ void __launch_bounds__(256) k_eig_prep(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                 int nprob, double shift_rel, int iter0) {
  pdl_enter();
  const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (g0 >= off[nprob]) return;
  const int p = find_problem(off, nprob, g0);
  const ProbDesc& d = descs[p];
  const uint32_t e0 = (uint32_t)(g0 - off[p]);
  if (e0 == 0) {
    d.stats[kConvFlag] = 0.0;
    d.stats[kPrevRes] = 0.0;
    d.stats[kIterCount] = (double)iter0;  // the unchecked leading steps
  }
  const uint32_t np = (uint32_t)npad_of(d), n = (uint32_t)d.n;
  const uint32_t i = e0 / np, j0 = e0 - i * np;
  // tau = shift_rel * trace(M) / n, trace(M) = accepted trials * n_minor, or computed from a
  // caller-supplied M (a shift: FP32 suffices for the mean)
  const float meanf = d.m_given || d.l1 ? (float)(d.stats[kStatTrace] / (double)n)
                      : d.variant == 2 ? (float)d.counters[7] / (float)n
                                       : (float)d.counters[0] * (float)d.n_minor / (float)n;
  const double tau = meanf > 0.f ? shift_rel * (double)meanf : 1.0;
  T v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t j = j0 + q;
    if (i < n && j < n) {
      const double mij = d.M[i * n + j];
      v[q] = (T)(i == j ? mij + tau : mij);
      const float hi = __double2float_rn(mij);
      d.Mdf[i * n + j] = make_float2(hi, __double2float_rn(mij - (double)hi));
    } else {
      v[q] = (i == j) ? (T)1 : (T)0;
    }
  }
  T* F1 = F1of<T>(d) + e0;
  T* F2 = F2of<T>(d) + e0;
  const bool lower = j0 / BS <= i / BS;  // the four entries share a 32-column block
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    F1[q] = v[q];
    if (lower) F2[q] = (i == j0 + q) ? (T)1 : (T)0;  // L^-1 starts as I (lower blocks)
  }
}

// ------------------------------------------------------------------ the 32 x 32 diagonal block
// Factor one diagonal block A_kk = L_u D L_u^T (L_u unit lower triangular)
// with one warp; lane i holds row i as a[c].  Step j takes the pivot d_j and
// the next row's entry a_{j+1,j} by shuffle (the chain from one pivot to the
// next runs through shuffles and registers only), publishes the rest of
// column j through the shared array col (16-byte broadcast reads), and updates
// the trailing entries a[c] -= (a[j] / d_j) a_cj (fully unrolled, so every
// register index is a constant).  On return a[c] = L_u[lane][c] (1 on the
// diagonal, 0 above) and the result is d_lane.  A non-positive pivot is
// flagged (counters[3]) and replaced by a tiny one.
template <typename T>
__device__ __forceinline__ T warp_ldl_block(T (&a)[BS], T* col, const ProbDesc& d) {
  const int lane = threadIdx.x & 31;
  constexpr int V = 16 / (int)sizeof(T);  // column entries per 16-byte shared load (col is 16-byte aligned)
  bool bad = false;
  T dl = (T)1;
#pragma unroll
  for (int j = 0; j < BS; ++j) {
    T piv = __shfl_sync(0xffffffffu, a[j], j);
    const T cnext = j + 1 < BS ? __shfl_sync(0xffffffffu, a[j], j + 1) : (T)0;  // a_{j+1,j}
    col[lane] = a[j];
    __syncwarp();
    if (!(piv > (T)0)) {  // not positive definite at this precision: flag, continue with a tiny pivot
      bad = true;
      piv = (T)1e-30;
    }
    const T t = a[j] * fast_rcp(piv);  // L_u[lane][j] for lane > j
    if (j + 1 < BS) a[j + 1] = fma(-t, cnext, a[j + 1]);
    T cv[BS];  // col[c] for c >= j + 2, read 16 bytes at a time
#pragma unroll
    for (int g = 0; g < BS / V; ++g) {
      if ((g + 1) * V - 1 < j + 2) continue;
      if constexpr (V == 4) {
        const float4 q = reinterpret_cast<const float4*>(col)[g];
        cv[4 * g] = q.x, cv[4 * g + 1] = q.y, cv[4 * g + 2] = q.z, cv[4 * g + 3] = q.w;
      } else {
        const double2 q = reinterpret_cast<const double2*>(col)[g];
        cv[2 * g] = q.x, cv[2 * g + 1] = q.y;
      }
    }
#pragma unroll
    for (int c = j + 2; c < BS; ++c) a[c] = fma(-t, cv[c], a[c]);
    if (lane == j) dl = piv;
    a[j] = lane > j ? t : (lane == j ? (T)1 : (T)0);
    __syncwarp();
  }
  if (bad && lane == 0) atomicAdd(&d.counters[3], 1ull);
  return dl;
}

// X = L^-1 of a unit lower-triangular 32 x 32 block by doubling, with all 256
// threads: with X holding the inverses of the diagonal blocks of size s,
//   [L11 0; L21 L22]^-1 = [X11 0; -X22 (L21 X11) X22]
// fills the blocks of size 2 s (s = 1, 2, ..., 16; at each size 16 s entries,
// one per thread).  L in l, X in x (its diagonal already 1, zero elsewhere),
// z scratch.
template <typename T>
__device__ __forceinline__ void tri_inverse_block(const T (*l)[BS + 1], T (*x)[BS + 1], T (*z)[BS + 1]) {
#pragma unroll
  for (int s = 1; s < BS; s *= 2) {
    const int e = threadIdx.x;
    const bool act = e < 16 * s;
    // entry e of this size: block b = e / (s s), row r0 + e % (s s) / s, column c0 + e % s
    const int b = e / (s * s), r = 2 * s * b + s + (e % (s * s)) / s, c = 2 * s * b + e % s;
    const int base = 2 * s * b;
    if (act) {
      T acc = (T)0;
#pragma unroll
      for (int t = 0; t < s; ++t) acc = fma(l[r][base + t], x[base + t][c], acc);  // (L21 X11)[r][c]
      z[r][c] = acc;
    }
    __syncthreads();
    if (act) {
      T acc = (T)0;
#pragma unroll
      for (int t = 0; t < s; ++t) acc = fma(x[r][base + s + t], z[base + s + t][c], acc);  // (X22 Y)[r][c]; X22 is 0 above its diagonal
      x[r][c] = -acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ factor tasks
// Each task is one 32 x 32 tile operation done by a CTA of 256 threads (4
// outputs per thread: row ty + 8 s, column tx) with its operands staged in
// the shared tiles x and y.  Offsets are 32-bit (npad^2 < 2^31).
template <typename T>
using Tile = T (*)[BS + 1];

// u -> (i, j) with 0 <= j <= i and u = i (i + 1) / 2 + j (u < 2^24, exact in FP32).
__device__ __forceinline__ void tri_index(int u, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= u) ++r;
  while (r * (r + 1) / 2 > u) --r;
  i = r;
  j = u - r * (r + 1) / 2;
}

// out (-)= X Y^T or X Y, 32 x 32 x 32, operands in the shared tiles.
template <typename T, bool YT>
__device__ __forceinline__ void tile_product(Tile<T> x, Tile<T> y, T (&acc)[4]) {
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
#pragma unroll
  for (int s = 0; s < 4; ++s) acc[s] = (T)0;
#pragma unroll 8
  for (int t = 0; t < BS; ++t) {
    const T yv = YT ? y[tx][t] : y[t][tx];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = fma(x[ty + 8 * s][t], yv, acc[s]);
  }
}

template <typename T>
__device__ __forceinline__ void load_two(Tile<T> x, const T* X, Tile<T> y, const T* Y, int ldx, int ldy) {
  // every global load is issued before the first shared store (the compiler
  // cannot reorder them across stores it cannot prove disjoint)
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T rx[4], ry[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    rx[s] = X[(ty + 8 * s) * ldx + tx];
    ry[s] = Y[(ty + 8 * s) * ldy + tx];
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    x[ty + 8 * s][tx] = rx[s];
    y[ty + 8 * s][tx] = ry[s];
  }
  __syncthreads();
}

// A contiguous 32 x 32 tile (a diagonal-block inverse) into shared memory.
template <typename T>
__device__ __forceinline__ void load_dense(Tile<T> x, const T* X) {
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T rx[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) rx[s] = X[(ty + 8 * s) * BS + tx];
#pragma unroll
  for (int s = 0; s < 4; ++s) x[ty + 8 * s][tx] = rx[s];
}

// Pair u of the trailing update of step k (t = nblk - k - 1 blocks remain):
// column by column, the diagonal tile first, so the next block column is
// complete early.
__device__ __forceinline__ void trail_pair(int k, int t, int u, int& i, int& j) {
  int a, b;
  tri_index(t * (t + 1) / 2 - 1 - u, a, b);
  j = k + 1 + (t - 1 - a);
  i = k + 1 + (t - 1 - b);
}

// ------------------------------------------------------------------ the factor as one dataflow launch
// The blocked Cholesky A = L L^T, the inverse factor X = L^-1 and T = A^-1 =
// X^T X are one launch of 32 x 32 tile tasks (nb blocks, step k = block
// column k):
//   C        the chain of one or more problems, step by step: A_kk -= L_{k,k-1}
//            L_{k,k-1}^T, factor, write inv(L_kk); the two blocks below the
//            diagonal of the previous column and of this one, L_{k+1,k-1} (its
//            last trailing update, from step k - 2, applied here) and L_{k+1,k}.
//            This is the critical path; one CTA runs it without handing over
//            between steps, and the only block it takes from another task
//            (L_{k+1,k-2}) was released two steps earlier.
//   P(k) i   i >= k + 3: A_ik -= L_{i,k-1} L_{k,k-1}^T, then L_ik = A_ik inv(L_kk)^T
//   T(k) i,j trailing update of the columns j >= k + 2: A_ij -= L_ik L_jk^T
//   S(k) j   row k of X: X_kj = inv(L_kk) (X_kj - L_{k,k-1} X_{k-1,j}) (j < k), X_kk = inv(L_kk)
//   U(k) i,j i >= k + 2, j <= k: X_ij -= L_ik X_kj
//   R(t) i,j j <= i <= t: row t's share of T_ij = sum_{t >= i} X_ti^T X_tj, added
//            in the order of t (the last one also writes T_ji = T_ij^T)
// Tasks are claimed from one counter: first the G chains (problem p belongs
// to chain p mod G), then for k = 0, 1, ...: P(k), T(k), S(k - lag),
// U(k - lag), R(k - lag); then the last lag steps of S, U and R.  Each task
// waits only for the tiles it reads and writes, through per-tile states
// (tflag, zeroed before the launch):
//   SA(i, j), j <= i:  trailing updates applied to tile (i, j) of A by T tasks
//                      (k after T(k - 1)); j + 1 once L_ij (i > j) or inv(L_jj)
//                      (i = j) is written.
//   SX(i, j), j <= i:  U updates applied to tile (i, j) of X (i - j - 1 after
//                      U(i - 2)); i - j + 1 once S(i) has made it final.
//   ST(i, j), j <= i:  rows of X added into T_ij (t - i + 1 after R(t)).
//   C step k:  SA(k, k), SA(k + 1, k) >= k - 1, SA(k + 1, k - 1) >= k - 2, SA(k + 1, k - 2) >= k - 1
//   P(k) i:    SA(k, k) > k, SA(i, k - 1) >= k, SA(k, k - 1) >= k, SA(i, k) >= k - 1
//   T(k) i,j:  SA(i, k) > k, SA(j, k) > k, SA(i, j) >= k
//   S(k) j:    SA(k, k) > k; for j < k also SA(k, k - 1) >= k, SX(k - 1, j) >= k - j, SX(k, j) >= k - 1 - j
//   U(k) i,j:  SX(k, j) > k - j, SA(i, k) > k, SX(i, j) >= k - j
//   R(t) i,j:  SX(t, i) > t - i, SX(t, j) > t - j, ST(i, j) >= t - i
// Apart from the chains, every task waits only for tasks claimed before it,
// and a chain at step k waits only for tasks of steps below k, which depend
// on chain steps below k: once G + 1 CTAs run, nothing can deadlock and no
// co-residency is needed.  Waits are bounded all the same: on expiry the
// launch is abandoned (sync[2] != 0) and counters[6] of every problem raised.
// sync[0..1] is the claim counter (64-bit); sync[3] stays zero (the test
// injection RSM_FAULT_DEVICE_WAIT waits for it); all zero before the launch.
constexpr uint32_t kDepPolls = 1u << 24;  // polls (64 ns sleeps) of one dependency wait
constexpr int kMaxDevices = 64;           // devices whose factor-launch width is cached
constexpr uint32_t kDepPollsInjected = 1u << 12;  // the same under RSM_FAULT_DEVICE_WAIT (a few ms)
__shared__ uint32_t s_poll_limit;  // the factor launch's bound, set by each CTA at its start
constexpr int kFactorTiles = 9;           // shared 32 x 33 tiles per CTA

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait of one thread for *p >= need (p null: none): relaxed polls with
// a short sleep, then an acquire fence, so that the CTA's later reads see what
// the flag publishes.  False if the wait ran out or the launch was abandoned.
__device__ __forceinline__ bool wait_flag(const unsigned* p, unsigned need, unsigned* sync,
                                          const ProbDesc* __restrict__ descs, int nprob) {
  if (p == nullptr) return true;
  bool ok = true;
  const uint32_t limit = s_poll_limit;
  for (uint32_t it = 0; ld_relaxed(p) < need; ++it) {
    if (it >= limit || ((it & 15u) == 15u && *(volatile unsigned*)&sync[2] != 0u)) {
      ok = false;
      break;
    }
    __nanosleep(64);
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  if (!ok && atomicExch(&sync[2], 1u) == 0u)
    for (int q = 0; q < nprob; ++q) atomicAdd(&descs[q].counters[6], 1ull);
  return ok;
}

// Each thread with p != null waits; false for every thread of the CTA if any wait failed.
__device__ __forceinline__ bool wait_tiles(const unsigned* p, unsigned need, unsigned* sync,
                                           const ProbDesc* __restrict__ descs, int nprob) {
  const bool ok = wait_flag(p, need, sync, descs, nprob);
  return __syncthreads_and(ok) != 0;
}

// AND of ok over the nthreads threads of named barrier id (a multiple of 32).
__device__ __forceinline__ bool bar_and(int id, int nthreads, bool ok) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((unsigned)ok), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Chain step k: wait for the tiles it reads to have had the trailing updates
// that other tasks apply, then load them:
//   Y  = A_kk, W1 = A_{k+1,k}                   (updates of steps below k - 1 applied)
//   Ls = L_{k,k-1}, Lq = L_{k-1,k-2}, Dp = inv(L_{k-1,k-1})   (written by this chain)
//   Wp = A_{k+1,k-1}                             (updates of steps below k - 2 applied)
//   Lp = L_{k+1,k-2}                             (from another task, two steps back)
// Warp 1 waits, so that the release of the previous step by thread 0 can overlap.
template <typename T>
__device__ bool chain_load(const ProbDesc& d, int k, Tile<T>* tl, unsigned* sync, const ProbDesc* __restrict__ descs,
                           int nprob, bool inject = false) {
  const int np = npad_of(d), nb = d.nblk, tid = threadIdx.x;
  const int tx = tid % BS, ty = tid / BS;
  const unsigned* SA = d.tflag;
  const bool b1 = k + 1 < nb;
  const unsigned* wp = nullptr;
  unsigned wn = 0;
  if (tid == 32 && k >= 2) wp = &SA[k * nb + k], wn = k - 1;
  if (tid == 33 && b1 && k >= 2) wp = &SA[(k + 1) * nb + k], wn = k - 1;
  if (tid == 34 && b1 && k >= 3) wp = &SA[(k + 1) * nb + k - 1], wn = k - 2;
  if (tid == 35 && b1 && k >= 2) wp = &SA[(k + 1) * nb + k - 2], wn = k - 1;
  if (tid == 36 && inject) wp = &sync[3], wn = 1;  // test injection: a word nothing sets
  if (!wait_tiles(wp, wn, sync, descs, nprob)) return false;
  const T* F = F1of<T>(d);
  const T* Dg = Dinvof<T>(d);
  T r[7][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int y = ty + 8 * s;
    r[0][s] = F[(k * BS + y) * np + k * BS + tx];
    r[1][s] = k >= 1 ? F[(k * BS + y) * np + (k - 1) * BS + tx] : (T)0;
    r[2][s] = b1 ? F[((k + 1) * BS + y) * np + k * BS + tx] : (T)0;
    r[3][s] = b1 && k >= 1 ? F[((k + 1) * BS + y) * np + (k - 1) * BS + tx] : (T)0;
    r[4][s] = b1 && k >= 2 ? F[((k + 1) * BS + y) * np + (k - 2) * BS + tx] : (T)0;
    r[5][s] = b1 && k >= 2 ? F[((k - 1) * BS + y) * np + (k - 2) * BS + tx] : (T)0;
    r[6][s] = b1 && k >= 1 ? Dg[(k - 1) * BS * BS + y * BS + tx] : (T)0;
  }
  constexpr int dst[7] = {0, 1, 2, 3, 6, 7, 8};  // Y, Ls, W1, Wp, Lp, Lq, Dp
#pragma unroll
  for (int q = 0; q < 7; ++q)
#pragma unroll
    for (int s = 0; s < 4; ++s) tl[dst[q]][ty + 8 * s][tx] = r[q][s];
  __syncthreads();
  return true;
}

// Chain step k with its tiles loaded (chain_load).  A_kk takes its last
// trailing update; then warp 0 factors the diagonal block while four other warps
// finish L_{k+1,k-1} = (A_{k+1,k-1} - L_{k+1,k-2} L_{k-1,k-2}^T) inv(L_{k-1,k-1})^T,
// release it, and apply the last trailing update to A_{k+1,k}; then all
// threads invert the factor and form L_{k+1,k}.
constexpr int kPanelWarps = 6, kPanelRows = (BS + kPanelWarps - 1) / kPanelWarps;  // the chain's panel warps, rows per thread
constexpr int kPanelBar = 32 * (kPanelWarps + 1);  // named barrier 1: the panel warps and warp 4
template <typename T>
__device__ bool chain_step(const ProbDesc& d, int k, Tile<T>* tl, unsigned* sync, const ProbDesc* __restrict__ descs,
                           int nprob) {
  const int np = npad_of(d), nb = d.nblk, tid = threadIdx.x;
  const int tx = tid % BS, ty = tid / BS;
  unsigned* SA = d.tflag;
  const bool b1 = k + 1 < nb;
  T* F = F1of<T>(d);
  Tile<T> Y = tl[0], Ls = tl[1], W1 = tl[2], Wp = tl[3], Dv = tl[4], Z = tl[5], Lp = tl[6], Lq = tl[7], Dp = tl[8];
  if (k >= 1) {
    T acc[4];
    tile_product<T, true>(Ls, Ls, acc);  // L_{k,k-1} L_{k,k-1}^T
#pragma unroll
    for (int s = 0; s < 4; ++s) Y[ty + 8 * s][tx] -= acc[s];
    __syncthreads();
  }
  // A_kk = L_u D L_u^T, so L_kk = L_u D^1/2 and inv(L_kk) = D^-1/2 inv(L_u)
  T* rs = &Z[0][0];  // D^-1/2 (the inverse below uses rows >= 1 of Z only)
  if (tid < 32) {
    T a[BS];
#pragma unroll
    for (int c = 0; c < BS; ++c) a[c] = Y[tid][c];
    const T dl = warp_ldl_block<T>(a, &Dv[0][0], d);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      Y[tid][c] = a[c];
      Dv[tid][c] = c == tid ? (T)1 : (T)0;
    }
    rs[tid] = fast_rsqrt(dl);
  } else if ((tid < 128 || tid >= 160) && b1 && k >= 1) {
    // warps 1, 2, 3, 5, 6 and 7 (warp 4 would share a scheduler with warp 0,
    // whose factorisation is the critical path): thread = column cx, rows wb +
    // 6 s.  Six warps rather than four: these three products took longer than
    // warp 0's factorisation (3.8 against 2.0 us per step at four warps).
    // Their barriers include warp 4, which publishes L_{k+1,k-1}.
    const int wb = tid < 128 ? tid / 32 - 1 : tid / 32 - 2, cx = tid % BS;
    auto in = [&](int s) { return s < kPanelRows - 1 || wb + kPanelWarps * s < BS; };  // row wb + 6 s exists
    T acc[kPanelRows];
    if (k >= 2) {  // A_{k+1,k-1} -= L_{k+1,k-2} L_{k-1,k-2}^T
#pragma unroll
      for (int s = 0; s < kPanelRows; ++s) acc[s] = (T)0;
#pragma unroll 8
      for (int t = 0; t < BS; ++t) {
        const T lv = Lq[cx][t];
#pragma unroll
        for (int s = 0; s < kPanelRows; ++s)
          if (in(s)) acc[s] = fma(Lp[wb + kPanelWarps * s][t], lv, acc[s]);
      }
#pragma unroll
      for (int s = 0; s < kPanelRows; ++s)
        if (in(s)) Wp[wb + kPanelWarps * s][cx] -= acc[s];
      bar_and(1, kPanelBar, true);
    }
    // L_{k+1,k-1} = A_{k+1,k-1} inv(L_{k-1,k-1})^T, into F1 and (for the next product) Lp
#pragma unroll
    for (int s = 0; s < kPanelRows; ++s) acc[s] = (T)0;
#pragma unroll 8
    for (int t = 0; t < BS; ++t) {
      const T dv = Dp[cx][t];
#pragma unroll
      for (int s = 0; s < kPanelRows; ++s)
        if (in(s)) acc[s] = fma(Wp[wb + kPanelWarps * s][t], dv, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kPanelRows; ++s)
      if (in(s)) {
        F[((k + 1) * BS + wb + kPanelWarps * s) * np + (k - 1) * BS + cx] = acc[s];
        Lp[wb + kPanelWarps * s][cx] = acc[s];
      }
    bar_and(1, kPanelBar, true);
    // A_{k+1,k} -= L_{k+1,k-1} L_{k,k-1}^T
#pragma unroll
    for (int s = 0; s < kPanelRows; ++s) acc[s] = (T)0;
#pragma unroll 8
    for (int t = 0; t < BS; ++t) {
      const T lv = Ls[cx][t];
#pragma unroll
      for (int s = 0; s < kPanelRows; ++s)
        if (in(s)) acc[s] = fma(Lp[wb + kPanelWarps * s][t], lv, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < kPanelRows; ++s)
      if (in(s)) W1[wb + kPanelWarps * s][cx] -= acc[s];
  } else if (b1 && k >= 1) {
    // warp 4: once L_{k+1,k-1} is in F1, its release (a GPU-scope fence) is
    // issued here, so that it does not hold up a warp with a product left to do
    if (k >= 2) bar_and(1, kPanelBar, true);
    bar_and(1, kPanelBar, true);
    if (tid == 128) st_release(&SA[(k + 1) * nb + k - 1], (unsigned)k);
  }
  __syncthreads();
  T rsr[4];  // D^-1/2 of the rows ty + 8 s, and of column tx
#pragma unroll
  for (int s = 0; s < 4; ++s) rsr[s] = rs[ty + 8 * s];
  const T rsc = rs[tx];
  tri_inverse_block<T>(Y, Dv, Z);  // inv(L_u); it never writes row 0 of Z
  T* Dg = Dinvof<T>(d) + k * BS * BS;
#pragma unroll
  for (int s = 0; s < 4; ++s) Dg[(ty + 8 * s) * BS + tx] = Dv[ty + 8 * s][tx] * rsr[s];
  if (b1) {
    T acc[4];
    tile_product<T, true>(W1, Dv, acc);  // A_{k+1,k} inv(L_u)^T, then the column scale D^-1/2
#pragma unroll
    for (int s = 0; s < 4; ++s) F[((k + 1) * BS + ty + 8 * s) * np + k * BS + tx] = acc[s] * rsc;
  }
  __syncthreads();
  if (tid == 0) {
    st_release(&SA[k * nb + k], (unsigned)k + 1u);
    if (b1) st_release(&SA[(k + 1) * nb + k], (unsigned)k + 1u);
  }
  return true;
}

// P(k) for tile (i, k), i >= k + 3: the last trailing update (step k - 1) is
// applied while the chain may still be factoring A_kk; then L_ik = A_ik inv(L_kk)^T.
template <typename T>
__device__ bool panel_task(const ProbDesc& d, int np, int k, int i, Tile<T> x, Tile<T> y, unsigned* sync,
                           const ProbDesc* __restrict__ descs, int nprob) {
  T* F = F1of<T>(d);
  T* Aik = F + i * BS * np + k * BS;
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) a[s] = Aik[(ty + 8 * s) * np + tx];
  if (k > 0) {
    load_two<T>(x, F + i * BS * np + (k - 1) * BS, y, F + k * BS * np + (k - 1) * BS, np, np);
    T acc[4];
    tile_product<T, true>(x, y, acc);
#pragma unroll
    for (int s = 0; s < 4; ++s) a[s] -= acc[s];
  }
  const int nb = d.nblk;
  if (!wait_tiles(threadIdx.x == 0 ? &d.tflag[k * nb + k] : nullptr, (unsigned)k + 1u, sync, descs, nprob))
    return false;
#pragma unroll
  for (int s = 0; s < 4; ++s) x[ty + 8 * s][tx] = a[s];
  load_dense<T>(y, Dinvof<T>(d) + k * BS * BS);
  __syncthreads();
  T acc[4];
  tile_product<T, true>(x, y, acc);  // A_ik inv(L_kk)^T
#pragma unroll
  for (int s = 0; s < 4; ++s) Aik[(ty + 8 * s) * np + tx] = acc[s];
  return true;
}

// T(k): A_ij -= L_ik L_jk^T.
template <typename T>
__device__ void trail_task(const ProbDesc& d, int np, int k, int i, int j, Tile<T> x, Tile<T> y) {
  T* F = F1of<T>(d);
  T* Aij = F + i * BS * np + j * BS;
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) a[s] = Aij[(ty + 8 * s) * np + tx];
  load_two<T>(x, F + i * BS * np + k * BS, y, F + j * BS * np + k * BS, np, np);
  T acc[4];
  tile_product<T, true>(x, y, acc);
#pragma unroll
  for (int s = 0; s < 4; ++s) Aij[(ty + 8 * s) * np + tx] = a[s] - acc[s];
}

// S(k): row k of X = L^-1 (block forward substitution; its last update, from
// step k - 1, is applied here).
template <typename T>
__device__ void linv_row_task(const ProbDesc& d, int np, int k, int j, Tile<T> x, Tile<T> y, Tile<T> z) {
  T* X = F2of<T>(d);
  T* Xkj = X + k * BS * np + j * BS;
  const T* D = Dinvof<T>(d) + k * BS * BS;
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  if (j == k) {
    T rx[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) rx[s] = D[(ty + 8 * s) * BS + tx];
#pragma unroll
    for (int s = 0; s < 4; ++s) Xkj[(ty + 8 * s) * np + tx] = rx[s];
    return;
  }
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) a[s] = Xkj[(ty + 8 * s) * np + tx];
  load_dense<T>(z, D);
  load_two<T>(x, F1of<T>(d) + k * BS * np + (k - 1) * BS, y, X + (k - 1) * BS * np + j * BS, np, np);
  T acc[4];
  tile_product<T, false>(x, y, acc);  // L_{k,k-1} X_{k-1,j}
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 4; ++s) y[ty + 8 * s][tx] = a[s] - acc[s];
  __syncthreads();
  tile_product<T, false>(z, y, acc);  // inv(L_kk) (...)
#pragma unroll
  for (int s = 0; s < 4; ++s) Xkj[(ty + 8 * s) * np + tx] = acc[s];
}

// U(k): X_ij -= L_ik X_kj.
template <typename T>
__device__ void linv_update_task(const ProbDesc& d, int np, int k, int i, int j, Tile<T> x, Tile<T> y) {
  T* X = F2of<T>(d);
  T* Xij = X + i * BS * np + j * BS;
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) a[s] = Xij[(ty + 8 * s) * np + tx];
  load_two<T>(x, F1of<T>(d) + i * BS * np + k * BS, y, X + k * BS * np + j * BS, np, np);
  T acc[4];
  tile_product<T, false>(x, y, acc);
#pragma unroll
  for (int s = 0; s < 4; ++s) Xij[(ty + 8 * s) * np + tx] = a[s] - acc[s];
}

// R(t): T_ij (+)= X_ti^T X_tj; the last row also writes T_ji = T_ij^T.
template <typename T>
__device__ void trow_task(const ProbDesc& d, int np, int t, int i, int j, Tile<T> x, Tile<T> y) {
  T* Tm = Tof<T>(d);
  const T* X = F2of<T>(d);
  T* Tij = Tm + i * BS * np + j * BS;
  const int tx = threadIdx.x % BS, ty = threadIdx.x / BS;
  T a[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) a[s] = t > i ? Tij[(ty + 8 * s) * np + tx] : (T)0;
  load_two<T>(x, X + t * BS * np + i * BS, y, X + t * BS * np + j * BS, np, np);
#pragma unroll 8
  for (int v = 0; v < BS; ++v) {
    const T yv = y[v][tx];
#pragma unroll
    for (int s = 0; s < 4; ++s) a[s] = fma(x[v][ty + 8 * s], yv, a[s]);
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) Tij[(ty + 8 * s) * np + tx] = a[s];
  if (t == d.nblk - 1 && i != j) {
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) x[ty + 8 * s][tx] = a[s];
    __syncthreads();
    T* Tji = Tm + j * BS * np + i * BS;
#pragma unroll
    for (int s = 0; s < 4; ++s) Tji[(ty + 8 * s) * np + tx] = x[tx][ty + 8 * s];
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    k_factor(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ tables, int nprob, FactorTables ft,
             unsigned* sync, int nchain) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char factor_smem[];
  Tile<T> tl[kFactorTiles];
#pragma unroll
  for (int q = 0; q < kFactorTiles; ++q) tl[q] = reinterpret_cast<Tile<T>>(factor_smem) + q * BS;
  Tile<T> x = tl[0], y = tl[1], z = tl[2];
  __shared__ unsigned long long s_task;
  if (threadIdx.x == 0) s_poll_limit = ft.poll_limit;
  const int K = ft.nsteps, lag = ft.lag;
  const int nseg = 5 * K + 3 * lag;
  const int64_t* seg_start = tables + ft.phase;  // task prefix over the segments after the chains
  const unsigned long long ntask = (unsigned long long)nchain + (unsigned long long)seg_start[nseg];
  const size_t n1 = (size_t)nprob + 1;
  unsigned long long* claim = reinterpret_cast<unsigned long long*>(sync);
  const int tid = threadIdx.x;
  int seg = 0;
  for (;;) {
    __syncthreads();  // the previous task is done with the tiles and s_task
    if (tid == 0) s_task = atomicAdd(claim, 1ull);
    __syncthreads();
    const unsigned long long task = s_task;
    if (task >= ntask) return;
    if (task < (unsigned long long)nchain) {
      // chain: for k = 0, 1, ...: every problem of the chain with nblk > k;
      // the next step's tiles are loaded right after each step's release
      const int c = (int)task;
      int k = 0, p = c;
      auto advance = [&](int& kk, int& pp) {  // next (step, problem) of the chain; kk = K at the end
        for (;;) {
          pp += nchain;
          if (pp >= nprob) {
            pp = c;
            if (++kk >= K) return;
          }
          if (kk < descs[pp].nblk) return;
        }
      };
      if (k >= descs[p].nblk) advance(k, p);
      if (k < K && !chain_load<T>(descs[p], k, tl, sync, descs, nprob, ft.fault_wait != 0 && c == 0)) return;
      while (k < K) {
        if (!chain_step<T>(descs[p], k, tl, sync, descs, nprob)) return;
        advance(k, p);
        if (k < K && !chain_load<T>(descs[p], k, tl, sync, descs, nprob)) return;
      }
      continue;
    }
    const int64_t u = (int64_t)(task - (unsigned long long)nchain);
    while (u >= seg_start[seg + 1]) ++seg;
    int kind, k;  // kind: 0 P, 1 T, 2 S, 3 U, 4 R
    if (seg < 5 * K) {
      k = seg / 5;
      kind = seg % 5;
      if (kind >= 2) k -= lag;
    } else {
      k = K - lag + (seg - 5 * K) / 3;
      kind = 2 + (seg - 5 * K) % 3;
    }
    const int64_t* tab = kind < 2 ? tables + ft.step + (size_t)k * 2 * n1 + (size_t)kind * n1
                                  : tables + ft.linv + (size_t)k * 3 * n1 + (size_t)(kind - 2) * n1;
    const int64_t g = u - seg_start[seg];
    const int p = find_problem(tab, nprob, g);
    const ProbDesc& d = descs[p];
    const int np = npad_of(d), nb = d.nblk;
    const int l = (int)(g - tab[p]);
    unsigned* SA = d.tflag;                // SA(i, j) = SA[i * nb + j]
    unsigned* SX = d.tflag + nb * nb;      // SX(i, j) = SX[i * nb + j]
    unsigned* ST = d.tflag + 2 * nb * nb;  // ST(i, j) = ST[i * nb + j]
    // the task's tiles, its conditions (thread t waits for condition t) and its output state
    int i = 0, j = 0;
    const unsigned* wp = nullptr;
    unsigned wn = 0;
    unsigned* out = nullptr;
    unsigned out_v = 0;
    switch (kind) {
      case 0:  // P(k), tile (i, k)
        i = k + 3 + l;
        if (k > 0) {
          if (tid == 0) wp = &SA[i * nb + k - 1], wn = k;
          if (tid == 1) wp = &SA[k * nb + k - 1], wn = k;
          if (tid == 2) wp = &SA[i * nb + k], wn = k - 1;
        }
        out = &SA[i * nb + k], out_v = k + 1;
        break;
      case 1:  // T(k), tile (i, j), j >= k + 2
        trail_pair(k + 1, nb - k - 2, l, i, j);
        if (tid == 0) wp = &SA[i * nb + k], wn = k + 1;
        if (tid == 1) wp = &SA[j * nb + k], wn = k + 1;
        if (tid == 2) wp = &SA[i * nb + j], wn = k;
        out = &SA[i * nb + j], out_v = k + 1;
        break;
      case 2:  // S(k), tile (k, j)
        j = l;
        if (tid == 0) wp = &SA[k * nb + k], wn = k + 1;
        if (j < k) {
          if (tid == 1) wp = &SA[k * nb + k - 1], wn = k;
          if (tid == 2) wp = &SX[(k - 1) * nb + j], wn = k - j;
          if (tid == 3) wp = &SX[k * nb + j], wn = k - 1 - j;
        }
        out = &SX[k * nb + j], out_v = k - j + 1;
        break;
      case 3:  // U(k), tile (i, j), i >= k + 2
        i = k + 2 + l / (k + 1), j = l % (k + 1);
        if (tid == 0) wp = &SX[k * nb + j], wn = k - j + 1;
        if (tid == 1) wp = &SA[i * nb + k], wn = k + 1;
        if (tid == 2) wp = &SX[i * nb + j], wn = k - j;
        out = &SX[i * nb + j], out_v = k - j + 1;
        break;
      default:  // R(k), tile (i, j), j <= i <= k
        tri_index(l, i, j);
        if (tid == 0) wp = &SX[k * nb + i], wn = k - i + 1;
        if (tid == 1) wp = &SX[k * nb + j], wn = k - j + 1;
        if (tid == 2) wp = &ST[i * nb + j], wn = k - i;
        out = &ST[i * nb + j], out_v = k - i + 1;
        break;
    }
    if (!wait_tiles(wp, wn, sync, descs, nprob)) return;
    switch (kind) {
      case 0:
        if (!panel_task<T>(d, np, k, i, x, y, sync, descs, nprob)) return;
        break;
      case 1: trail_task<T>(d, np, k, i, j, x, y); break;
      case 2: linv_row_task<T>(d, np, k, j, x, y, z); break;
      case 3: linv_update_task<T>(d, np, k, i, j, x, y); break;
      default: trow_task<T>(d, np, k, i, j, x, y); break;
    }
    __syncthreads();
    if (tid == 0) st_release(out, out_v);
  }
}

// ------------------------------------------------------------------ block iteration (FP64)
// X (n x kx, row-major) starts from deterministic Philox noise in [-1, 1).
__global__ void __launch_bounds__(256) k_init_X(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  pdl_enter();
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
constexpr int kPSplit = 16;  // split of the inner dimension of the preconditioner product (R slots 1..16)
constexpr int kMxRows = 128;  // rows per CTA of M X (one per thread)
constexpr int kMxSub = 64;    // columns of X staged per pass
constexpr int kMxGroup = 16;  // loads of M issued together (L2 latency is hidden by their number, not by warps)

// out = M X to about FP64 accuracy on the FP32 pipes (FP64 instructions issue
// far slower than FP32 ones here).  M is held as FP32 pairs (hi + lo, 48
// significant bits, written by k_eig_prep); X is split the same way when it is
// staged.  Per term: the head product hi*hi is split exactly (TwoProduct by
// FMA), the cross terms hi*lo + lo*hi are single FP32 products, and the running
// sum is a float pair updated by TwoSum (Knuth), so the accumulation carries
// about 2^-44 relative accuracy; the lo*lo term (2^-48) is dropped.
// Thread = row i (M is symmetric, so M[j][i] is read: consecutive threads read
// consecutive addresses); split s covers columns j in [s n / kSplit, (s+1) n / kSplit);
// the parts go to R slots and sum_mx_slots adds them in FP64 in a fixed order.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int KXB>
__global__ void __launch_bounds__(kMxRows) k_gemm_MX(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                    int nprob) {
  pdl_enter();
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
      // the loads of a group of kMxGroup columns are all in flight before the first product
      for (int g0 = 0; g0 < jn; g0 += kMxGroup) {
        float2 mv[kMxGroup];
#pragma unroll
        for (int u = 0; u < kMxGroup; ++u)
          mv[u] = g0 + u < jn ? __ldg(Mdf + (j0 + g0 + u) * n + i) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < kMxGroup; ++u) {
          if (g0 + u >= jn) break;
          const float2 m = mv[u];
#pragma unroll
          for (int c = 0; c < KXB; ++c) {
            const float2 x = xs[g0 + u][c];
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
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < KXB; ++c)
      if (c < kx) d.R[(split * n + i) * kx + c] = (double)sh[c] + (double)sl[c];
}

// out = M X in IEEE FP64 (FMA), for the refinement passes that end the
// eigensolve: the same split over the inner dimension and the same R slots as
// k_gemm_MX, with M read in FP64 (thread = row i, M[j][i] = M[i][j] by symmetry,
// so consecutive threads read consecutive addresses).
template <int KXB>
__global__ void __launch_bounds__(kMxRows) k_gemm_MX64(const ProbDesc* __restrict__ descs,
                                                      const int64_t* __restrict__ off, int nprob) {
  pdl_enter();
  __shared__ double xs[kMxSub][KXB];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int local = (int)(blockIdx.x - off[p]);
  const int n = (int)d.n;
  const int kx = d.kx;
  const int ntile = (n + kMxRows - 1) / kMxRows;
  const int split = local / ntile;
  const int i = (local % ntile) * kMxRows + threadIdx.x;
  const int j_begin = split * n / kSplit, j_end = (split + 1) * n / kSplit;
  double acc[KXB];
#pragma unroll
  for (int c = 0; c < KXB; ++c) acc[c] = 0.0;
  const double* __restrict__ M = d.M;
  for (int j0 = j_begin; j0 < j_end; j0 += kMxSub) {
    const int jn = j_end - j0 < kMxSub ? j_end - j0 : kMxSub;
    __syncthreads();
    for (int e = threadIdx.x; e < jn * KXB; e += kMxRows) {
      const int jj = e / KXB, c = e % KXB;
      xs[jj][c] = c < kx ? d.X[(j0 + jj) * kx + c] : 0.0;
    }
    __syncthreads();
    if (i < n) {
      for (int g0 = 0; g0 < jn; g0 += kMxGroup) {
        double mv[kMxGroup];
#pragma unroll
        for (int u = 0; u < kMxGroup; ++u) mv[u] = g0 + u < jn ? __ldg(M + (j0 + g0 + u) * n + i) : 0.0;
#pragma unroll
        for (int u = 0; u < kMxGroup; ++u) {
          if (g0 + u >= jn) break;
#pragma unroll
          for (int c = 0; c < KXB; ++c) acc[c] = fma(mv[u], xs[g0 + u][c], acc[c]);
        }
      }
    }
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < KXB; ++c)
      if (c < kx) d.R[(split * n + i) * kx + c] = acc[c];
}

// Start of the FP64 refinement: every problem runs it, converged or not.
__global__ void k_refine_begin(const ProbDesc* __restrict__ descs, int nprob) {
  pdl_enter();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nprob) descs[p].stats[kConvFlag] = 0.0;
}


// Partial Gram sums over chunks of kChunk rows: part[chunk] = [X^T X | X^T MX]
// (2 kx^2 values; the second half only when WITH_H).
// M X entry e (row-major n x kx): the kSplit partial products of k_gemm_MX in
// slot order (every load in flight first); stored into MX for the later steps.
__device__ __forceinline__ double sum_mx_slots(const ProbDesc& d, int e) {
  const int nk = (int)d.n * d.kx;
  double v[kSplit];
#pragma unroll
  for (int q = 0; q < kSplit; ++q) v[q] = d.R[q * nk + e];
  double s = v[0];
#pragma unroll
  for (int q = 1; q < kSplit; ++q) s += v[q];
  d.MX[e] = s;
  return s;
}

constexpr int kChunk = 64;
constexpr int kXtxThreads = 320;  // 2 kx^2 = 288 outputs at kx = 12 in one round
// With H, M X is first formed from its kSplit slots (sum_mx_slots).  Each
// partial is written as an FP32 pair.  PAIRS (FP32 factor): X and M X are
// staged as FP32 pairs and the 64-term dot products run in pair arithmetic on
// the FP32 pipes (small_df.cuh).  Otherwise (FP64 factor, an almost exact
// shift-invert whose steps leave X with column norms spread over many orders of
// magnitude until it is orthonormalised) the products run in FP64: X^T X then
// needs every bit of its smallest directions.
template <bool WITH_H, bool PAIRS>
__global__ void __launch_bounds__(kXtxThreads) k_xtx(const ProbDesc* __restrict__ descs,
                                                    const int64_t* __restrict__ off, int nprob,
                                                    double* __restrict__ part_base,
                                                    const int64_t* __restrict__ part_off) {
  pdl_enter();
  extern __shared__ DF xtx_smem[];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;  // converged: the rest of the iteration is skipped
  const int chunk = (int)(blockIdx.x - off[p]);
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  const int i0 = chunk * kChunk;
  float2* part = reinterpret_cast<float2*>(part_base + part_off[p] + chunk * 2 * kx * kx);
  const int outs = (WITH_H ? 2 : 1) * kx * kx;
  if constexpr (PAIRS) {
    DF* xs = xtx_smem;                  // kChunk x kx
    DF* ys = xtx_smem + kChunk * kx;    // kChunk x kx
    for (int e = threadIdx.x; e < kChunk * kx; e += kXtxThreads) {
      const int i = i0 + dkx.q(e);
      xs[e] = i < d.n ? df_from(d.X[i0 * kx + e]) : DF{0.f, 0.f};
      if (WITH_H) ys[e] = i < d.n ? df_from(sum_mx_slots(d, i0 * kx + e)) : DF{0.f, 0.f};
    }
    __syncthreads();
    for (int e = threadIdx.x; e < outs; e += kXtxThreads) {
      const int which = e / (kx * kx), ab = e % (kx * kx), a = dkx.q(ab), b = dkx.r(ab);
      const DF* y = which == 0 ? xs : ys;
      DFAcc s0, s1;
      for (int r = 0; r < kChunk; r += 2) {
        s0.add_prod(xs[r * kx + a], y[r * kx + b]);
        s1.add_prod(xs[(r + 1) * kx + a], y[(r + 1) * kx + b]);
      }
      DFAcc t;
      t.add(s0.get());
      t.add(s1.get());
      const DF v = t.get();
      part[e] = make_float2(v.hi, v.lo);
    }
  } else {
    double* xs = reinterpret_cast<double*>(xtx_smem);
    double* ys = xs + kChunk * kx;
    for (int e = threadIdx.x; e < kChunk * kx; e += kXtxThreads) {
      const int i = i0 + dkx.q(e);
      xs[e] = i < d.n ? d.X[i0 * kx + e] : 0.0;
      if (WITH_H) ys[e] = i < d.n ? sum_mx_slots(d, i0 * kx + e) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < outs; e += kXtxThreads) {
      const int which = e / (kx * kx), ab = e % (kx * kx), a = dkx.q(ab), b = dkx.r(ab);
      const double* y = which == 0 ? xs : ys;
      double s0 = 0.0, s1 = 0.0;
      for (int r = 0; r < kChunk; r += 2) {
        s0 = fma(xs[r * kx + a], y[r * kx + b], s0);
        s1 = fma(xs[(r + 1) * kx + a], y[(r + 1) * kx + b], s1);
      }
      const DF v = df_from(s0 + s1);
      part[e] = make_float2(v.hi, v.lo);
    }
  }
}

// ------------------------------------------------------------------ small dense algebra (one CTA per problem)
constexpr int kLs = kMaxL + 1;
constexpr int kSmallThreads = 128;  // four warps: the FP64 products use all four schedulers
typedef double DRow[kLs];
typedef float FRow[kLs];

// Sum the per-chunk partials (FP32 pairs, see k_xtx) in chunk order: S = X^T X
// (and H = X^T M X), as FP32 pairs.
__device__ inline void reduce_partials(const ProbDesc& d, const float2* part, DFRow* S, DFRow* H, int kx,
                                       int nthreads) {
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  const int nchunk = (int)((d.n + kChunk - 1) / kChunk);
  for (int e = threadIdx.x; e < kx * kx; e += nthreads) {
    DFAcc s, h;
    for (int c0 = 0; c0 < nchunk; c0 += 8) {  // the loads of 8 chunks in flight, then the sums in chunk order
      float2 xv[8], yv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + u;
        xv[u] = c < nchunk ? part[c * 2 * kx * kx + e] : make_float2(0.f, 0.f);
        yv[u] = (H && c < nchunk) ? part[c * 2 * kx * kx + kx * kx + e] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + u < nchunk) {
          s.add(DF{xv[u].x, xv[u].y});
          if (H) h.add(DF{yv[u].x, yv[u].y});
        }
    }
    S[dkx.q(e)][dkx.r(e)] = s.get();
    if (H) H[dkx.q(e)][dkx.r(e)] = h.get();
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

// Orthonormalisation step of the subspace iteration: S = X^T X (FP32-pair
// partial sums), S + s I = C C^T, small[0 .. kx^2) = Q = C^-T so that X Q has
// orthonormal columns.  FP32 factor (KP > 0): one warp, rows in registers.
// FP64 factor (KP == 0): the FP64 warp Cholesky in shared memory.
template <int KP>
__global__ void __launch_bounds__(kSmallThreads) k_orth(const ProbDesc* __restrict__ descs, int nprob,
                                                      const float2* __restrict__ part_base,
                                                      const int64_t* __restrict__ part_off) {
  pdl_enter();
  __shared__ DFRow Sp[kMaxL];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  reduce_partials(d, part_base + part_off[p], Sp, nullptr, kx, kSmallThreads);
  __syncthreads();
  if constexpr (KP > 0) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      float a[KP], y[KP];
#pragma unroll
      for (int j = 0; j < KP; ++j) a[j] = (lane < kx && j < kx) ? Sp[lane][j].hi : (lane == j ? 1.f : 0.f);
      float rdiag = 1.f;
      reg_cholesky<KP>(a, rdiag, 1e-6f, kx);
      reg_tri_inverse<KP>(a, rdiag, y);
      if (lane < kx)
#pragma unroll
        for (int c = 0; c < KP; ++c)
          if (c < kx) d.small[c * kx + lane] = (double)y[c];  // Q = C^-T: Q[c][lane] = (C^-1)[lane][c]
    }
  } else {
    __shared__ double S[kMaxL][kLs], Q[kMaxL][kLs];
    __shared__ double rdiag[kMaxL];
    for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) S[dkx.q(e)][dkx.r(e)] = df_to(Sp[dkx.q(e)][dkx.r(e)]);
    __syncthreads();
    if (threadIdx.x < 32) warp_chol_shifted<double>(S, rdiag, kx, 1e-15);
    __syncthreads();
    inv_transpose_factor<double>(S, rdiag, Q, kx);
    __syncthreads();
    for (int e = threadIdx.x; e < kx * kx; e += kSmallThreads) d.small[e] = Q[dkx.q(e)][dkx.r(e)];
  }
}

// Rayleigh-Ritz step of the block iteration, one CTA per problem, in FP32
// pairs (small_df.cuh) with FP32 seeds:
//  - S = X^T X and H = X^T M X from the partial sums;
//  - FP32 Cholesky S + s I = C C^T and Q0 = C^-T (one warp, registers), then
//    one Newton-Schulz step Q1 = Q0 (3I - Q0^T S Q0) / 2, which squares the
//    FP32 error: X Q1 is orthonormal to the pair precision;
//  - H1 = Q1^T H Q1; FP32 Jacobi of H1 gives eigenvectors to FP32 accuracy,
//    sorted by Ritz value; two Lowdin steps Q2 <- Q2 (3I - Q2^T Q2) / 2 make
//    them orthogonal to the pair precision;
//  - B = Q2^T H1 Q2 is diagonal up to the FP32 error; what matters is the
//    coupling B12 between the r wanted and the kx - r other columns, which a
//    first-order rotation removes: G = I + A with A_pq = B_pq / (B_qq - B_pp)
//    (p < r <= q, A_qp = -A_pq; the gap theta_{r+1} - theta_r keeps it
//    defined), made orthogonal by one Lowdin step.  The coupling left is
//    second order, ||B12||^2 / gap.  Mixing inside the wanted (or the other)
//    block is harmless: only the two subspaces matter.
// Writes small = [Q | H' | theta] (FP64) with Q = Q1 Q2 G, H' = Q^T H Q and
// theta = diag(H') in ascending order of the FP32 Ritz values.
constexpr int kRRThreads = 256;
constexpr size_t kRRSmem = sizeof(DFRow) * kMaxL * 8;

template <int KP>
__global__ void __launch_bounds__(kRRThreads) k_rr(const ProbDesc* __restrict__ descs, int nprob,
                                                   const float2* __restrict__ part_base,
                                                   const int64_t* __restrict__ part_off) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char rr_smem[];
  DFRow* S = reinterpret_cast<DFRow*>(rr_smem);
  DFRow* H = S + kMaxL;
  DFRow* Q1 = H + kMaxL;
  DFRow* H1 = Q1 + kMaxL;
  DFRow* Q2 = H1 + kMaxL;
  DFRow* B = Q2 + kMaxL;
  DFRow* W1 = B + kMaxL;
  DFRow* W2 = W1 + kMaxL;
  __shared__ int coupled, rotated;
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] != 0.0) return;
  const int kx = d.kx, r = d.r, tid = threadIdx.x, lane = tid & 31;
  const SmallDiv dkx((uint32_t)kx);  // quotient and remainder by kx without an integer division
  reduce_partials(d, part_base + part_off[p], S, H, kx, kRRThreads);
  __syncthreads();
  if (tid < 32) {  // Q0 = C^-T of the FP32 factor, into Q2
    float a[KP], y[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) a[j] = (lane < kx && j < kx) ? S[lane][j].hi : (lane == j ? 1.f : 0.f);
    float rdiag = 1.f;
    reg_cholesky<KP>(a, rdiag, 1e-7f, kx);
    reg_tri_inverse<KP>(a, rdiag, y);
    if (lane < kx)
#pragma unroll
      for (int c = 0; c < KP; ++c)
        if (c < kx) Q2[c][lane] = DF{y[c], 0.f};
  }
  __syncthreads();
  df_congruence(W2, Q2, S, W1, kx, kRRThreads);  // Z = Q0^T S Q0
  df_three_minus_half(W1, W2, kx, kRRThreads);   // (3I - Z) / 2
  __syncthreads();
  df_prod(Q1, Q2, false, W1, kx, kRRThreads);  // Q1 = Q0 (3I - Z) / 2
  __syncthreads();
  df_congruence(H1, Q1, H, W1, kx, kRRThreads);  // H1 = Q1^T H Q1
  if (tid < 32) {
    // FP32 Jacobi of H1 (when FP32 resolves its off-diagonal part); Q2 = its
    // eigenvector columns in ascending order of the Ritz values
    float a[KP], v[KP];
    float f = 0.f, o = 0.f;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      a[j] = (lane < kx && j < kx) ? H1[lane][j].hi : 0.f;
      v[j] = (j == lane) ? 1.f : 0.f;
      f += a[j] * a[j];
      if (j != lane) o = fmaxf(o, fabsf(a[j]));
    }
#pragma unroll
    for (int s = 16; s; s >>= 1) {
      f += __shfl_xor_sync(0xffffffffu, f, s);
      o = fmaxf(o, __shfl_xor_sync(0xffffffffu, o, s));
    }
    const float tol = 4.f * FLT_EPSILON * sqrtf(f);
    if (o > tol) reg_jacobi<KP>(a, v, tol, 40);
    const float lam = reg_pick<KP>(a, lane);
    int rank = 0;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const float lk = __shfl_sync(0xffffffffu, lam, k);
      if (k < kx && (lk < lam || (lk == lam && k < lane))) ++rank;
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int rj = __shfl_sync(0xffffffffu, rank, j);
      if (lane < kx && j < kx) Q2[lane][rj] = DF{v[j], 0.f};
    }
    if (lane == 0) {
      coupled = 0;
      rotated = o > tol;
    }
  }
  __syncthreads();
  // FP32 rotations: orthogonal in pairs, then B = Q2^T H1 Q2.  Without a Jacobi
  // rotation Q2 is a permutation, for which the Lowdin step is exactly the identity.
  if (rotated) {
    df_lowdin(Q2, W1, W2, kx, kRRThreads);
    df_lowdin(Q2, W1, W2, kx, kRRThreads);
  }
  df_congruence(B, Q2, H1, W1, kx, kRRThreads);
  // first-order decoupling of the wanted block: G = I + A (into H1), then one Lowdin step
  for (int e = tid; e < kx * kx; e += kRRThreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    float g = (a == b) ? 1.f : 0.f;
    if (a < r && b >= r)
      g = B[a][b].hi * __frcp_rn(B[b][b].hi - B[a][a].hi);
    else if (a >= r && b < r)
      g = -B[b][a].hi * __frcp_rn(B[a][a].hi - B[b][b].hi);
    if (a != b && fabsf(g) > 1e-9f) atomicOr(&coupled, 1);
    H1[a][b] = DF{g, 0.f};
  }
  __syncthreads();
  // I + A is orthogonal up to ||A||^2: below 1e-18 it needs no Lowdin step
  if (coupled) df_lowdin(H1, W1, W2, kx, kRRThreads);
  df_prod(W1, Q2, false, H1, kx, kRRThreads);  // W1 = Q2 G
  __syncthreads();
  df_prod(Q2, Q1, false, W1, kx, kRRThreads);  // Q = Q1 Q2 G (into Q2)
  __syncthreads();
  df_congruence(W2, Q2, H, W1, kx, kRRThreads);  // H' = Q^T H Q
  double* out = d.small;
  for (int e = tid; e < kx * kx; e += kRRThreads) {
    out[e] = df_to(Q2[dkx.q(e)][dkx.r(e)]);
    out[kx * kx + e] = df_to(W2[dkx.q(e)][dkx.r(e)]);
  }
  for (int c = tid; c < kx; c += kRRThreads) out[2 * kx * kx + c] = df_to(W2[c][c]);
}

// X <- X Q (FULL: also MX <- MX Q and R = MX - X H').  A CTA takes 8 rows;
// thread (row, column) computes one entry of each product from rows staged in
// shared memory.
constexpr int kRotRows = 8;
constexpr int kResSlot = 31;  // R slot of the per-tile residual sums of squares (slots 1..kPSplit: preconditioner parts)
static_assert(kResSlot > kPSplit && kResSlot < kSplit, "R slots of the residual sums and the preconditioner parts");
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
    for (int t0 = g; t0 < ntile; t0 += 8 * 8) {  // 8 loads in flight, summed in tile order
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = t0 + 8 * u < ntile ? __ldcg(pr + (t0 + 8 * u) * kx + c) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
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
// Run by the last CTA of k_rotate<true, true> to finish.
__device__ __forceinline__ void conv_check(const ProbDesc& d) {
  const int kx = d.kx, r = d.r;
  const double mx = wanted_residual_norm(d);
  if (threadIdx.x == 0) {
    const double* th = d.small + 2 * kx * kx;
    const double gap = r < kx ? th[r] - th[r - 1] : 0.0;
    const double prev = d.stats[kPrevRes];
    // converged: below the target; or predicted to reach it in one more step
    // at the rate of the last one (the FP64 refinement that follows takes that
    // step: a correction X <- X - A^-1 R with R in FP64); or no longer falling
    // (at the rounding floor of M X - X Theta) while already below kStallTol * gap
    const bool predicted = prev > 0.0 && mx < prev && mx * (mx / prev) <= kConvTol * gap;
    const bool stalled = prev > 0.0 && mx > 0.5 * prev && mx <= kStallTol * gap;
    if (gap > 0.0 && (mx <= kConvTol * gap || stalled))
      d.stats[kConvFlag] = 1.0;
    else if (gap > 0.0 && predicted)
      d.stats[kConvFlag] = 2.0;
    d.stats[kPrevRes] = mx;
    d.stats[kIterCount] += 1.0;
  }
}

template <bool FULL, bool CHECK>
__global__ void __launch_bounds__(256) k_rotate(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  pdl_enter();
  __shared__ double q[2 * kMaxL * kMaxL];
  __shared__ double xs[kRotRows][kMaxL], ms[kRotRows][kMaxL], nxs[kRotRows][kMaxL];
  __shared__ double rsq[FULL ? kRotRows : 1][kMaxL];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const double flag = d.stats[kConvFlag];
  if (flag != 0.0) {  // converged: the rest of the iteration is skipped
    // the step after a predicted stop has taken its correction: skip from now on
    if (CHECK && flag == 2.0 && blockIdx.x == off[p] && threadIdx.x == 0) d.stats[kConvFlag] = 1.0;
    return;
  }
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
  if (CHECK) {
    // the last CTA of the problem to finish runs the convergence check (counters[9]
    // counts the finished tiles and is reset for the next step)
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned long long ntile = (unsigned long long)((d.n + kRotRows - 1) / kRotRows);
      last = atomicAdd(&d.counters[9], 1ull) == ntile - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      conv_check(d);
      if (threadIdx.x == 0) d.counters[9] = 0ull;
    }
  }
}

// Product with the preconditioner A^-1 = (M + tau I)^-1 at precision T.  SRC 0:
// of the residual R (block iteration); SRC 1: of X itself (subspace iteration).
// Split over the inner dimension: CTA (row tile of 16, part s) writes its
// partial product to R slot 1 + s; k_precond_apply sums the parts in a fixed order.
constexpr int kPRows = 16;
template <typename T, int SRC, bool WIDE>  // WIDE: kx > 16 (a second output column per thread)
__global__ void __launch_bounds__(256) k_precond(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  pdl_enter();
  __shared__ T ts[kPRows][65];
  __shared__ T rs[64][kMaxL + 1];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] == 1.0) return;  // converged (a predicted stop still takes this step)
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
      ts[r][c] = (i < n && j < j_end) ? Tof<T>(d)[i * np + j] : (T)0;
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
      if (WIDE) acc[1] = fma(tv, rs[u][tc + 16 < kx ? tc + 16 : tc], acc[1]);
    }
  }
  const int i = i0 + tr;
  double* part = d.R + (1 + split) * n * kx;
  if (i < n) {
    if (tc < kx) part[i * kx + tc] = (double)acc[0];
    if (WIDE && tc + 16 < kx) part[i * kx + tc + 16] = (double)acc[1];
  }
}

// MODE 0: X <- X - sum of the parts (block iteration); MODE 1: X <- sum of the parts.
template <int MODE>
__global__ void __launch_bounds__(256) k_precond_apply(const ProbDesc* __restrict__ descs,
                                                      const int64_t* __restrict__ off, int nprob) {
  pdl_enter();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.stats[kConvFlag] == 1.0) return;  // converged (a predicted stop still takes this step)
  const int e = (int)(g - off[p]);
  const int nk = (int)d.n * d.kx;
  double v[kPSplit];
#pragma unroll
  for (int q = 0; q < kPSplit; ++q) v[q] = d.R[(1 + q) * nk + e];  // every load in flight, summed in order
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPSplit; ++q) s += v[q];
  d.X[e] = MODE == 0 ? d.X[e] - s : s;
}

// V = first r columns of X (n x r column-major, ldv); Ritz values; residual norm.
__global__ void __launch_bounds__(256) k_eig_finish(const ProbDesc* __restrict__ descs, int nprob) {
  pdl_enter();
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int kx = d.kx, r = d.r;
  for (int64_t i = threadIdx.x; i < d.n; i += 256) {  // row i of X: its r loads in flight, then the stores
    double x[kMaxR];
#pragma unroll
    for (int c = 0; c < kMaxR; ++c) x[c] = c < r ? d.X[i * kx + c] : 0.0;
#pragma unroll
    for (int c = 0; c < kMaxR; ++c)
      if (c < r) d.V[(int64_t)c * d.ldv + i] = x[c];
  }
  const double mx = wanted_residual_norm(d);
  if (threadIdx.x < kx && threadIdx.x < 32) d.stats[threadIdx.x] = d.small[2 * kx * kx + threadIdx.x];
  if (threadIdx.x == 0) d.stats[34] = mx;
}

// trace(M) of a caller-supplied M into stats[kStatTrace]: one CTA per problem,
// fixed-order tree over the diagonal.
__global__ void __launch_bounds__(256) k_trace_M(const ProbDesc* __restrict__ descs, int nprob) {
  pdl_enter();
  __shared__ double red[256];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  const int n = (int)d.n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += d.M[i * n + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.stats[kStatTrace] = red[0];
}

cudaError_t launch_trace_M(const ProbDesc* descs, int nprob, cudaStream_t s) {
  k_trace_M<<<nprob, 256, 0, s>>>(descs, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
// Every kernel of the eigen stage is launched with programmatic stream
// serialisation: each launch of the chain is scheduled as the previous one's
// CTAs exit and blocks in pdl_enter() until that grid has completed, so the ~70
// dependent launches of a decomposition do not each pay the launch latency in
// full (eigen stage 1.03 -> 0.88 ms at n = 1024).
#define RSM_LAUNCH_SMEM(kernel, blocks, threads, smem, ...)                                             \
  do {                                                                                                 \
    if ((blocks) > 0) {                                                                                \
      cudaError_t e_ = launch_chained(kernel, (unsigned)(blocks), (unsigned)(threads), (size_t)(smem), s, \
                                      __VA_ARGS__);                                                    \
      ++g_kernel_launches;                                                                             \
      if (e_ != cudaSuccess) return e_;                                                                \
    }                                                                                                  \
  } while (0)
#define RSM_LAUNCH(kernel, blocks, threads, ...) RSM_LAUNCH_SMEM(kernel, blocks, threads, 0, __VA_ARGS__)

template <typename T>
static cudaError_t launch_eig_t(const EigPlan& P, double shift_rel, int iters, cudaStream_t s) {
  const int xtx_smem = (int)(2 * kChunk * kMaxL * sizeof(double));
  auto* rot_x = k_rotate<false, false>;     // X <- X Q
  auto* rot_full = k_rotate<true, false>;   // also M X and R
  auto* rot_check = k_rotate<true, true>;   // ... and the convergence check by the last CTA
  auto* xtx_s = k_xtx<false, sizeof(T) == 4>;  // X^T X
  auto* xtx_h = k_xtx<true, sizeof(T) == 4>;   // X^T X and X^T M X
  cudaError_t ea = cudaFuncSetAttribute(xtx_h, cudaFuncAttributeMaxDynamicSharedMemorySize, xtx_smem);
  if (ea == cudaSuccess) ea = cudaFuncSetAttribute(xtx_s, cudaFuncAttributeMaxDynamicSharedMemorySize, xtx_smem);
  // the register algebra of the small steps is compiled for padded sizes KP >= kx
  const int kp = P.kx_max <= 4 ? 4 : (P.kx_max + 3) / 4 * 4;
  void (*rr)(const ProbDesc*, int, const float2*, const int64_t*) = nullptr;
  void (*orth)(const ProbDesc*, int, const float2*, const int64_t*) = nullptr;
  switch (kp) {
#define RSM_KP(K)          \
  case K:                  \
    rr = k_rr<K>;          \
    orth = k_orth<K>;      \
    break;
    RSM_KP(4) RSM_KP(8) RSM_KP(12) RSM_KP(16) RSM_KP(20) RSM_KP(24) RSM_KP(28) RSM_KP(32)
#undef RSM_KP
    default: return cudaErrorInvalidValue;
  }
  if (sizeof(T) == 8) orth = k_orth<0>;
  if (ea == cudaSuccess) ea = cudaFuncSetAttribute(rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRRSmem);
  if (ea != cudaSuccess) return ea;
  const float2* part = reinterpret_cast<const float2*>(P.part);
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
  const bool wide = P.kx_max > 16;
  auto* precond_x = wide ? k_precond<T, 1, true> : k_precond<T, 1, false>;  // A^-1 X
  auto* precond_r = wide ? k_precond<T, 0, true> : k_precond<T, 0, false>;  // A^-1 R
  RSM_LAUNCH(k_eig_prep<T>, (total(P.pad2) / 4 + 255) / 256, 256, D, dev(P.pad2), np, shift_rel, a_iters);
  // The factor, its inverse and T = A^-1 in one launch (see k_factor).  The
  // attribute is set on every call (it is per device); the CTA count of a full
  // wave is cached per device (worker threads may race to fill it with the same value).
  const int factor_smem = kFactorTiles * BS * (BS + 1) * (int)sizeof(T);
  int dev_id = 0;
  cudaError_t eo = cudaFuncSetAttribute(k_factor<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, factor_smem);
  if (eo == cudaSuccess) eo = cudaGetDevice(&dev_id);
  if (eo != cudaSuccess) return eo;
  static std::atomic<int> factor_ctas[2][kMaxDevices];
  const int slot_id = dev_id < kMaxDevices ? dev_id : kMaxDevices - 1;
  int fc = factor_ctas[sizeof(T) == 8][slot_id].load(std::memory_order_relaxed);
  if (fc == 0) {
    int sms = 0, per_sm = 0;
    eo = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    if (eo == cudaSuccess) eo = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_factor<T>, 256, factor_smem);
    if (eo != cudaSuccess) return eo;
    fc = std::max(2, sms * per_sm);
    factor_ctas[sizeof(T) == 8][slot_id].store(fc, std::memory_order_relaxed);
  }
  // one chain per problem while they take at most half the CTAs (so that at
  // least as many CTAs serve the other tasks), else problems share chains
  const int nchain = std::min(np, std::max(1, fc / 2));
  FactorTables ft{P.step, P.linv, P.phase, P.max_nblk, kFactorLag, P.fault_wait ? kDepPollsInjected : kDepPolls,
                  P.fault_wait ? 1 : 0};
  const int64_t ntask = nchain + P.hT[P.phase + 5 * P.max_nblk + 3 * kFactorLag];
  RSM_LAUNCH_SMEM(k_factor<T>, std::min<int64_t>(ntask, fc), 256, factor_smem, D, P.dT, np, ft, P.sync, nchain);
  RSM_LAUNCH(k_init_X, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
  auto orthonormalise = [&]() -> cudaError_t {
    RSM_LAUNCH_SMEM(xtx_s, total(P.chunk), kXtxThreads, xtx_smem, D, dev(P.chunk), np, P.part, dev(P.part_off));
    RSM_LAUNCH(orth, np, kSmallThreads, D, np, part, dev(P.part_off));
    RSM_LAUNCH(rot_x, total(P.rot), 256, D, dev(P.rot), np);
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
  // FP32-pair products with M and a Rayleigh-Ritz step each time; every step
  // ends with a convergence check, and a converged problem skips everything
  // after it (a predicted stop after the correction of that step).  With the
  // FP64 factor a step can again collapse the block, so X is re-orthonormalised
  // before each product.
  for (int it = 0; it <= iters; ++it) {
    if (sizeof(T) == 8 && it > 0)
      if ((e = orthonormalise()) != cudaSuccess) return e;
    if (P.kx_max <= 12)
      RSM_LAUNCH(k_gemm_MX<12>, total(P.mx), kMxRows, D, dev(P.mx), np);
    else if (P.kx_max <= 16)
      RSM_LAUNCH(k_gemm_MX<16>, total(P.mx), kMxRows, D, dev(P.mx), np);
    else
      RSM_LAUNCH(k_gemm_MX<32>, total(P.mx), kMxRows, D, dev(P.mx), np);
    RSM_LAUNCH_SMEM(xtx_h, total(P.chunk), kXtxThreads, xtx_smem, D, dev(P.chunk), np, P.part, dev(P.part_off));
    RSM_LAUNCH_SMEM(rr, np, kRRThreads, kRRSmem, D, np, part, dev(P.part_off));
    RSM_LAUNCH(rot_check, total(P.rot), 256, D, dev(P.rot), np);
    RSM_LAUNCH(precond_r, total(P.row_tile), 256, D, dev(P.row_tile), np);
    RSM_LAUNCH(k_precond_apply<0>, (total(P.nk) + 255) / 256, 256, D, dev(P.nk), np);
  }
  // FP64 refinement.  The iteration above carries M X in FP32 pairs (about
  // 2^-44 relative), which bounds its residual at ~2^-44 ||M||.  Then passes
  // with M X in IEEE FP64, ending in a Rayleigh-Ritz step whose residual (also
  // FP64) is the one reported and tested on the host.  With the FP32 factor one
  // pass: the block iteration's last correction (a predicted stop) already
  // brings the block to the FP32-pair floor, which the FP64 residual then
  // certifies.  With the FP64 factor two: the first gives the FP64 residual R
  // of the Ritz vectors and the correction X <- X - A^-1 R, the second the
  // Rayleigh-Ritz step on the re-orthonormalised, corrected block.
  RSM_LAUNCH(k_refine_begin, (np + 127) / 128, 128, D, np);
  const int passes = sizeof(T) == 8 ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    if (sizeof(T) == 8 && pass > 0)
      if ((e = orthonormalise()) != cudaSuccess) return e;
    if (P.kx_max <= 12)
      RSM_LAUNCH(k_gemm_MX64<12>, total(P.mx), kMxRows, D, dev(P.mx), np);
    else if (P.kx_max <= 16)
      RSM_LAUNCH(k_gemm_MX64<16>, total(P.mx), kMxRows, D, dev(P.mx), np);
    else
      RSM_LAUNCH(k_gemm_MX64<32>, total(P.mx), kMxRows, D, dev(P.mx), np);
    RSM_LAUNCH_SMEM(xtx_h, total(P.chunk), kXtxThreads, xtx_smem, D, dev(P.chunk), np, P.part, dev(P.part_off));
    RSM_LAUNCH_SMEM(rr, np, kRRThreads, kRRSmem, D, np, part, dev(P.part_off));
    RSM_LAUNCH(rot_full, total(P.rot), 256, D, dev(P.rot), np);
    if (pass + 1 < passes) {
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
