// Small dense algebra of the Rayleigh-Ritz step and of the minor vectors on
// the FP32 pipes.
//
// FP64 instructions issue at a small fraction of the FP32 rate on this part,
// and the Rayleigh-Ritz step of the eigen stage is a chain of kx x kx
// operations on one SM, so its latency is what counts.  Here:
//   * products of kx x kx matrices run in FP32-pair ("double-float")
//     arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2 (48 significant
//     bits); a product term is split exactly by FMA (TwoProduct) and the sum
//     is carried by TwoSum (Knuth), as in Dekker's double-length arithmetic;
//   * the Cholesky factorisation, its inverse and the Jacobi eigensolver are
//     FP32, one warp (or half warp), one matrix row per lane held in
//     registers: the FP32 results only seed steps that are then completed in
//     FP32 pairs or FP64 (a Newton-Schulz step for the factor, Lowdin steps and
//     a first-order decoupling for the eigenvectors, Newton refinement of the
//     minor vectors).
// The Jacobi sweep uses the round-robin ordering of the circle method with a
// fixed permutation after every round, so that the rotated pairs are always
// positions (2k, 2k + 1) and every register index is a compile-time constant.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace rsm {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ DF df_norm(float s, float e) {
  DF r;
  df_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ DF df_from(double x) {
  const float h = __double2float_rn(x);
  return DF{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

// Running sum of FP32-pair terms: the head by TwoSum, the tails added plainly.
struct DFAcc {
  float sh = 0.f, sl = 0.f;
  __device__ __forceinline__ void add_prod(DF a, DF b) {
    const float ph = __fmul_rn(a.hi, b.hi);
    const float pe = __fmaf_rn(a.hi, b.hi, -ph);
    const float cross = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    float s, er;
    df_two_sum(sh, ph, s, er);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(er, __fadd_rn(pe, cross)));
  }
  __device__ __forceinline__ void add(DF a) {
    float s, er;
    df_two_sum(sh, a.hi, s, er);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(er, a.lo));
  }
  __device__ __forceinline__ DF get() const { return df_norm(sh, sl); }
};

constexpr int kDfLs = 33;  // row stride (kx <= 32)
typedef DF DFRow[kDfLs];

// C = op(A) B, kx x kx, all `nthreads` threads of the CTA (no barrier inside).
__device__ inline void df_prod(DFRow* C, const DFRow* A, bool transA, const DFRow* B, int kx, int nthreads) {
  const SmallDiv dkx((uint32_t)kx);
  for (int e = threadIdx.x; e < kx * kx; e += nthreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    DFAcc acc;
    for (int t = 0; t < kx; ++t) acc.add_prod(transA ? A[t][a] : A[a][t], B[t][b]);
    C[a][b] = acc.get();
  }
}

// out = Q^T A Q for symmetric A (the lower triangle is computed and mirrored); W: work.
__device__ inline void df_congruence(DFRow* out, const DFRow* Q, const DFRow* A, DFRow* W, int kx, int nthreads) {
  df_prod(W, A, false, Q, kx, nthreads);
  __syncthreads();
  const SmallDiv dkx((uint32_t)kx);
  for (int e = threadIdx.x; e < kx * kx; e += nthreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    if (b > a) continue;
    DFAcc acc;
    for (int t = 0; t < kx; ++t) acc.add_prod(Q[t][a], W[t][b]);
    const DF v = acc.get();
    out[a][b] = v;
    out[b][a] = v;
  }
  __syncthreads();
}

// W1 = (3I - Z) / 2 in pairs (the Newton-Schulz / Lowdin factor).
__device__ inline void df_three_minus_half(DFRow* W1, const DFRow* Z, int kx, int nthreads) {
  const SmallDiv dkx((uint32_t)kx);
  for (int e = threadIdx.x; e < kx * kx; e += nthreads) {
    const int a = dkx.q(e), b = dkx.r(e);
    const DF z = Z[a][b];
    DF v = df_norm(-z.hi, -z.lo);
    if (a == b) v = df_norm(__fadd_rn(3.f, v.hi), v.lo);
    W1[a][b] = DF{0.5f * v.hi, 0.5f * v.lo};
  }
}

// Q <- Q (3I - Q^T Q) / 2 (Lowdin / Newton-Schulz orthogonalisation step: the
// departure from orthogonality is squared).  W1, W2: work.
__device__ inline void df_lowdin(DFRow* Q, DFRow* W1, DFRow* W2, int kx, int nthreads) {
  df_prod(W2, Q, true, Q, kx, nthreads);
  __syncthreads();
  df_three_minus_half(W1, W2, kx, nthreads);
  __syncthreads();
  df_prod(W2, Q, false, W1, kx, nthreads);
  __syncthreads();
  const SmallDiv dkx((uint32_t)kx);
  for (int e = threadIdx.x; e < kx * kx; e += nthreads) Q[dkx.q(e)][dkx.r(e)] = W2[dkx.q(e)][dkx.r(e)];
  __syncthreads();
}

// ------------------------------------------------------------------ one-warp register algebra (FP32)
// Lane i < KP holds row i of a KP x KP matrix in a[0 .. KP).

// a[idx] for a runtime idx without dynamic register indexing.
template <typename T, int KP>
__device__ __forceinline__ T reg_pick(const T (&a)[KP], int idx) {
  T v = 0;
#pragma unroll
  for (int j = 0; j < KP; ++j) v = (j == idx) ? a[j] : v;
  return v;
}
template <int KP>
__device__ __forceinline__ float reg_pick(const float (&a)[KP], int idx) {
  return reg_pick<float, KP>(a, idx);
}

// In place: a (symmetric, rows per lane, the shift s * trace of its leading
// n x n block added to the diagonal first) -> its lower Cholesky factor C (row
// i of C in lane i, entries above the diagonal left as they were); rdiag =
// 1 / C_ii of this lane.  Pivots below 1e-30 are replaced by 1e-30 (a
// rank-deficient block stays finite).  The whole warp calls it.
template <int KP>
__device__ __forceinline__ void reg_cholesky(float (&a)[KP], float& rdiag, float shift, int n) {
  const int lane = threadIdx.x & 31;
  float tr = lane < n ? reg_pick<KP>(a, lane) : 0.f;
#pragma unroll
  for (int o = 16; o; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
#pragma unroll
  for (int j = 0; j < KP; ++j)
    if (j == lane) a[j] += shift * tr;
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    const float djj = __shfl_sync(0xffffffffu, a[j], j);
    const float l = djj > 1e-30f ? sqrtf(djj) : 1e-30f;
    const float rl = __frcp_rn(l);
    if (lane == j) {
      a[j] = l;
      rdiag = rl;
    } else if (lane > j) {
      a[j] *= rl;
    }
#pragma unroll
    for (int c = j + 1; c < KP; ++c) {
      const float lcj = __shfl_sync(0xffffffffu, a[j], c);
      if (lane > j) a[c] = __fmaf_rn(-a[j], lcj, a[c]);
    }
  }
}

// y = row `lane` of C^-1 for the lower factor C of reg_cholesky (forward
// substitution, the rows of C^-1 broadcast one after the other).
template <int KP>
__device__ __forceinline__ void reg_tri_inverse(const float (&a)[KP], float rdiag, float (&y)[KP]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < KP; ++c) y[c] = (c == lane) ? 1.f : 0.f;
#pragma unroll
  for (int t = 0; t < KP; ++t) {
    if (lane == t) {
#pragma unroll
      for (int c = 0; c <= t; ++c) y[c] *= rdiag;
    }
#pragma unroll
    for (int c = 0; c <= t; ++c) {
      const float yt = __shfl_sync(0xffffffffu, y[c], t);
      if (lane > t) y[c] = __fmaf_rn(-a[t], yt, y[c]);
    }
  }
}

// Position the player at position x moves to after a round of the circle
// method with pairs (2k, 2k + 1): position 0 stays, the others turn on one cycle
// 1 -> 2 -> 4 -> ... -> KP - 2 -> KP - 1 -> KP - 3 -> ... -> 3 -> 1.
template <int KP>
__host__ __device__ constexpr int circle_next(int x) {
  return x == 0 ? 0 : (x == 1 ? (KP > 2 ? 2 : 1) : ((x & 1) == 0 ? (x + 2 < KP ? x + 2 : x + 1) : x - 2));
}
// ... and the position whose player moves to y.
template <int KP>
__host__ __device__ constexpr int circle_prev(int y) {
  return y == 0 ? 0 : (y == 2 ? 1 : ((y & 1) == 0 ? y - 2 : (y + 2 < KP ? y + 2 : (KP > 2 ? KP - 2 : 1))));
}

// Cyclic Jacobi (symmetric Schur decomposition, Golub & Van Loan Sec. 8.5) of
// the symmetric matrix in a (row `lane`), eigenvectors accumulated into v (row
// `lane` of V, starting from I): a rotation in plane (p, q) annihilates a_pq
// with tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1 / sqrt(1 + t^2), s = t c.  A rotation is skipped when |a_pq| <= tol or
// a_pq^2 <= eps^2 |a_pp a_qq|; the sweeps stop after one that skipped them all.
// The KP - 1 rounds of a sweep rotate the pairs at positions (2k, 2k + 1), then
// move the players by the circle permutation (rows by shuffles, columns by
// register moves); after a whole sweep every player is back at its position.
// Rows and columns of padding (index >= the true size) must be zero off the
// diagonal: their pairs are never rotated.  W = 32: the whole warp holds one
// matrix; W = 16: each half warp holds its own (lane = lane within the half),
// and the halves sweep independently.  T = float (hardware reciprocal and
// square roots) or double (the Newton-Raphson forms of common.cuh).  Returns the
// sweeps that rotated.
template <typename T>
__device__ __forceinline__ T jac_rcp(T x);
template <>
__device__ __forceinline__ float jac_rcp<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double jac_rcp<double>(double x) { return rcp64(x); }
template <typename T>
__device__ __forceinline__ T jac_sqrt(T x);
template <>
__device__ __forceinline__ float jac_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double jac_sqrt<double>(double x) { return sqrt64(x); }
template <typename T>
__device__ __forceinline__ T jac_rsqrt(T x);
template <>
__device__ __forceinline__ float jac_rsqrt<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double jac_rsqrt<double>(double x) { return rsqrt64(x); }

template <typename T, int KP, int W = 32>
__device__ __forceinline__ int reg_jacobi_t(T (&a)[KP], T (&v)[KP], T tol, int max_sweeps) {
  static_assert(KP % 2 == 0 && KP >= 2 && KP <= W && (W == 16 || W == 32), "KP: even, 2..W");
  const int wl = threadIdx.x & 31;
  const int lane = wl & (W - 1), base = wl - lane;
  const unsigned mask = W == 32 ? 0xffffffffu : (0xffffu << base);
  const T eps = sizeof(T) == 4 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
  const T eps2 = eps * eps;
  const int src = base + (lane < KP ? circle_prev<KP>(lane) : lane);
  int rotated = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    for (int round = 0; round < KP - 1; ++round) {
      const bool even = (lane & 1) == 0;
      const T own = reg_pick<T, KP>(a, lane);
      const T off = reg_pick<T, KP>(a, lane ^ 1);
      const T other = __shfl_xor_sync(mask, own, 1);
      const T apq = __shfl_sync(mask, off, wl & ~1);  // the even lane's a_pq for both
      const T app = even ? own : other, aqq = even ? other : own;
      T c = 1, s = 0;
      if (lane < KP && fabs(apq) > tol && apq * apq > eps2 * fabs(app * aqq)) {
        const T tau = (aqq - app) * jac_rcp<T>(2 * apq);
        const T t = (tau >= 0 ? (T)1 : (T)-1) * jac_rcp<T>(fabs(tau) + jac_sqrt<T>(1 + tau * tau));
        c = jac_rsqrt<T>(1 + t * t);
        s = t * c;
      }
      const bool rot = s != (T)0;
      any |= __any_sync(mask, rot);
      // columns: every pair (2k, 2k + 1) with the rotation of lane 2k
#pragma unroll
      for (int k = 0; k < KP / 2; ++k) {
        const T ck = __shfl_sync(mask, c, base + 2 * k), sk = __shfl_sync(mask, s, base + 2 * k);
        const T x = a[2 * k], y = a[2 * k + 1];
        a[2 * k] = ck * x - sk * y;
        a[2 * k + 1] = sk * x + ck * y;
        const T vx = v[2 * k], vy = v[2 * k + 1];
        v[2 * k] = ck * vx - sk * vy;
        v[2 * k + 1] = sk * vx + ck * vy;
      }
      // rows: this lane's row with its partner's
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        const T o = __shfl_xor_sync(mask, a[j], 1);
        a[j] = even ? (c * a[j] - s * o) : (s * o + c * a[j]);
      }
      if (rot) {  // the annihilated entry, exactly
#pragma unroll
        for (int j = 0; j < KP; ++j)
          if (j == (lane ^ 1)) a[j] = 0;
      }
      // the circle permutation: rows from lane circle_prev(lane), columns (of a and v) by moves
#pragma unroll
      for (int j = 0; j < KP; ++j) a[j] = __shfl_sync(mask, a[j], src);
      T ta[KP], tv[KP];
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        ta[circle_next<KP>(j)] = a[j];
        tv[circle_next<KP>(j)] = v[j];
      }
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        a[j] = ta[j];
        v[j] = tv[j];
      }
    }
    if (!any) break;
    ++rotated;
  }
  return rotated;
}

template <int KP, int W = 32>
__device__ __forceinline__ int reg_jacobi(float (&a)[KP], float (&v)[KP], float tol, int max_sweeps) {
  return reg_jacobi_t<float, KP, W>(a, v, tol, max_sweeps);
}

}  // namespace rsm
