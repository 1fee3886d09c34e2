// One-warp cyclic Jacobi eigensolver for a small symmetric matrix in shared
// memory.  Textbook two-sided Jacobi (symmetric Schur decomposition, Golub &
// Van Loan, "Matrix Computations", Sec. 8.5): a rotation in plane (p, q) with
// tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c annihilates a_pq.  The parallel round-robin
// ordering applies the k/2 disjoint rotations of a round together.
//
// A rotation is skipped when |a_pq| <= tol_abs or |a_pq| <= eps sqrt(|a_pp a_qq|);
// the sweeps stop when a whole sweep skips every rotation.  tol_abs is a few
// units of rounding of ||A||_F: below it the off-diagonal entries are rounding
// noise, and rotating on them only creates new noise of the same size.
#pragma once

#include <cfloat>

#include "common.cuh"

namespace rsm {

template <typename T>
struct JacobiScratchT {
  int p[16], q[16];
  T c[16], s[16];
};
using JacobiScratch = JacobiScratchT<double>;

template <typename T>
__device__ __forceinline__ T jacobi_eps();
template <>
__device__ __forceinline__ double jacobi_eps<double>() { return DBL_EPSILON; }
template <>
__device__ __forceinline__ float jacobi_eps<float>() { return FLT_EPSILON; }

// Below this |u| = |a_pq / (a_qq - a_pp)| the series rotation is exact to rounding.
template <typename T>
__device__ __forceinline__ T small_rot();
template <>
__device__ __forceinline__ double small_rot<double>() { return 1e-4; }
template <>
__device__ __forceinline__ float small_rot<float>() { return 1e-2f; }

// ||A||_F of a k x k matrix in shared memory (row stride ls), all lanes get it.
template <typename T>
__device__ inline T warp_frobenius(const T* A, int k, int ls) {
  const int lane = threadIdx.x & 31;
  T s = 0;
  for (int i = lane; i < k * k; i += 32) {
    const T v = A[(i / k) * ls + (i % k)];
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return fast_sqrt(s);
}

// S: k x k symmetric (row stride ls), overwritten by its eigenvalues on the
// diagonal; Vm: k x k (row stride ls) receives the eigenvectors as columns
// (Vm is set to I first unless keep_v).  k <= 32.  All 32 lanes must call it.
// Returns the number of sweeps that applied at least one rotation (0: S was
// already diagonal to the tolerance and Vm is the identity / unchanged).
// Lane r < ceil(k/2) computes the rotation of pair r of the round; the other
// lanes fetch it by shuffle, so the updates read no indices from memory.
template <typename T>
__device__ inline int warp_jacobi(T* S, T* Vm, int k, int ls, JacobiScratchT<T>& /*unused*/, T tol_abs,
                                  int max_sweeps = 40, bool keep_v = false) {
  const int lane = threadIdx.x & 31;
  if (!keep_v)
    for (int i = lane; i < k * k; i += 32) {
      const int a = i / k, b = i % k;
      Vm[a * ls + b] = (a == b) ? (T)1 : (T)0;
    }
  __syncwarp();
  const T eps = jacobi_eps<T>();
  const int ne = (k + 1) & ~1;
  const int np = ne / 2;
  const int nitem = np * k;  // (pair, row) items of one round
  // this lane's items it = lane + 32 m as (pair, row), computed once (no division in the rounds)
  constexpr int kMaxItems = (16 * 32 + 31) / 32;
  int it_r[kMaxItems], it_i[kMaxItems];
  {
    const SmallDiv dk((uint32_t)k);
#pragma unroll
    for (int m = 0; m < kMaxItems; ++m) {
      uint32_t q, rr;
      dk.divmod((uint32_t)(lane + 32 * m), q, rr);
      it_r[m] = (int)q;
      it_i[m] = (int)rr;
    }
  }
  int rotated = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    for (int round = 0; round < ne - 1; ++round) {
      int a = 0, b = 0;
      T c = 1, s = 0;
      if (lane < np) {
        const int s0 = lane, s1 = ne - 1 - lane;
        int pa = s0 - 1 + round, pb = s1 - 1 + round;  // positions on the ring of ne - 1
        if (pa >= ne - 1) pa -= ne - 1;
        if (pb >= ne - 1) pb -= ne - 1;
        a = (s0 == 0) ? 0 : pa + 1;
        b = (s1 == 0) ? 0 : pb + 1;
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        if (b < k) {
          const T apq = S[a * ls + b];
          const T app = S[a * ls + a], aqq = S[b * ls + b];
          if (fabs(apq) > tol_abs && apq * apq > eps * eps * fabs(app * aqq)) {
            // u = a_pq / (a_qq - a_pp) = 1 / (2 tau).  When |u| is small, t = u (1 - u^2)
            // and c = 1 - t^2 / 2 are exact to O(u^4) (series of the textbook formulas),
            // which saves the square roots; otherwise use the textbook formulas.
            const T den = aqq - app;
            const T u = (fabs(den) > (T)0) ? apq * fast_rcp(den) : (T)1;
            if (fabs(u) < small_rot<T>()) {
              const T tt = u * (1 - u * u);
              c = 1 - (T)0.5 * tt * tt;
              s = tt * c;
            } else {
              const T tau = den * fast_rcp(2 * apq);
              const T tt = (tau >= 0 ? (T)1 : (T)-1) * fast_rcp(fabs(tau) + fast_sqrt(1 + tau * tau));
              c = fast_rsqrt(1 + tt * tt);
              s = tt * c;
            }
          }
        } else {
          b = a;
        }
      }
      if (!__any_sync(0xffffffffu, s != (T)0)) continue;
      any = true;
      __syncwarp();
      // columns p, q of S and Vm
#pragma unroll
      for (int m = 0; m < kMaxItems; ++m) {
        if (32 * m >= nitem) break;
        const int it = 32 * m + lane;
        const int r = it < nitem ? it_r[m] : 0, i = it < nitem ? it_i[m] : 0;
        const int pr = __shfl_sync(0xffffffffu, a, r), qr = __shfl_sync(0xffffffffu, b, r);
        const T cr = __shfl_sync(0xffffffffu, c, r), sr = __shfl_sync(0xffffffffu, s, r);
        if (it < nitem && sr != (T)0) {
          const T xp = S[i * ls + pr], xq = S[i * ls + qr];
          const T vp = Vm[i * ls + pr], vq = Vm[i * ls + qr];
          S[i * ls + pr] = cr * xp - sr * xq;
          S[i * ls + qr] = sr * xp + cr * xq;
          Vm[i * ls + pr] = cr * vp - sr * vq;
          Vm[i * ls + qr] = sr * vp + cr * vq;
        }
      }
      __syncwarp();
      // rows p, q of S
#pragma unroll
      for (int m = 0; m < kMaxItems; ++m) {
        if (32 * m >= nitem) break;
        const int it = 32 * m + lane;
        const int r = it < nitem ? it_r[m] : 0, j = it < nitem ? it_i[m] : 0;
        const int pr = __shfl_sync(0xffffffffu, a, r), qr = __shfl_sync(0xffffffffu, b, r);
        const T cr = __shfl_sync(0xffffffffu, c, r), sr = __shfl_sync(0xffffffffu, s, r);
        if (it < nitem && sr != (T)0) {
          const T xp = S[pr * ls + j], xq = S[qr * ls + j];
          S[pr * ls + j] = cr * xp - sr * xq;
          S[qr * ls + j] = sr * xp + cr * xq;
        }
      }
      __syncwarp();
      if (lane < np && s != (T)0) {
        S[a * ls + b] = 0;
        S[b * ls + a] = 0;
      }
      __syncwarp();
    }
    if (!any) break;
    ++rotated;
  }
  return rotated;
}

// Eigendecomposition of a k x k symmetric FP64 matrix (k <= 32) in two
// precisions: Jacobi in FP32 on a rounded copy gives Q32 that nearly
// diagonalises A; Q32 is made orthogonal in FP64 (Lowdin steps), B = Q^T A Q is
// formed in FP64 and polished by FP64 Jacobi sweeps (quadratic convergence from
// ~1e-7 off-diagonals), and the eigenvectors are Q * Q64.  The FP64 work is a
// few sweeps instead of a full solve.
// A (k x k, stride ls, FP64) is overwritten: eigenvalues on its diagonal.
// Vd (k x k, stride ls, FP64) receives the eigenvectors.  Work areas: Sf, Vf
// (FP32, stride ls), Td (FP64, stride ls).
__device__ inline void warp_eig_mixed(double* A, double* Vd, float* Sf, float* Vf, double* Td, int k, int ls,
                                      JacobiScratchT<float>& jsf, JacobiScratchT<double>& jsd) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < k * k; i += 32) Sf[(i / k) * ls + (i % k)] = (float)A[(i / k) * ls + (i % k)];
  __syncwarp();
  const double fro = warp_frobenius(A, k, ls);
  warp_jacobi<float>(Sf, Vf, k, ls, jsf, (float)(4.0 * FLT_EPSILON * fro));
  // Q = Q32 made orthogonal to FP64 accuracy by two Lowdin steps, Q <- Q (3I - Q^T Q) / 2
  // (Q32 is orthogonal only to FP32 accuracy).  Q lives in Vd.
  for (int i = lane; i < k * k; i += 32) Vd[(i / k) * ls + (i % k)] = (double)Vf[(i / k) * ls + (i % k)];
  __syncwarp();
  for (int step = 0; step < 2; ++step) {
    for (int i = lane; i < k * k; i += 32) {  // Td = Q^T Q
      const int a = i / k, b = i % k;
      double s = 0.0;
      for (int t = 0; t < k; ++t) s = fma(Vd[t * ls + a], Vd[t * ls + b], s);
      Td[a * ls + b] = s;
    }
    __syncwarp();
    double out[32];
    int cnt = 0;
    for (int i = lane; i < k * k; i += 32) {  // Q (3I - Td) / 2
      const int a = i / k, b = i % k;
      double s = 0.0;
      for (int t = 0; t < k; ++t) s = fma(Vd[a * ls + t], ((t == b) ? 3.0 : 0.0) - Td[t * ls + b], s);
      out[cnt++] = 0.5 * s;
    }
    __syncwarp();
    cnt = 0;
    for (int i = lane; i < k * k; i += 32) Vd[(i / k) * ls + (i % k)] = out[cnt++];
    __syncwarp();
  }
  // Td = A * Q
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i % k;
    double s = 0.0;
    for (int t = 0; t < k; ++t) s = fma(A[a * ls + t], Vd[t * ls + b], s);
    Td[a * ls + b] = s;
  }
  __syncwarp();
  // B = Q^T Td (symmetrised; upper triangle mirrored), the nearly diagonal matrix to polish
  double bv[32];
  int nb = 0;
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i % k;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    double s = 0.0;
    for (int t = 0; t < k; ++t) s = fma(Vd[t * ls + lo], Td[t * ls + hi], s);
    bv[nb++] = s;
  }
  __syncwarp();
  nb = 0;
  for (int i = lane; i < k * k; i += 32) A[(i / k) * ls + (i % k)] = bv[nb++];
  __syncwarp();
  warp_jacobi<double>(A, Td, k, ls, jsd, 4.0 * DBL_EPSILON * fro, 4);
  // eigenvectors Q * Q64 (computed into registers, then stored in Vd)
  nb = 0;
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i % k;
    double s = 0.0;
    for (int t = 0; t < k; ++t) s = fma(Vd[a * ls + t], Td[t * ls + b], s);
    bv[nb++] = s;
  }
  __syncwarp();
  nb = 0;
  for (int i = lane; i < k * k; i += 32) Vd[(i / k) * ls + (i % k)] = bv[nb++];
  __syncwarp();
}

}  // namespace rsm
