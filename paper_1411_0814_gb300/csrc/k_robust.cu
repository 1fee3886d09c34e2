// The L1 forms of V-hat and U-hat (Section IV-A: eq. solve.barV_L1_norm "with
// the regularization constraints", and eq. solve.barU with the L1 norm), by
// iteratively reweighted least squares from the L2 solution.
//
// V-hat: minimise sum_j ||V^T xi_j||_2 over the null vectors (the 1-norm over
// the vectors of their Euclidean residuals, which does not depend on the basis
// of V-hat), subject to V^T V = I.  A step takes the weights
// w_j = delta / max(||V^T xi_j||, delta) <= 1 from the current V, builds
// M_w = sum_j w_j xi_j xi_j^T in the same fixed-point accumulator as M
// (k_l1_scatter, from the minor vectors each trial stored), and takes its r
// smallest eigenvectors with the eigen stage.
//
// U-hat: per row, minimise sum_{j in K_i} |y_ij - u_i . v_j|: a step takes the
// weights w = delta / max(|r_ij|, delta) (delta = delta_u times the RMS residual
// e of the L2 solution), accumulates N = sum w v v^T and b = sum w y v, and
// solves N u = b by Cholesky in FP64 (k_irls_u).  One thread per row, which
// holds the r(r+1)/2 + r sums in registers: r <= 8.
#include "common.cuh"
#include "kernels.h"

namespace rsm {

constexpr int kL1Warps = 4;

// M_w into the fixed-point accumulator (zeroed by the host), one warp per trial.
__global__ void __launch_bounds__(32 * kL1Warps) k_l1_scatter(const ProbDesc* __restrict__ descs,
                                                             const int64_t* __restrict__ trial_off, int nprob) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kL1Warps + wid;
  if (g >= trial_off[nprob]) return;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  if (!d.Zst) return;
  const int64_t t = g - trial_off[p];
  const int l = d.l, nm = d.n_minor, r = d.r;
  if (d.row_counts[t] < l) return;  // rejected trial
  const int32_t* C = d.cols + t * l;
  const double* Z = d.Zst + t * l * nm;
  double w[kMaxL];
  for (int j = 0; j < nm; ++j) {
    // ||V[C]^T z_j||: lane a < r takes column a of V
    double s = 0.0;
    if (lane < r)
      for (int b = 0; b < l; ++b) s = fma(d.V[(int64_t)lane * d.ldv + C[b]], Z[b * nm + j], s);
    double s2 = s * s;
#pragma unroll
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const double res = sqrt(s2);
    w[j] = d.delta_v / (res > d.delta_v ? res : d.delta_v);
  }
  const int f = macc_frac_bits(d.counters[2]);
  const double scale = ldexp(1.0, f);
  for (int it = lane; it < l * l; it += 32) {
    const int a = it / l, b = it - a * l;
    double pr = 0.0;
    for (int j = 0; j < nm; ++j) pr = fma(w[j] * Z[a * nm + j], Z[b * nm + j], pr);
    const long long v = llrint(pr * scale);
    if (v) atomicAdd(&d.macc[(uint32_t)C[a] * (uint32_t)d.n + (uint32_t)C[b]], (unsigned long long)v);
  }
}

// One IRLS step of the L1 rows.  T: accumulation type of N and b (FP32 in the
// FP32 form, FP64 in the FP64 form); the r x r solve is FP64.  Rows with fewer
// than r known entries (the minimum-norm rows) keep their solution.
constexpr int kIrlsRows = 128;
constexpr int kIrlsCols = 32;
template <typename T, int RM>
__global__ void __launch_bounds__(kIrlsRows) k_irls_u(const ProbDesc* __restrict__ descs,
                                                     const int64_t* __restrict__ row_off, int nprob) {
  __shared__ T vs[kIrlsCols][RM + 1];
  // row_off holds each problem's m rounded up to kIrlsRows, so a block belongs to one problem
  const int p = find_problem(row_off, nprob, (int64_t)blockIdx.x * kIrlsRows);
  const ProbDesc& d = descs[p];
  const int64_t i = (int64_t)blockIdx.x * kIrlsRows - row_off[p] + threadIdx.x;
  const bool in = i < d.m;
  const int r = d.r;
  constexpr int P = RM * (RM + 1) / 2;
  double u[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) u[a] = (in && a < r) ? d.U[(int64_t)a * d.ldu + i] : 0.0;
  T uf[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) uf[a] = (T)u[a];
  T N[P], bb[RM];
#pragma unroll
  for (int q = 0; q < P; ++q) N[q] = (T)0;
#pragma unroll
  for (int a = 0; a < RM; ++a) bb[a] = (T)0;
  const T delta = (T)(d.delta_u * d.stats[33]);
  const T dl = delta > (T)0 ? delta : (T)1e-300;
  int known = 0;
  const uint32_t ldy = (uint32_t)d.ldy, ldb = (uint32_t)d.ldb;
  const uint32_t irow = (uint32_t)(in ? i : 0);
  for (int64_t j0 = 0; j0 < d.n; j0 += kIrlsCols) {
    __syncthreads();
    for (int e = threadIdx.x; e < kIrlsCols * RM; e += kIrlsRows) {
      const int jj = e / RM, a = e % RM;
      const int64_t j = j0 + jj;
      vs[jj][a] = (j < d.n && a < r) ? (T)d.V[(int64_t)a * d.ldv + j] : (T)0;
    }
    __syncthreads();
    const int jn = d.n - j0 < kIrlsCols ? (int)(d.n - j0) : kIrlsCols;
    if (in)
      for (int jj = 0; jj < jn; ++jj) {
        const uint32_t j = (uint32_t)(j0 + jj);
        if (!((__ldg(d.bits + (j * ldb + (irow >> 5))) >> (irow & 31)) & 1u)) continue;
        ++known;
        const T y = d.y_dtype == 0 ? (T)__ldg(static_cast<const double*>(d.Y) + (j * ldy + irow))
                                   : (T)__ldg(static_cast<const float*>(d.Y) + (j * ldy + irow));
        T pred = (T)0;
#pragma unroll
        for (int a = 0; a < RM; ++a) pred = fma(uf[a], vs[jj][a], pred);
        const T res = y - pred;
        const T ar = res < (T)0 ? -res : res;
        const T w = dl / (ar > dl ? ar : dl);
#pragma unroll
        for (int a = 0; a < RM; ++a) {
          const T wv = w * vs[jj][a];
          bb[a] = fma(wv, y, bb[a]);
#pragma unroll
          for (int b2 = a; b2 < RM; ++b2) N[a * RM - a * (a - 1) / 2 + (b2 - a)] = fma(wv, vs[jj][b2], N[a * RM - a * (a - 1) / 2 + (b2 - a)]);
        }
      }
  }
  if (!in || known < r) return;
  // Cholesky of N (r x r, packed upper a <= b) in FP64; on a bad pivot the row keeps its solution
  double L[P];
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < RM; ++a)
#pragma unroll
    for (int b2 = 0; b2 <= a; ++b2) {
      L[a * (a + 1) / 2 + b2] = (a < r && b2 < r) ? (double)N[b2 * RM - b2 * (b2 - 1) / 2 + (a - b2)] : 0.0;
      if (a == b2 && a < r) tr += L[a * (a + 1) / 2 + a];
    }
  double x[RM];
#pragma unroll
  for (int j = 0; j < RM; ++j) {
    if (j >= r) break;
    double v = L[j * (j + 1) / 2 + j];
#pragma unroll
    for (int t = 0; t < j; ++t) v = fma(-L[j * (j + 1) / 2 + t], L[j * (j + 1) / 2 + t], v);
    if (!(v > 1e-13 * tr)) return;
    v = sqrt(v);
    L[j * (j + 1) / 2 + j] = v;
#pragma unroll
    for (int k = j + 1; k < RM; ++k) {
      if (k >= r) break;
      double w2 = L[k * (k + 1) / 2 + j];
#pragma unroll
      for (int t = 0; t < j; ++t) w2 = fma(-L[k * (k + 1) / 2 + t], L[j * (j + 1) / 2 + t], w2);
      L[k * (k + 1) / 2 + j] = w2 / v;
    }
  }
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    if (a >= r) break;
    double v = (double)bb[a];
#pragma unroll
    for (int t = 0; t < a; ++t) v = fma(-L[a * (a + 1) / 2 + t], x[t], v);
    x[a] = v / L[a * (a + 1) / 2 + a];
  }
#pragma unroll
  for (int a = RM - 1; a >= 0; --a) {
    if (a >= r) continue;
    double v = x[a];
#pragma unroll
    for (int t = a + 1; t < RM; ++t)
      if (t < r) v = fma(-L[t * (t + 1) / 2 + a], x[t], v);
    x[a] = v / L[a * (a + 1) / 2 + a];
  }
  for (int a = 0; a < r; ++a) d.U[(int64_t)a * d.ldu + i] = x[a];
}

cudaError_t launch_l1_scatter(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total,
                              cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  k_l1_scatter<<<(unsigned)((total + kL1Warps - 1) / kL1Warps), 32 * kL1Warps, 0, s>>>(descs, trial_off, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_irls_u(const ProbDesc* descs, const int64_t* row_off, int nprob, int64_t total, int rmax,
                          bool fp64, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + kIrlsRows - 1) / kIrlsRows);
#define RSM_IRLS(T, RM) k_irls_u<T, RM><<<blocks, kIrlsRows, 0, s>>>(descs, row_off, nprob)
  if (rmax > 8) return cudaErrorNotSupported;  // validated on the host: the L1 forms take r <= 8
  if (fp64) {
    if (rmax <= 4) RSM_IRLS(double, 4); else RSM_IRLS(double, 8);
  } else {
    if (rmax <= 4) RSM_IRLS(float, 4); else RSM_IRLS(float, 8);
  }
#undef RSM_IRLS
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
