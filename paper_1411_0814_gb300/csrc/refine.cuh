// One step of mixed-precision iterative refinement of a row of U-hat (the
// FP32 form of the normal equations, eq. solve.barU), shared by the residual
// kernels.
#pragma once

#include "common.cuh"

namespace rsm {

// The caller has the residual r0 = y_K - V_K u32 of the FP32 copy u32 of u_i and
// c = V_K^T r0 (both in FP32); delta = N_i^-1 c through the row's stored FP32
// Cholesky factor (forward, then back substitution).  u_i becomes u32 + delta
// in FP64, and the row's sum of squared residuals drops by exactly c . delta
// (||r0 - V_K delta||^2 = ||r0||^2 - 2 c.delta + delta^T N delta, N delta = c),
// which is returned.  Rows whose factor is marked -1 (minimum-norm path) are
// left as they are (returns 0).  The FP32 accumulation of N_i and b_i on the
// tensor cores carries errors of about 1e-6 relative, which this step removes
// down to the size of the correction times that.
template <int RM>
__device__ __forceinline__ double refine_row(const ProbDesc& d, uint32_t row, const float (&u32)[RM],
                                             const float (&c)[RM]) {
  const int r = d.r, P = r * (r + 1) / 2;
  const float* __restrict__ lf = d.Lf + (size_t)row * P;
  if (!(lf[0] > 0.f)) return 0.0;
  float y[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) {  // L y = c
    if (a >= r) break;
    float v = c[a];
#pragma unroll
    for (int t = 0; t < a; ++t) v = fmaf(-lf[a * (a + 1) / 2 + t], y[t], v);
    y[a] = v / lf[a * (a + 1) / 2 + a];
  }
#pragma unroll
  for (int a = RM - 1; a >= 0; --a) {  // L^T delta = y
    if (a >= r) continue;
    float v = y[a];
#pragma unroll
    for (int t = a + 1; t < RM; ++t)
      if (t < r) v = fmaf(-lf[t * (t + 1) / 2 + a], y[t], v);
    y[a] = v / lf[a * (a + 1) / 2 + a];
  }
  double drop = 0.0;
#pragma unroll
  for (int a = 0; a < RM; ++a)
    if (a < r) {
      d.U[(int64_t)a * d.ldu + row] = (double)u32[a] + (double)y[a];
      drop += (double)c[a] * (double)y[a];
    }
  return drop;
}

}  // namespace rsm
