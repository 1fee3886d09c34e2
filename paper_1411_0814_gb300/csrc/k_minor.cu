// Stages a5 + a6: minor eigenvectors of each trial's Gram and their exact,
// order-independent accumulation into M.
//
// a5: the right singular vectors of A_t for its l - r smallest singular values
// (Section III) are the eigenvectors of G_t = A_t^T A_t for its smallest
// eigenvalues.  One warp per trial runs the cyclic two-sided Jacobi method in
// FP64 (jacobi.cuh).
//
// a6: M = Xi Xi^T = sum_t sum_j xi xi^T with xi = e(zeta) (eq. get_xi, eq. XI).
// Trial t adds the projector Z_t Z_t^T (l x l) to M[C_t, C_t].  Contributions
// are rounded to 64-bit fixed point (2^-f, f chosen so no sum can overflow)
// and added with integer atomics: integer addition is associative, so the
// result is bit-identical for any order of the trials.
#include <cfloat>

#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace rsm {

constexpr int kMinorWarps = 4;

__global__ void __launch_bounds__(32 * kMinorWarps) k_minor_scatter(const ProbDesc* __restrict__ descs,
                                                                   const int64_t* __restrict__ trial_off, int nprob,
                                                                   int lmax) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kMinorWarps + wid;
  if (g >= trial_off[nprob]) return;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - trial_off[p];
  const int l = d.l;
  const int ls = lmax + 1;  // row stride of the shared matrices
  double* S = sm + (size_t)wid * 2 * lmax * ls;
  double* Vm = S + (size_t)lmax * ls;
  __shared__ JacobiScratch js[kMinorWarps];
  __shared__ int pick[kMinorWarps][kMaxL];

  const int count = d.row_counts[t];
  if (count < l) {  // rejected trial (fewer than l rows, i.e. not more than r)
    if (d.debug_Z)
      for (int i = lane; i < l * d.n_minor; i += 32) d.debug_Z[t * l * d.n_minor + i] = 0.0;
    return;
  }
  if (lane == 0) atomicAdd(&d.counters[0], 1ull);

  // load the packed Gram into a full symmetric matrix, V = I
  const int P = l * (l + 1) / 2;
  const double* G = d.gram + t * P;
  for (int q = lane; q < P; q += 32) {
    int a = 0, rem = q;
    while (rem >= l - a) {
      rem -= l - a;
      ++a;
    }
    const int b = a + rem;
    const double v = G[q];
    S[a * ls + b] = v;
    S[b * ls + a] = v;
  }
  __syncwarp();

  warp_jacobi(S, Vm, l, ls, js[wid]);

  // the n_minor smallest eigenvalues (ties broken by index)
  if (lane == 0) {
    int used[kMaxL];
    for (int i = 0; i < l; ++i) used[i] = 0;
    for (int j = 0; j < d.n_minor; ++j) {
      int best = -1;
      for (int i = 0; i < l; ++i)
        if (!used[i] && (best < 0 || S[i * ls + i] < S[best * ls + best])) best = i;
      used[best] = 1;
      pick[wid][j] = best;
    }
  }
  __syncwarp();
  const int nm = d.n_minor;
  if (d.debug_Z)
    for (int it = lane; it < l * nm; it += 32) {
      const int a = it / nm, j = it % nm;
      d.debug_Z[t * l * nm + it] = Vm[a * ls + pick[wid][j]];
    }

  // scatter Z Z^T into M[C_t, C_t] in fixed point
  const int f = macc_frac_bits(d.counters[2]);
  const double scale = ldexp(1.0, f);
  const int32_t* C = d.cols + t * l;
  for (int it = lane; it < l * l; it += 32) {
    const int a = it / l, b = it % l;
    double pr = 0.0;
    for (int j = 0; j < nm; ++j) pr = fma(Vm[a * ls + pick[wid][j]], Vm[b * ls + pick[wid][j]], pr);
    const long long v = llrint(pr * scale);
    if (v) atomicAdd(&d.macc[(int64_t)C[a] * d.n + C[b]], (unsigned long long)v);
  }
}

// M = macc * 2^-f (two's-complement words read as signed).  Grid over all
// entries of all problems.
__global__ void __launch_bounds__(256) k_finalize_M(const ProbDesc* __restrict__ descs,
                                                  const int64_t* __restrict__ ent_off, int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ent_off[nprob]) return;
  const int p = find_problem(ent_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - ent_off[p];
  const int f = macc_frac_bits(d.counters[2]);
  const double v = ldexp((double)(long long)d.macc[e], -f);
  d.M[e] = v;
  if (d.debug_M) d.debug_M[e] = v;
}

cudaError_t launch_minor_scatter(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total, int lmax,
                                 cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const size_t dyn = sizeof(double) * (size_t)kMinorWarps * 2 * lmax * (lmax + 1);
  cudaError_t e = cudaFuncSetAttribute(k_minor_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  k_minor_scatter<<<(unsigned)((total + kMinorWarps - 1) / kMinorWarps), 32 * kMinorWarps, dyn, s>>>(descs, trial_off,
                                                                                                   nprob, lmax);
  return cudaGetLastError();
}

cudaError_t launch_finalize_M(const ProbDesc* descs, const int64_t* ent_off, int nprob, int64_t total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  k_finalize_M<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(descs, ent_off, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
