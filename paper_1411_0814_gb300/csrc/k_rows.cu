// Method M2 of Section III (the row variant): choose k rows at random, keep the
// columns known in all of them, and take the right singular vectors of the
// k x c_t submatrix A_t = Y[R_t, C_t] beyond its r largest singular values
// (the c_t - k exact null vectors and the k - r of small singular values;
// Section IV-A step 2, "null or small singular values").  Together they span
// the orthogonal complement of Q_t, the top-r right singular vectors, so trial
// t adds I - Q_t Q_t^T to M[C_t, C_t]: the sum of xi xi^T over its vectors
// (eqs. get_xi, XI and the text after eq. solve.barV_L2_norm).
//
//  k_pack_rows:  W -> row-packed bit mask (m rows of ldr words, bit (j mod 32)
//                of word j / 32 of row i is W[i, j] != 0).
//  k_m2_trial:   one warp per trial: C_t = AND of the k row words, c_t, the
//                k x k FP64 Gram A A^T, its eigenpairs (warp Jacobi), and
//                B_t = U_r diag(1 / sigma) (k x r), so that row j of Q_t is
//                B_t^T y_{R_t, c_j}.  A trial is used when c_t > r.
//  k_m2_scatter: one CTA per trial: C_t again, then I - Q Q^T over all pairs
//                of C_t in 64 x 64 blocks (Q rows recomputed from Y and B_t),
//                rounded to the fixed-point accumulator of M like the column
//                variant (integer atomics: the sum is order-independent).
#include <cfloat>

#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"

namespace rsm {

namespace {

constexpr int kRowWarps = 4;   // trials per CTA of k_m2_trial
constexpr int kListCap = 1024; // columns listed per round of 32 words (32 x 32 bits)
constexpr int kQB = 64;        // columns per block of the scatter

__device__ __forceinline__ double load_yd(const ProbDesc& d, uint32_t idx) {
  if (d.y_dtype == 0) return __ldg(static_cast<const double*>(d.Y) + idx);
  return (double)__ldg(static_cast<const float*>(d.Y) + idx);
}

}  // namespace

// Row-packed mask: one thread per (row, word); the warp's 32 threads are 32
// consecutive rows, so each of the 32 column reads is one coalesced segment.
__global__ void __launch_bounds__(256) k_pack_rows(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - off[p];  // over ldr x ceil(m / 32) * 32 (word-major, so a warp shares a word)
  const int64_t mpad = (d.m + 31) / 32 * 32;
  const int64_t w = e / mpad, i = e - w * mpad;
  if (i >= d.m) return;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int64_t j = w * 32 + b;
    if (j < d.n && d.W[j * d.ldw + i]) word |= 1u << b;
  }
  d.rbits[i * d.ldr + w] = word;
}

// Shared memory of one warp of k_m2_trial (kmax rows per trial).
__host__ __device__ inline size_t m2_trial_smem_per_warp(int kmax) {
  const int ks = kmax + 1;
  return sizeof(int) * kListCap + sizeof(double) * (size_t)32 * ks + 2 * sizeof(double) * (size_t)kmax * ks;
}

__global__ void __launch_bounds__(32 * kRowWarps) k_m2_trial(const ProbDesc* __restrict__ descs,
                                                            const int64_t* __restrict__ off, int nprob, int kmax) {
  extern __shared__ __align__(16) unsigned char m2raw[];
  __shared__ JacobiScratchT<double> jsd[kRowWarps];
  __shared__ int order[kRowWarps][kMaxL];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kRowWarps + wid;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - off[p];
  const int k = d.l, r = d.r, ks = kmax + 1;
  unsigned char* base = m2raw + (size_t)wid * m2_trial_smem_per_warp(kmax);
  int* list = reinterpret_cast<int*>(base);
  double* ys = reinterpret_cast<double*>(list + kListCap);  // 32 columns x k values
  double* G = ys + 32 * ks;                                 // k x k Gram, then eigenvalues on its diagonal
  double* U = G + (size_t)kmax * ks;                        // eigenvectors (columns)
  const int32_t* R = d.cols + t * k;
  const uint32_t ldr = (uint32_t)d.ldr, ldy = (uint32_t)d.ldy;
  int rows[kMaxL];
#pragma unroll
  for (int a = 0; a < kMaxL; ++a) rows[a] = a < k ? R[a] : 0;
  auto sel_word = [&](uint32_t w) {
    uint32_t s = 0xffffffffu;
    for (int a = 0; a < k; ++a) s &= __ldg(d.rbits + ((uint32_t)rows[a] * ldr + w));
    return s;
  };
  // c_t: the columns known in every chosen row
  int cnt = 0;
  for (uint32_t w = lane; w < ldr; w += 32) cnt += __popc(sel_word(w));
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
    d.row_counts[t] = cnt;
    if (d.debug_row_counts) d.debug_row_counts[t] = cnt;
  }
  if (cnt <= r) return;  // not more than r columns: no vector beyond the r largest
  if (lane == 0) {
    atomicAdd(&d.counters[0], 1ull);
    atomicAdd(&d.counters[7], (unsigned long long)(cnt - r));  // trace of I - Q Q^T
  }
  const int P = k * (k + 1) / 2;
  double acc[(kMaxL * (kMaxL + 1) / 2 + 31) / 32];
#pragma unroll
  for (int q = 0; q < (kMaxL * (kMaxL + 1) / 2 + 31) / 32; ++q) acc[q] = 0.0;
  int vmax = 0;
  const uint32_t ldb = (uint32_t)d.ldb;
  for (uint32_t w0 = 0; w0 < ldr; w0 += 32) {
    // list the columns of 32 words (one per lane), in ascending order
    const uint32_t w = w0 + lane;
    const uint32_t s = w < ldr ? sel_word(w) : 0u;
    const int c = __popc(s);
    int pre = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += y;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    pre -= c;
    for (uint32_t bits = s; bits; bits &= bits - 1) list[pre++] = (int)(w * 32 + __ffs(bits) - 1);
    __syncwarp();
    for (int c0 = 0; c0 < total; c0 += 32) {
      const int nc = total - c0 < 32 ? total - c0 : 32;
      if (lane < nc) {
        const uint32_t col = (uint32_t)list[c0 + lane];
        for (int a = 0; a < k; ++a) ys[lane * ks + a] = load_yd(d, col * ldy + (uint32_t)rows[a]);
        vmax = max(vmax, atomicAdd(&d.colcount[col], 1) + 1);
        if (d.visited)
          for (int a = 0; a < k; ++a)
            atomicOr(d.visited + (col * ldb + ((uint32_t)rows[a] >> 5)), 1u << (rows[a] & 31));
      }
      __syncwarp();
      int q = lane;
#pragma unroll
      for (int qi = 0; qi < (kMaxL * (kMaxL + 1) / 2 + 31) / 32; ++qi, q += 32) {
        if (q >= P) break;
        int a = 0, rem = q;
        while (rem >= k - a) {
          rem -= k - a;
          ++a;
        }
        const int b = a + rem;
        double sacc = acc[qi];
        for (int cc = 0; cc < nc; ++cc) sacc = fma(ys[cc * ks + a], ys[cc * ks + b], sacc);
        acc[qi] = sacc;
      }
      __syncwarp();
    }
  }
  // the largest column count bounds every entry of M (fixed-point scale)
#pragma unroll
  for (int o = 16; o; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if (lane == 0) atomicMax(&d.counters[2], (unsigned long long)vmax);
  {
    int q = lane;
#pragma unroll
    for (int qi = 0; qi < (kMaxL * (kMaxL + 1) / 2 + 31) / 32; ++qi, q += 32) {
      if (q >= P) break;
      int a = 0, rem = q;
      while (rem >= k - a) {
        rem -= k - a;
        ++a;
      }
      const int b = a + rem;
      G[a * ks + b] = acc[qi];
      G[b * ks + a] = acc[qi];
    }
  }
  __syncwarp();
  const double fro = warp_frobenius(G, k, ks);
  warp_jacobi<double>(G, U, k, ks, jsd[wid], 4.0 * DBL_EPSILON * fro);
  if (lane == 0) {  // eigenvalues descending
    for (int i = 0; i < k; ++i) order[wid][i] = i;
    for (int a = 1; a < k; ++a) {
      const int v = order[wid][a];
      int b = a - 1;
      while (b >= 0 && G[order[wid][b] * ks + order[wid][b]] < G[v * ks + v]) {
        order[wid][b + 1] = order[wid][b];
        --b;
      }
      order[wid][b + 1] = v;
    }
  }
  __syncwarp();
  // B_t = U_r diag(1 / sigma_r): row j of Q_t is B_t^T y_j (a zero column when sigma is 0)
  double* Bt = d.Bt + t * k * r;
  for (int e = lane; e < k * r; e += 32) {
    const int a = e / r, sidx = e % r;
    const int col = order[wid][sidx];
    const double lam = G[col * ks + col];
    Bt[e] = lam > 1e-300 ? U[a * ks + col] * rsqrt64(lam) : 0.0;
  }
}

// I - Q Q^T into M[C_t, C_t], one CTA per trial (rejected trials return).
__host__ __device__ inline size_t m2_scatter_smem(int64_t n, int kmax, int rmax) {
  return sizeof(int) * (size_t)n + sizeof(double) * ((size_t)kmax * rmax + 2 * (size_t)kQB * rmax);
}

__global__ void __launch_bounds__(256) k_m2_scatter(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                   int nprob, int64_t nmax, int kmax, int rmax) {
  extern __shared__ __align__(16) unsigned char scraw[];
  __shared__ int warp_sums[8];
  const int64_t g = blockIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - off[p];
  const int k = d.l, r = d.r;
  const int c_t = d.row_counts[t];
  if (c_t <= r) return;
  int* list = reinterpret_cast<int*>(scraw);
  double* Bs = reinterpret_cast<double*>(scraw + ((sizeof(int) * (size_t)nmax + 15) / 16 * 16));
  double* QA = Bs + (size_t)kmax * rmax;
  double* QB = QA + (size_t)kQB * rmax;
  const int32_t* R = d.cols + t * k;
  const uint32_t ldr = (uint32_t)d.ldr, ldy = (uint32_t)d.ldy, n = (uint32_t)d.n;
  for (int e = threadIdx.x; e < k * r; e += 256) Bs[e] = d.Bt[t * k * r + e];
  // the column list, ascending: 256 words per pass
  int base = 0;
  for (uint32_t w0 = 0; w0 < ldr; w0 += 256) {
    const uint32_t w = w0 + threadIdx.x;
    uint32_t s = 0;
    if (w < ldr) {
      s = 0xffffffffu;
      for (int a = 0; a < k; ++a) s &= __ldg(d.rbits + ((uint32_t)R[a] * ldr + w));
    }
    int total;
    int pre = block_exclusive_scan<256>(__popc(s), warp_sums, &total);
    for (uint32_t bits = s; bits; bits &= bits - 1) list[base + pre++] = (int)(w * 32 + __ffs(bits) - 1);
    base += total;
    __syncthreads();
  }
  __syncthreads();
  const int f = macc_frac_bits(d.counters[2]);
  const double scale = ldexp(1.0, f);
  auto q_rows = [&](double* Q, int j0, int nj) {  // Q[j][s] = sum_a y[R_a, C_{j0 + j}] B[a][s]
    for (int e = threadIdx.x; e < nj * r; e += 256) {
      const int j = e / r, sidx = e % r;
      const uint32_t col = (uint32_t)list[j0 + j];
      double v = 0.0;
      for (int a = 0; a < k; ++a) v = fma(load_yd(d, col * ldy + (uint32_t)R[a]), Bs[a * r + sidx], v);
      Q[j * r + sidx] = v;
    }
  };
  for (int i0 = 0; i0 < c_t; i0 += kQB) {
    const int ni = c_t - i0 < kQB ? c_t - i0 : kQB;
    __syncthreads();
    q_rows(QA, i0, ni);
    for (int j0 = i0; j0 < c_t; j0 += kQB) {
      const int nj = c_t - j0 < kQB ? c_t - j0 : kQB;
      __syncthreads();
      const double* QJ = QA;
      if (j0 != i0) {
        q_rows(QB, j0, nj);
        QJ = QB;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < ni * nj; e += 256) {
        const int i = e / nj, j = e % nj;
        double v = (i0 + i == j0 + j) ? 1.0 : 0.0;
        for (int sidx = 0; sidx < r; ++sidx) v = fma(-QA[i * r + sidx], QJ[j * r + sidx], v);
        const long long fx = llrint(v * scale);
        if (fx) {
          const uint32_t ci = (uint32_t)list[i0 + i], cj = (uint32_t)list[j0 + j];
          atomicAdd(&d.macc[ci * n + cj], (unsigned long long)fx);
          if (j0 != i0) atomicAdd(&d.macc[cj * n + ci], (unsigned long long)fx);
        }
      }
    }
  }
}

cudaError_t launch_rows_variant(const ProbDesc* descs, const int64_t* pack_off, int64_t pack_total,
                                const int64_t* trial_off, int64_t trials_total, int nprob, int kmax, int rmax,
                                int64_t nmax, cudaStream_t s) {
  cudaError_t e;
  if (pack_total > 0) {
    k_pack_rows<<<(unsigned)((pack_total + 255) / 256), 256, 0, s>>>(descs, pack_off, nprob);
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (trials_total <= 0) return cudaSuccess;
  const size_t tsm = kRowWarps * m2_trial_smem_per_warp(kmax);
  if ((e = cudaFuncSetAttribute(k_m2_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsm)) != cudaSuccess)
    return e;
  k_m2_trial<<<(unsigned)((trials_total + kRowWarps - 1) / kRowWarps), 32 * kRowWarps, tsm, s>>>(descs, trial_off,
                                                                                                 nprob, kmax);
  ++g_kernel_launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ssm = m2_scatter_smem(nmax, kmax, rmax) + 16;
  if ((e = cudaFuncSetAttribute(k_m2_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm)) != cudaSuccess)
    return e;
  k_m2_scatter<<<(unsigned)trials_total, 256, ssm, s>>>(descs, trial_off, nprob, nmax, kmax, rmax);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
