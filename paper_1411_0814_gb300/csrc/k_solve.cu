// Stages a8 (U-hat) and a9 (the error e).
//
// a8, eq. (solve.barU) with the L2 norm: for every row i, with
// K_i = {j : w_ij = 1}, u_i solves N_i u_i = b_i where N_i = sum_{j in K_i} v_j v_j^T
// and b_i = sum_{j in K_i} y_ij v_j.  For all rows at once this is a product:
//   [N_flat | b | |K_i|] (m x q) = [W | W o Y | W] (per output column) x Kmat (n x q)
// with Kmat[j] = (v_ja v_jb for a <= b, v_j, 1).  k_normal computes it as a tiled
// product (64 rows x 64 outputs per CTA); k_row_solve then solves each r x r
// system by Cholesky in FP64, falling back to the minimum-norm solution (a
// pseudo-inverse from a Jacobi eigendecomposition) for rank-deficient rows.
//
// a9, eq. (ep): e = (sum w_ij)^-1/2 || W o (Y - U V^T) ||_F, one thread per row,
// per-CTA partial sums reduced in a fixed order.  In the FP32 form the same pass
// applies one step of iterative refinement to U (refine_row) and reports the e of
// the refined U.
#include <cfloat>

#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"
#include "refine.cuh"

namespace rsm {

__device__ __forceinline__ void pair_of(int q, int r, int& a, int& b) {
  a = 0;
  int rem = q;
  while (rem >= r - a) {
    rem -= r - a;
    ++a;
  }
  b = a + rem;
}

template <typename TK>
__global__ void __launch_bounds__(256) k_build_K(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                int nprob) {
  pdl_enter();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - off[p];
  const int64_t j = e / d.q_pad;
  const int qq = (int)(e % d.q_pad);
  const int r = d.r, P = r * (r + 1) / 2;
  double v = 0.0;
  if (qq < P) {
    int a, b;
    pair_of(qq, r, a, b);
    v = d.V[(int64_t)a * d.ldv + j] * d.V[(int64_t)b * d.ldv + j];
  } else if (qq < P + r) {
    v = d.V[(int64_t)(qq - P) * d.ldv + j];
  } else if (qq == P + r) {
    v = 1.0;
  }
  static_cast<TK*>(static_cast<void*>(d.Kmat))[e] = (TK)v;  // FP32 forms keep Kmat in FP32
}

// Element offsets inside Y, the mask and Kmat are 32-bit (the host checks that
// they fit): 64-bit integer multiplies and adds are slow on this part.
template <typename T>
__device__ __forceinline__ T load_y(const ProbDesc& d, uint32_t idx) {
  if (d.y_dtype == 0) return (T)__ldg(static_cast<const double*>(d.Y) + idx);
  return (T)__ldg(static_cast<const float*>(d.Y) + idx);
}

constexpr int kNT = 64;  // rows per tile
constexpr int kQT = 64;  // outputs per tile
constexpr int kJT = 16;  // inner chunk

// MODE 0: FP64 multiply-add; MODE 2: FP32 multiply-add (output stored as FP64).
// Per 16-column chunk every thread loads 4 (row, column) entries of Y and
// their mask words (32 consecutive rows of one column per warp: coalesced) and
// 4 entries of Kmat; the loads of chunk k + 1 are issued before the products of
// chunk k, so their latency overlaps the arithmetic.  Y is read whether or not
// the entry is known and masked afterwards (unknown entries never reach the sum).
template <int MODE>
__global__ void __launch_bounds__(256) k_normal(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                               int nprob) {
  pdl_enter();
  using T = typename std::conditional<MODE == 0, double, float>::type;
  __shared__ T ys[kJT][kNT], ws[kJT][kNT], ks[kJT][kQT];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const T* __restrict__ Kmat = static_cast<const T*>(static_cast<const void*>(d.Kmat));
  const int64_t local = blockIdx.x - off[p];
  const int nqt = d.q_pad / kQT;
  const int64_t i0 = (local / nqt) * kNT;
  const int q0 = (int)(local % nqt) * kQT;
  const int P = d.r * (d.r + 1) / 2;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  bool isy[4];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int qq = q0 + tx + 16 * o;
    isy[o] = qq >= P && qq < P + d.r;
  }
  T acc[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int o = 0; o < 4; ++o) acc[s][o] = (T)0;
  const int64_t m = d.m, n = d.n;
  // loader mapping: entry e = threadIdx.x + 256 k -> (column e / 64, row or output e % 64)
  const int lr = threadIdx.x & 63, lj = threadIdx.x >> 6;
  const uint32_t li = (uint32_t)(i0 + lr);
  const uint32_t ldy = (uint32_t)d.ldy, ldb = (uint32_t)d.ldb, qp = (uint32_t)d.q_pad;
  T ypre[4], kpre[4];
  uint32_t wpre[4];
  auto load_chunk = [&](uint32_t j0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t j = j0 + lj + 4 * k;
      const bool in = li < (uint32_t)m && j < (uint32_t)n;
      wpre[k] = in ? __ldg(d.bits + (j * ldb + (li >> 5))) : 0u;
      ypre[k] = in ? load_y<T>(d, j * ldy + li) : (T)0;
      kpre[k] = j < (uint32_t)n ? __ldg(Kmat + (j * qp + q0 + lr)) : (T)0;
    }
  };
  load_chunk(0);
  for (uint32_t j0 = 0; j0 < (uint32_t)n; j0 += kJT) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool known = (wpre[k] >> (li & 31)) & 1u;
      ws[lj + 4 * k][lr] = known ? (T)1 : (T)0;
      ys[lj + 4 * k][lr] = known ? ypre[k] : (T)0;
      ks[lj + 4 * k][lr] = kpre[k];
    }
    __syncthreads();
    if (j0 + kJT < (uint32_t)n) load_chunk(j0 + kJT);
#pragma unroll 4
    for (int jj = 0; jj < kJT; ++jj) {
      T kv[4], wv[4], yv[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) kv[o] = ks[jj][tx + 16 * o];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        wv[s] = ws[jj][ty + 16 * s];
        yv[s] = ys[jj][ty + 16 * s];
      }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int o = 0; o < 4; ++o) acc[s][o] = fma(isy[o] ? yv[s] : wv[s], kv[o], acc[s][o]);
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t i = i0 + ty + 16 * s;
    if (i < m)
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const int qq = q0 + tx + 16 * o;
        if (qq < d.q) d.NB[i * d.q_pad + qq] = (double)acc[s][o];
      }
  }
}

// Cholesky solve of one row's r x r system (FP64), r <= RM, packed lower factor
// in registers.  A row with fewer than r known entries, or whose pivot falls
// below 1e-13 trace(N_i), is appended to the batch's fail list for the
// minimum-norm path (k_row_pinv).
template <int RM>
__global__ void __launch_bounds__(128) k_row_solve(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                  int nprob, unsigned long long* __restrict__ fail_list,
                                                  unsigned long long* __restrict__ fail_count) {
  pdl_enter();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t i = g - off[p];
  const int r = d.r, P = r * (r + 1) / 2;
  const double* row = d.NB + i * d.q_pad;
  double L[RM * (RM + 1) / 2];  // packed lower triangle, row-major: (a, b<=a) -> a(a+1)/2 + b
  double u[RM];
  double tr = 0.0;
#pragma unroll
  for (int a = 0; a < RM; ++a) {
    if (a >= r) break;
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      // N[a][b] = N[b][a]: packed upper index of (b, a) with b <= a
      const int qq = b * r - b * (b - 1) / 2 + (a - b);
      L[a * (a + 1) / 2 + b] = row[qq];
    }
    tr += L[a * (a + 1) / 2 + a];
  }
  const double known = row[P + r];
  bool ok = known >= (double)r;
#pragma unroll
  for (int j = 0; j < RM; ++j) {
    if (j >= r || !ok) break;
    double v = L[j * (j + 1) / 2 + j];
#pragma unroll
    for (int t = 0; t < j; ++t) v -= L[j * (j + 1) / 2 + t] * L[j * (j + 1) / 2 + t];
    if (!(v > 1e-13 * tr)) {
      ok = false;
      break;
    }
    v = sqrt(v);
    L[j * (j + 1) / 2 + j] = v;
#pragma unroll
    for (int k = j + 1; k < RM; ++k) {
      if (k >= r) break;
      double w = L[k * (k + 1) / 2 + j];
#pragma unroll
      for (int t = 0; t < j; ++t) w -= L[k * (k + 1) / 2 + t] * L[j * (j + 1) / 2 + t];
      L[k * (k + 1) / 2 + j] = w / v;
    }
  }
  if (!ok) {
    if (known < (double)r) atomicAdd(&d.counters[4], 1ull);
    const unsigned long long slot = atomicAdd(fail_count, 1ull);
    fail_list[slot] = ((unsigned long long)p << 32) | (unsigned long long)i;
    if (d.Lf) d.Lf[(size_t)i * P] = -1.f;  // no refinement: the minimum-norm path owns this row
    return;
  }
  if (d.Lf) {  // FP32 normal equations: the factor, for the refinement step of the residual pass
    float* lf = d.Lf + (size_t)i * P;
#pragma unroll
    for (int q = 0; q < RM * (RM + 1) / 2; ++q)
      if (q < P) lf[q] = (float)L[q];
  }
#pragma unroll
  for (int a = 0; a < RM; ++a) {  // C y = b
    if (a >= r) break;
    double v = row[P + a];
#pragma unroll
    for (int t = 0; t < a; ++t) v -= L[a * (a + 1) / 2 + t] * u[t];
    u[a] = v / L[a * (a + 1) / 2 + a];
  }
#pragma unroll
  for (int a = RM - 1; a >= 0; --a) {  // C^T u = y
    if (a >= r) continue;
    double v = u[a];
#pragma unroll
    for (int t = a + 1; t < RM; ++t)
      if (t < r) v -= L[t * (t + 1) / 2 + a] * u[t];
    u[a] = v / L[a * (a + 1) / 2 + a];
  }
  for (int a = 0; a < r; ++a) d.U[(int64_t)a * d.ldu + i] = u[a];
}

// Minimum-norm solution u = N^+ b for the rows of the fail list: one warp per
// row, eigendecomposition of N by the warp Jacobi solver, eigenvalues below
// 1e-12 of the largest treated as zero.
constexpr int kPinvWarps = 2;
__global__ void __launch_bounds__(32 * kPinvWarps) k_row_pinv(const ProbDesc* __restrict__ descs,
                                                             const unsigned long long* __restrict__ fail_list,
                                                             const unsigned long long* __restrict__ fail_count) {
  pdl_enter();
  __shared__ double S[kPinvWarps][kMaxR][kMaxR + 1], Q[kPinvWarps][kMaxR][kMaxR + 1];
  __shared__ JacobiScratch js[kPinvWarps];
  const double tol_scale = 4.0 * DBL_EPSILON;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned long long total = *fail_count;
  for (unsigned long long f = (unsigned long long)blockIdx.x * kPinvWarps + wid; f < total;
       f += (unsigned long long)gridDim.x * kPinvWarps) {
    const unsigned long long code = fail_list[f];
    const ProbDesc& d = descs[code >> 32];
    const int64_t i = (int64_t)(code & 0xffffffffull);
    const int r = d.r, P = r * (r + 1) / 2;
    const double* row = d.NB + i * d.q_pad;
    for (int qq = lane; qq < P; qq += 32) {
      int a, b;
      pair_of(qq, r, a, b);
      S[wid][a][b] = row[qq];
      S[wid][b][a] = row[qq];
    }
    __syncwarp();
    const double fro = warp_frobenius(&S[wid][0][0], r, kMaxR + 1);
    warp_jacobi<double>(&S[wid][0][0], &Q[wid][0][0], r, kMaxR + 1, js[wid], tol_scale * fro);
    double lmax = 0.0;
    for (int k = 0; k < r; ++k) lmax = fmax(lmax, S[wid][k][k]);
    // u_a = sum_k [lambda_k > tol] q_ak (q_k . b) / lambda_k, one output per lane
    for (int a = lane; a < r; a += 32) {
      double ua = 0.0;
      for (int k = 0; k < r; ++k) {
        const double lam = S[wid][k][k];
        if (!(lam > 1e-12 * lmax)) continue;
        double qb = 0.0;
        for (int t = 0; t < r; ++t) qb += Q[wid][t][k] * row[P + t];
        ua += Q[wid][a][k] * qb / lam;
      }
      d.U[(int64_t)a * d.ldu + i] = ua;
    }
    __syncwarp();
  }
}

// One step of iterative refinement of a row of U for the FP32 normal equations.
// e numerator: sum over known entries of (y_ij - u_i . v_j)^2.  A CTA takes 32
// consecutive rows (lane = row, so each column read is one coalesced 32-row
// segment and one mask word) and its 8 warps split the columns; V is staged in
// shared memory 64 columns at a time.  One partial per CTA, fixed-order tree.
// FP32 form (T = float): each thread also accumulates c = V_K^T r0 for its row
// over its columns; the 8 warps' parts are added in warp order in shared memory
// and warp 0 applies the refinement step (refine_row) to its 32 rows.
constexpr int kResRows = 32;
constexpr int kResCols = 64;
template <typename T, int RM>
__global__ void __launch_bounds__(256) k_residual(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                 int nprob, double* __restrict__ partial, int refine) {
  pdl_enter();
  constexpr bool kRefine = sizeof(T) == 4;
  __shared__ __align__(16) T vs[kResCols][RM];  // zero past r, so the products need no guard
  __shared__ float cred[kRefine ? kResRows : 1][RM + 1];
  __shared__ double red[8];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  const int64_t i0 = (blockIdx.x - off[p]) * kResRows;
  const int64_t i = i0 + lane;
  const bool row_in = i < d.m;
  const int r = d.r;
  // V: the FP32 forms keep a copy of V in FP32 (row j at vf32 + j * vf_ld)
  T u[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) u[a] = (a < r && row_in) ? (T)d.U[(int64_t)a * d.ldu + i] : (T)0;
  float cacc[RM];
#pragma unroll
  for (int a = 0; a < RM; ++a) cacc[a] = 0.f;
  // at most n / 8 terms per thread in the working precision (FP64 arithmetic is
  // far slower than FP32 on this part; one conversion per thread at the end)
  T acc = (T)0;
  const uint32_t wcol = (uint32_t)(i0 >> 5);
  const uint32_t irow = (uint32_t)(row_in ? i : i0);  // in-bounds row for the unconditional load
  const uint32_t ldy = (uint32_t)d.ldy, ldb = (uint32_t)d.ldb;
  for (int64_t j0 = 0; j0 < d.n; j0 += kResCols) {
    __syncthreads();
    for (int e = threadIdx.x; e < kResCols * RM; e += 256) {
      const int jj = e / RM, a = e % RM;
      const int64_t j = j0 + jj;
      T v = (T)0;
      if (j < d.n && a < r) v = sizeof(T) == 8 ? (T)d.V[(int64_t)a * d.ldv + j] : (T)d.vf32[j * d.vf_ld + a];
      vs[jj][a] = v;
    }
    __syncthreads();
    const int jn = d.n - j0 < kResCols ? (int)(d.n - j0) : kResCols;
#pragma unroll 4
    for (int jj = wg; jj < jn; jj += 8) {
      const uint32_t j = (uint32_t)j0 + jj;
      const uint32_t word = __ldg(d.bits + (j * ldb + wcol));
      const T y = load_y<T>(d, j * ldy + irow);
      T pred = (T)0;
      if constexpr (kRefine) {  // V row by 16-byte shared-memory loads
        float vr[RM];
        const float4* v4 = reinterpret_cast<const float4*>(&vs[jj][0]);
#pragma unroll
        for (int a4 = 0; a4 < RM / 4; ++a4) {
          const float4 v = v4[a4];
          vr[4 * a4] = v.x, vr[4 * a4 + 1] = v.y, vr[4 * a4 + 2] = v.z, vr[4 * a4 + 3] = v.w;
        }
#pragma unroll
        for (int a = 0; a < RM; ++a) pred = fmaf(u[a], vr[a], pred);
        const float diff = (row_in && ((word >> lane) & 1u)) ? y - pred : 0.f;
        acc = fmaf(diff, diff, acc);
#pragma unroll
        for (int a = 0; a < RM; ++a) cacc[a] = fmaf(diff, vr[a], cacc[a]);
      } else {
#pragma unroll
        for (int a = 0; a < RM; ++a) pred = fma(u[a], vs[jj][a], pred);
        const T diff = (row_in && ((word >> lane) & 1u)) ? y - pred : (T)0;
        acc = fma(diff, diff, acc);
      }
    }
  }
  double dacc = (double)acc;
  if constexpr (kRefine) {
    for (int w = 0; w < 8; ++w) {  // c of each row: the warps' parts in warp order
      if (wg == w)
#pragma unroll
        for (int a = 0; a < RM; ++a) cred[lane][a] = (w == 0 ? 0.f : cred[lane][a]) + cacc[a];
      __syncthreads();
    }
    if (wg == 0 && row_in && refine) {
      float c[RM], u32[RM];
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        c[a] = cred[lane][a];
        u32[a] = (float)u[a];
      }
      dacc -= refine_row<RM>(d, (uint32_t)i, u32, c);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
  if (lane == 0) red[wg] = dacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    partial[blockIdx.x] = t;
  }
}

// FP32 form of FP32 Y with 16-byte aligned columns: each lane takes 2
// consecutive rows (one 8-byte load per column), a CTA 64 rows, and its 8
// warps split the columns, 8 columns per pass, all loaded before any is used
// (2 KB of Y in flight per warp).  Each lane also accumulates c = V_K^T r0 for
// its 2 rows; the warps' parts are added in warp order in shared memory and
// threads 0..63 apply the refinement step (refine_row), one row each.  The
// per-lane state (2 rows x (u, c)) leaves room for three CTAs (24 warps) per
// SM.  Partials as in k_residual.
constexpr int kResVRows = 64;
constexpr int kResVCols = 8;      // columns in flight per warp and pass
constexpr int kResVStage = 512;   // columns of V staged per barrier (8 passes of each warp)
// RM = 16 (8 < r <= 16): the same with two CTAs per SM (its per-lane state is
// twice as large).  A CTA returns at once for a problem with r outside [rlo,
// rhi], which the other instantiation (or the TMA-fed pass) takes.
template <int RM>
__global__ void __launch_bounds__(256, RM <= 8 ? 3 : 2) k_residual2(const ProbDesc* __restrict__ descs,
                                                                  const int64_t* __restrict__ off, int nprob,
                                                                  double* __restrict__ partial, int refine, int rlo,
                                                                  int rhi) {
  pdl_enter();
  __shared__ __align__(16) float vs[kResVStage][RM];
  __shared__ float cred[kResVRows][RM + 1];
  __shared__ double red[8];
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  if (d.r < rlo || d.r > rhi) return;
  const int lane = threadIdx.x & 31, wg = threadIdx.x >> 5;
  const uint32_t i0 = (uint32_t)(blockIdx.x - off[p]) * kResVRows;
  const uint32_t ib = i0 + 2u * lane;  // first of this lane's 2 rows
  const uint32_t m = (uint32_t)d.m;
  const bool pair_in = ib < m;  // m is even or the second row is masked out below
  const int r = d.r;
  float u[2][RM], cacc[2][RM];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      u[k][a] = (a < r && ib + k < m) ? (float)d.U[(int64_t)a * d.ldu + ib + k] : 0.f;
      cacc[k][a] = 0.f;
    }
  const float* __restrict__ Y = static_cast<const float*>(d.Y);
  const uint32_t ldy = (uint32_t)d.ldy, ldb = (uint32_t)d.ldb, n = (uint32_t)d.n;
  const uint32_t wrow = ib >> 5, shift = ib & 31u;
  const uint32_t keep = ib + 1 < m ? 3u : 1u;  // the second row exists
  float acc = 0.f;
  for (uint32_t j0 = 0; j0 < n; j0 += kResVStage) {
    __syncthreads();
    for (int e = threadIdx.x; e < kResVStage * RM; e += 256) {
      const int jj = e / RM, a = e % RM;
      const uint32_t j = j0 + jj;
      vs[jj][a] = (j < n && a < r) ? d.vf32[j * d.vf_ld + a] : 0.f;
    }
    __syncthreads();
    const int jn = n - j0 < (uint32_t)kResVStage ? (int)(n - j0) : kResVStage;
    for (int jb = wg; jb < jn; jb += 8 * kResVCols) {  // columns jb, jb + 8, ..., jb + 56
      float2 y[kResVCols];
      uint32_t bits[kResVCols];
#pragma unroll
      for (int q = 0; q < kResVCols; ++q) {
        const int jj = jb + 8 * q;
        const uint32_t j = j0 + jj;
        const bool ok = jj < jn && pair_in;
        y[q] = ok ? __ldg(reinterpret_cast<const float2*>(Y + (j * ldy + ib))) : make_float2(0.f, 0.f);
        bits[q] = ok ? (__ldg(d.bits + (j * ldb + wrow)) >> shift) & keep : 0u;
      }
#pragma unroll
      for (int q = 0; q < kResVCols; ++q) {
        const int jj = jb + 8 * q;
        if (jj >= jn) break;
        float vr[RM];
        const float4* v4 = reinterpret_cast<const float4*>(&vs[jj][0]);
#pragma unroll
        for (int a4 = 0; a4 < RM / 4; ++a4) {
          const float4 v = v4[a4];
          vr[4 * a4] = v.x, vr[4 * a4 + 1] = v.y, vr[4 * a4 + 2] = v.z, vr[4 * a4 + 3] = v.w;
        }
        const float yv[2] = {y[q].x, y[q].y};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          float pr = 0.f;
#pragma unroll
          for (int a = 0; a < RM; ++a) pr = fmaf(u[k][a], vr[a], pr);
          const float diff = ((bits[q] >> k) & 1u) ? yv[k] - pr : 0.f;
          acc = fmaf(diff, diff, acc);
#pragma unroll
          for (int a = 0; a < RM; ++a) cacc[k][a] = fmaf(diff, vr[a], cacc[k][a]);
        }
      }
    }
  }
  double dacc = (double)acc;
  if (refine) {  // uniform over the CTA
    for (int w = 0; w < 8; ++w) {  // c of each row: the warps' parts in warp order
      if (wg == w)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int a = 0; a < RM; ++a) cred[2 * lane + k][a] = (w == 0 ? 0.f : cred[2 * lane + k][a]) + cacc[k][a];
      __syncthreads();
    }
    if (threadIdx.x < kResVRows && i0 + threadIdx.x < m) {
      const uint32_t row = i0 + threadIdx.x;
      float c[RM], u32[RM];
#pragma unroll
      for (int a = 0; a < RM; ++a) {
        c[a] = cred[threadIdx.x][a];
        u32[a] = a < r ? (float)d.U[(int64_t)a * d.ldu + row] : 0.f;
      }
      dacc -= refine_row<RM>(d, row, u32, c);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
  if (lane == 0) red[wg] = dacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_residual_final(const ProbDesc* __restrict__ descs,
                                                       const int64_t* __restrict__ off, const int64_t* __restrict__ off4,
                                                       int64_t base4, int nprob, const double* __restrict__ partial) {
  pdl_enter();
  __shared__ double red[256];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  double s = 0.0;  // strided partial sums over this problem's partials (one of the two ranges), then a fixed tree
  for (int64_t b = off[p] + threadIdx.x; b < off[p + 1]; b += 256) s += partial[b];
  for (int64_t b = base4 + off4[p] + threadIdx.x; b < base4 + off4[p + 1]; b += 256) s += partial[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double known = (double)d.counters[1];
    d.stats[32] = red[0];
    d.stats[33] = known > 0.0 ? sqrt(red[0] / known) : 0.0;
  }
}

cudaError_t launch_solve_u(const SolvePlan& S, int mode, cudaStream_t s) {
  const ProbDesc* D = S.descs;
  const int np = S.nprob;
  cudaError_t e;
  if (S.k_total > 0) {
    if (mode == 0)
      (void)launch_chained(k_build_K<double>, (unsigned)((S.k_total + 255) / 256), 256, 0, s, D, S.k_off, np);
    else
      (void)launch_chained(k_build_K<float>, (unsigned)((S.k_total + 255) / 256), 256, 0, s, D, S.k_off, np);
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (S.tc_tiles > 0 || S.b_total > 0) {
    if ((e = launch_normal_tc(S, S.tc_rb, S.tc_npad_max, s)) != cudaSuccess) return e;
  }
  if (S.tile_off_host_total > 0) {
    if (mode == 0) {
      (void)launch_chained(k_normal<0>, (unsigned)S.tile_off_host_total, 256, 0, s, D, S.tile_off, np);
    } else {
      (void)launch_chained(k_normal<2>, (unsigned)S.tile_off_host_total, 256, 0, s, D, S.tile_off, np);
    }
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (S.row_total > 0) {
    const unsigned blocks = (unsigned)((S.row_total + 127) / 128);
    if (S.rmax <= 4) {
      (void)launch_chained(k_row_solve<4>, blocks, 128, 0, s, D, S.row_off, np, S.fail_list, S.fail_count);
    } else if (S.rmax <= 8) {
      (void)launch_chained(k_row_solve<8>, blocks, 128, 0, s, D, S.row_off, np, S.fail_list, S.fail_count);
    } else if (S.rmax <= 16) {
      (void)launch_chained(k_row_solve<16>, blocks, 128, 0, s, D, S.row_off, np, S.fail_list, S.fail_count);
    } else {
      (void)launch_chained(k_row_solve<32>, blocks, 128, 0, s, D, S.row_off, np, S.fail_list, S.fail_count);
    }
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (S.any_solve) {  // rows that any of the solvers handed to the minimum-norm path
    (void)launch_chained(k_row_pinv, 152, 32 * kPinvWarps, 0, s, D, S.fail_list, S.fail_count);
    ++g_kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(const SolvePlan& S, int mode, double* partial, cudaStream_t s, bool refine) {
  const ProbDesc* D = S.descs;
  const int np = S.nprob;
  const int rf = refine ? 1 : 0;
  if (S.res_blocks > 0) {
#define RSM_RES(T, RM) \
  (void)launch_chained(k_residual<T, RM>, (unsigned)S.res_blocks, 256, 0, s, D, S.res_off, np, partial, rf)
    if (mode == 0) {
      if (S.rmax <= 8) RSM_RES(double, 8); else if (S.rmax <= 16) RSM_RES(double, 16); else RSM_RES(double, 32);
    } else {
      if (S.rmax <= 8) RSM_RES(float, 8); else if (S.rmax <= 16) RSM_RES(float, 16); else RSM_RES(float, 32);
    }
#undef RSM_RES
    ++g_kernel_launches;
  }
  if (S.resv_blocks > 0) {  // r <= 8: the TMA-fed pass or the 2-row kernel; 8 < r <= 16: the 2-row kernel at RM = 16
    if (S.tc_tma) {
      cudaError_t et = launch_residual_tma(S, partial + S.res_blocks, rf, s);
      if (et != cudaSuccess) return et;
    } else {
      (void)launch_chained(k_residual2<8>, (unsigned)S.resv_blocks, 256, 0, s, D, S.resv_off, np, partial + S.res_blocks,
                           rf, 1, 8);
      ++g_kernel_launches;
    }
    if (S.resv_rmax > 8) {
      (void)launch_chained(k_residual2<16>, (unsigned)S.resv_blocks, 256, 0, s, D, S.resv_off, np,
                           partial + S.res_blocks, rf, 9, 16);
      ++g_kernel_launches;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (void)launch_chained(k_residual_final, np, 256, 0, s, D, S.res_off, S.resv_off, S.res_blocks, np, partial);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
