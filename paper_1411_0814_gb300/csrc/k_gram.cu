// Stages a3 + a4, fused: for each trial, select the rows known in all chosen
// columns (Section III, M1) and accumulate the l x l Gram matrix A_t^T A_t of
// the submatrix A_t = Y[R_t, C_t] (its right singular vectors are the
// eigenvectors of the Gram; Section III takes those of the smallest singular
// values).  The row list is never written to global memory.
//
// One CTA (256 threads) per trial, flattened over the problems of a batch.
// Per step the CTA ANDs the l packed mask words of 256 x 32 rows, places the
// selected rows in shared memory with a block scan, gathers their l values of
// Y into a shared tile, and adds the tile's outer products to per-thread
// partial sums (one packed pair (a, b), a <= b, per thread, rows split over
// thread groups).  The partial sums are reduced in a fixed order, so the result
// is deterministic.
#include "common.cuh"
#include "kernels.h"

namespace rsm {

// Arithmetic of the Gram: MODE 0 = FP64, 1 = FP32 pairs (hi + lo), 2 = FP32.
template <int MODE>
struct GramTraits;

template <>
struct GramTraits<0> {
  using elem = double;
  struct acc {
    double s = 0.0;
  };
  __device__ static elem load(const ProbDesc& d, int64_t idx) {
    return d.y_dtype == 0 ? __ldg(static_cast<const double*>(d.Y) + idx)
                          : (double)__ldg(static_cast<const float*>(d.Y) + idx);
  }
  __device__ static void fma(acc& a, elem x, elem y) { a.s = ::fma(x, y, a.s); }
  __device__ static void add(acc& a, const acc& b) { a.s += b.s; }
  __device__ static void renorm(acc&) {}
  __device__ static double value(const acc& a) { return a.s; }
};

// Unevaluated float pairs: y = hi + lo with hi = fl32(y), lo = fl32(y - hi)
// (about 48 significant bits of y).  Products hi*hi are split exactly with an
// FMA (Dekker's TwoProduct via FMA), cross terms are single FP32 products, and
// sums use Knuth's TwoSum (error-free), so the Gram carries about 2^-44
// relative accuracy while running on the FP32 pipes.
template <>
struct GramTraits<1> {
  using elem = float2;
  struct acc {
    float h = 0.f, l = 0.f;
  };
  __device__ static elem load(const ProbDesc& d, int64_t idx) {
    if (d.y_dtype == 0) {
      double v = __ldg(static_cast<const double*>(d.Y) + idx);
      float hi = __double2float_rn(v);
      float lo = __double2float_rn(v - (double)hi);
      return make_float2(hi, lo);
    }
    return make_float2(__ldg(static_cast<const float*>(d.Y) + idx), 0.f);
  }
  __device__ static void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  __device__ static void fma(acc& a, elem x, elem y) {
    float ph = __fmul_rn(x.x, y.x);
    float pe = __fmaf_rn(x.x, y.x, -ph);
    float cross = __fmaf_rn(x.x, y.y, __fmul_rn(x.y, y.x));
    float s, e;
    two_sum(a.h, ph, s, e);
    a.l = __fadd_rn(a.l, __fadd_rn(e, __fadd_rn(pe, cross)));
    a.h = s;
  }
  __device__ static void renorm(acc& a) {
    float s = __fadd_rn(a.h, a.l);
    a.l = __fsub_rn(a.l, __fsub_rn(s, a.h));
    a.h = s;
  }
  __device__ static void add(acc& a, const acc& b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    a.l = __fadd_rn(a.l, __fadd_rn(e, b.l));
    a.h = s;
    renorm(a);
  }
  __device__ static double value(const acc& a) { return (double)a.h + (double)a.l; }
};

template <>
struct GramTraits<2> {
  using elem = float;
  struct acc {
    float s = 0.f;
  };
  __device__ static elem load(const ProbDesc& d, int64_t idx) {
    return d.y_dtype == 1 ? __ldg(static_cast<const float*>(d.Y) + idx)
                          : __double2float_rn(__ldg(static_cast<const double*>(d.Y) + idx));
  }
  __device__ static void fma(acc& a, elem x, elem y) { a.s = fmaf(x, y, a.s); }
  __device__ static void add(acc& a, const acc& b) { a.s += b.s; }
  __device__ static void renorm(acc&) {}
  __device__ static double value(const acc& a) { return (double)a.s; }
};

constexpr int kGramThreads = 256;
constexpr int kMaxPairs = kMaxL * (kMaxL + 1) / 2;  // 528
constexpr int kPairsPerThread = (kMaxPairs + kGramThreads - 1) / kGramThreads;  // 3

template <int MODE>
__global__ void __launch_bounds__(kGramThreads) k_select_gram(const ProbDesc* __restrict__ descs,
                                                             const int64_t* __restrict__ trial_off, int nprob,
                                                             int cap) {
  using T = GramTraits<MODE>;
  using E = typename T::elem;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int warp_sums[kGramThreads / 32];
  __shared__ int32_t cidx[kMaxL];
  __shared__ uint8_t pa[kMaxPairs], pb[kMaxPairs];

  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - trial_off[p];
  const int l = d.l;
  const int P = l * (l + 1) / 2;
  E* tile = reinterpret_cast<E*>(smem);                         // cap x l
  int32_t* rows = reinterpret_cast<int32_t*>(smem + sizeof(E) * (size_t)cap * l);  // cap

  if (tid < l) cidx[tid] = d.cols[t * l + tid];
  for (int q = tid; q < P; q += kGramThreads) {
    // packed upper triangle, row-major: q -> (a, b) with a <= b
    int a = 0, rem = q;
    while (rem >= l - a) {
      rem -= l - a;
      ++a;
    }
    pa[q] = (uint8_t)a;
    pb[q] = (uint8_t)(a + rem);
  }
  __syncthreads();

  // work split: P <= 256 -> G groups of P threads, one pair each; else up to 3 pairs per thread
  const int G = P <= kGramThreads ? kGramThreads / P : 1;
  const int grp = P <= kGramThreads ? tid / P : 0;
  int my_q[kPairsPerThread];
  int nq = 0;
  if (P <= kGramThreads) {
    if (tid < G * P) my_q[nq++] = tid % P;
  } else {
    for (int q = tid; q < P; q += kGramThreads) my_q[nq++] = q;
  }
  int qa[kPairsPerThread], qb[kPairsPerThread];
  for (int i = 0; i < nq; ++i) {
    qa[i] = pa[my_q[i]];
    qb[i] = pb[my_q[i]];
  }
  typename T::acc acc[kPairsPerThread];

  const int64_t nwords = (d.m + 31) / 32;
  const uint32_t* __restrict__ bits = d.bits;
  const int64_t ldb = d.ldb, ldy = d.ldy;
  int64_t count = 0;
  for (int64_t w0 = 0; w0 < nwords; w0 += kGramThreads) {
    const int64_t w = w0 + tid;
    uint32_t mask = 0;
    if (w < nwords) {
      mask = 0xffffffffu;
      for (int k = 0; k < l; ++k) mask &= __ldg(bits + (int64_t)cidx[k] * ldb + w);
    }
    int total;
    const int off = block_exclusive_scan<kGramThreads>(__popc(mask), warp_sums, &total);
    for (int base = 0; base < total; base += cap) {
      // place my selected rows whose rank falls in [base, base + cap)
      uint32_t mm = mask;
      int rank = off;
      while (mm) {
        const int b = __ffs(mm) - 1;
        mm &= mm - 1;
        if (rank >= base && rank < base + cap) rows[rank - base] = (int32_t)(w * 32 + b);
        ++rank;
      }
      __syncthreads();
      const int nr = min(cap, total - base);
      // gather the submatrix rows: consecutive threads read consecutive rows of one column
#pragma unroll 4
      for (int idx = tid; idx < nr * l; idx += kGramThreads) {
        const int i = idx % nr, k = idx / nr;
        tile[i * l + k] = T::load(d, (int64_t)rows[i] + (int64_t)cidx[k] * ldy);
      }
      __syncthreads();
      for (int j = 0; j < nq; ++j) {
        const int a = qa[j], b = qb[j];
        typename T::acc s = acc[j];
        for (int i = grp; i < nr; i += G) T::fma(s, tile[i * l + a], tile[i * l + b]);
        T::renorm(s);
        acc[j] = s;
      }
      __syncthreads();
    }
    count += total;
  }

  // fixed-order reduction of the group partials
  typename T::acc* red = reinterpret_cast<typename T::acc*>(smem);
  if (P <= kGramThreads) {
    if (nq) red[grp * P + my_q[0]] = acc[0];
    __syncthreads();
    if (tid < P) {
      typename T::acc s = red[tid];
      for (int gg = 1; gg < G; ++gg) T::add(s, red[gg * P + tid]);
      d.gram[t * P + tid] = T::value(s);
    }
  } else {
    for (int j = 0; j < nq; ++j) d.gram[t * P + my_q[j]] = T::value(acc[j]);
  }
  if (tid == 0) {
    d.row_counts[t] = (int32_t)count;
    if (count) atomicAdd(&d.counters[5], (unsigned long long)count);
    if (d.debug_row_counts) d.debug_row_counts[t] = (int32_t)count;
  }
}

size_t gram_elem_bytes(int mode) { return mode == 0 ? 8 : mode == 1 ? 8 : 4; }

int gram_cap_rows(int mode, int lmax) {
  // dynamic shared memory budget of 64 KB: cap rows of l elements + cap row indices
  const size_t budget = 64 * 1024;
  size_t per_row = gram_elem_bytes(mode) * (size_t)lmax + 4;
  int cap = (int)(budget / per_row);
  return cap > 4096 ? 4096 : cap;
}

cudaError_t launch_select_gram(int mode, const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total,
                               int lmax, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int cap = gram_cap_rows(mode, lmax);
  const size_t smem = gram_elem_bytes(mode) * (size_t)cap * lmax + 4 * (size_t)cap;
  // the reduction buffer reuses the tile: needs 256 accumulators
  const size_t need_red = 256 * 16;
  const size_t dyn = smem > need_red ? smem : need_red;
  cudaError_t e;
  switch (mode) {
    case 0:
      e = cudaFuncSetAttribute(k_select_gram<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
      k_select_gram<0><<<(unsigned)total, kGramThreads, dyn, s>>>(descs, trial_off, nprob, cap);
      ++g_kernel_launches;
      break;
    case 1:
      e = cudaFuncSetAttribute(k_select_gram<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
      k_select_gram<1><<<(unsigned)total, kGramThreads, dyn, s>>>(descs, trial_off, nprob, cap);
      ++g_kernel_launches;
      break;
    default:
      e = cudaFuncSetAttribute(k_select_gram<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
      k_select_gram<2><<<(unsigned)total, kGramThreads, dyn, s>>>(descs, trial_off, nprob, cap);
      ++g_kernel_launches;
      break;
  }
  return cudaGetLastError();
}

}  // namespace rsm
