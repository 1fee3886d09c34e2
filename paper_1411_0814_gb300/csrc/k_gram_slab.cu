// Stages a3 + a4 with an L2-resident row-slab schedule.
//
// Same result as k_select_gram (per trial: the rows known in all chosen
// columns, and the Gram A_t^T A_t of the submatrix), organised for the memory
// system: Y is swept in row slabs small enough to stay in L2 (32 MiB of Y per
// slab), and one launch serves a slab to every trial.  The first trial that
// touches a sector of the slab brings it from HBM; the ~l/n share of all other
// trials that draw the same column then read it from L2.  HBM traffic drops
// from ~32 B per selected element (one sector each) to about one read of Y.
//
// One warp per (trial, slab): lanes AND the l packed mask words of 32
// consecutive 32-row groups, selected rows go to a per-warp ring buffer, and
// every full batch of 32 rows is gathered (lane = row) and multiplied into
// register accumulators of the l(l+1)/2 products.  At the end of the slab the
// warp reduces its accumulators through shared memory (fixed order) and adds
// them to the trial's FP64 Gram; slab 0 writes, later slabs add, one launch per
// slab, so the sum over slabs is in a fixed order too.
#include "common.cuh"
#include "kernels.h"

namespace rsm {

constexpr int kSlabWarps = 4;
// CTAs per SM that the register file allows without spills: each lane holds the
// l(l+1)/2 accumulators, the l gathered values and the l prefetched mask words
// (FP64 values take two registers), plus about 40 for indices and addresses.
// Capped at five, which keeps the ring buffers of the warps in shared memory.
template <int MODE, int L>
constexpr int slab_minb() {
  constexpr int w = MODE == 0 ? 2 : 1;
  constexpr int need = w * (L * (L + 1) / 2) + (w + 1) * L + 40;
  constexpr int fit = 65536 / (32 * kSlabWarps * ((need + 7) / 8 * 8));
  // l = 9 FP32 (the paper-scale case) fits five CTAs per SM at 96 registers: measured
  // 2.39 ms against 2.48 ms at four per decomposition of the 131072 x 1024 workload
  if (MODE == 2 && L == 9) return 5;
  return fit < 1 ? 1 : (fit > 5 ? 5 : fit);
}
constexpr int kRing = 1088;  // pending rows per warp: < 32 + 32 * 32
constexpr int kMeta = 40;    // per warp: the l column offsets into Y (from 0), then into the mask (from 20)

template <int MODE>
struct SlabT;
template <>
struct SlabT<0> {  // FP64 Gram of FP64 Y
  using acc_t = double;
  using val_t = double;
  using src_t = double;
  __device__ static val_t cvt(src_t x) { return x; }
};
template <>
struct SlabT<2> {  // FP32 Gram of FP32 Y
  using acc_t = float;
  using val_t = float;
  using src_t = float;
  __device__ static val_t cvt(src_t x) { return x; }
};

// V = 0: the CTAs per SM of slab_minb; V = 1: one fewer (more registers per
// thread); the autotuner picks between them per problem shape.
// OCC = 1 asks for one CTA per SM fewer than slab_minb (more registers per thread)
template <int MODE, int L, int OCC>
__global__ void __launch_bounds__(32 * kSlabWarps, (slab_minb<MODE, L>() - OCC > 1 ? slab_minb<MODE, L>() - OCC : 1))
    k_gram_slab(const ProbDesc* __restrict__ descs,
                                                               const int64_t* __restrict__ task_off, int nprob,
                                                               int slab) {
  pdl_enter();
  using Tr = SlabT<MODE>;
  using A = typename Tr::acc_t;
  using V = typename Tr::val_t;
  constexpr int P = L * (L + 1) / 2;
  constexpr int kRedWords = (P * 33 * sizeof(A) + 3) / 4;
  constexpr int kWarpWords = kRedWords > kRing ? kRedWords : kRing;
  extern __shared__ __align__(16) int slab_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* ring = slab_smem + wid * (kWarpWords + kMeta);
  A* red = reinterpret_cast<A*>(ring);
  uint32_t* meta = reinterpret_cast<uint32_t*>(ring + kWarpWords);

  const int64_t g = (int64_t)blockIdx.x * kSlabWarps + wid;
  if (g >= task_off[nprob]) return;
  const int p = find_problem(task_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - task_off[p];
  // 32-bit column offsets into Y and the mask (the host checks ldy n, ldb n <
  // 2^32), kept in shared memory (broadcast reads) rather than in 2 l
  // registers, which leaves room for five CTAs per SM
  const typename Tr::src_t* __restrict__ Yb = static_cast<const typename Tr::src_t*>(d.Y);
  const uint32_t* __restrict__ Bb = d.bits;
  if (lane < L) {
    const uint32_t c = (uint32_t)__ldg(d.cols + t * L + lane);
    meta[lane] = c * (uint32_t)d.ldy;
    meta[20 + lane] = c * (uint32_t)d.ldb;
  }
  __syncwarp();
  // word indices are 32-bit (m < 2^31, so m / 32 words fit)
  const int64_t r0 = (int64_t)slab * d.slab_rows;
  const int64_t r1 = r0 + d.slab_rows < d.m ? r0 + d.slab_rows : d.m;
  const uint32_t w_begin = (uint32_t)(r0 >> 5), w_end = (uint32_t)((r1 + 31) >> 5);

  A acc[P];
#pragma unroll
  for (int q = 0; q < P; ++q) acc[q] = (A)0;
  int pending = 0, count = 0;

  auto consume = [&](int k) {  // gather row ring[k] and add its outer product
    const uint32_t row = (uint32_t)ring[k];
    V v[L];
#pragma unroll
    for (int a = 0; a < L; ++a) v[a] = Tr::cvt(__ldg(Yb + (meta[a] + row)));
#pragma unroll
    for (int a = 0; a < L; ++a)
#pragma unroll
      for (int b = a; b < L; ++b) {
        const int q = a * L - a * (a - 1) / 2 + (b - a);
        acc[q] = fma(v[a], v[b], acc[q]);
      }
  };

  // The mask words of the next 32-word step are loaded before this step's rows
  // are gathered, so their latency overlaps the gathers and products.
  uint32_t nextw[L];
  auto load_words = [&](uint32_t w0) {
    const uint32_t w = w0 + lane;
    const bool in = w < w_end;
#pragma unroll
    for (int k = 0; k < L; ++k) nextw[k] = in ? __ldg(Bb + (meta[20 + k] + w)) : 0u;
  };
  if (w_begin < w_end) load_words(w_begin);
  for (uint32_t w0 = w_begin; w0 < w_end; w0 += 32) {
    const uint32_t w = w0 + lane;
    uint32_t mask = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < L; ++k) mask &= nextw[k];
    if (w0 + 32 < w_end) load_words(w0 + 32);
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = pending + incl - cnt;
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      ring[pos++] = (int)(w * 32u + (uint32_t)b);
    }
    __syncwarp();
    pending += total;
    count += total;
    int done = 0;
    while (pending - done >= 32) {
      consume(done + lane);
      done += 32;
    }
    __syncwarp();
    if (done) {  // move the remainder (< 32 rows) to the front
      const int rest = pending - done;
      const int keep = lane < rest ? ring[done + lane] : 0;
      __syncwarp();
      if (lane < rest) ring[lane] = keep;
      __syncwarp();
      pending = rest;
    }
  }
  if (lane < pending) consume(lane);
  __syncwarp();

  // reduce the 32 lanes' accumulators through shared memory, lane q sums entry q
#pragma unroll
  for (int q = 0; q < P; ++q) red[q * 33 + lane] = acc[q];
  __syncwarp();
  double* G = d.gram + t * P;
  for (int q = lane; q < P; q += 32) {
    A s = (A)0;
    for (int k = 0; k < 32; ++k) s += red[q * 33 + k];
    G[q] = (slab == 0 ? 0.0 : G[q]) + (double)s;
  }
  if (lane == 0) {
    const int32_t c0 = slab == 0 ? 0 : d.row_counts[t];
    const int32_t c = c0 + count;
    d.row_counts[t] = c;
    if (d.debug_row_counts) d.debug_row_counts[t] = c;
    if (count) atomicAdd(&d.counters[5], (unsigned long long)count);
  }
}

template <int MODE, int L>
static size_t slab_smem_bytes() {
  using A = typename SlabT<MODE>::acc_t;
  constexpr int P = L * (L + 1) / 2;
  constexpr int kRedWords = (P * 33 * sizeof(A) + 3) / 4;
  constexpr int kWarpWords = kRedWords > kRing ? kRedWords : kRing;
  return (size_t)kSlabWarps * (kWarpWords + kMeta) * 4;
}

// regs != NULL: report the kernel's registers per thread instead of launching
template <int MODE, int L, int OCC>
static cudaError_t launch_slab_l(const SlabPlan* Sp, cudaStream_t s, int* regs) {
  if (regs) {
    cudaFuncAttributes a{};
    cudaError_t e = cudaFuncGetAttributes(&a, k_gram_slab<MODE, L, OCC>);
    *regs = e == cudaSuccess ? a.numRegs : -1;
    return e;
  }
  const SlabPlan& S = *Sp;
  const size_t smem = slab_smem_bytes<MODE, L>();
  cudaError_t e = cudaFuncSetAttribute(k_gram_slab<MODE, L, OCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int sl = 0; sl < S.nslab; ++sl) {
    const int64_t tasks = S.hT[S.task_pos + (size_t)sl * (S.nprob + 1) + S.nprob];
    if (tasks <= 0) continue;
    (void)launch_chained(k_gram_slab<MODE, L, OCC>, (unsigned)((tasks + kSlabWarps - 1) / kSlabWarps), 32 * kSlabWarps,
                         smem, s, S.descs, S.dT + S.task_pos + (size_t)sl * (S.nprob + 1), S.nprob, sl);
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The slab kernel reads Y in the Gram's own precision (FP32 Gram of FP32 Y,
// FP64 Gram of FP64 Y); other combinations take the per-trial kernel.
bool slab_supported(int mode, int l, int y_dtype) {
  if (mode == 2) return y_dtype == 1 && l >= 2 && l <= 17;
  if (mode == 0) return y_dtype == 0 && l >= 2 && l <= 12;
  return false;
}

static cudaError_t slab_dispatch(int mode, int l, int variant, const SlabPlan* S, cudaStream_t s, int* regs) {
#define RSM_SLAB_CASE(M, LL)                                                  \
  case LL:                                                                    \
    return variant ? launch_slab_l<M, LL, 1>(S, s, regs) : launch_slab_l<M, LL, 0>(S, s, regs);
  if (mode == 2) {
    switch (l) {
      RSM_SLAB_CASE(2, 2) RSM_SLAB_CASE(2, 3) RSM_SLAB_CASE(2, 4) RSM_SLAB_CASE(2, 5) RSM_SLAB_CASE(2, 6)
      RSM_SLAB_CASE(2, 7) RSM_SLAB_CASE(2, 8) RSM_SLAB_CASE(2, 9) RSM_SLAB_CASE(2, 10) RSM_SLAB_CASE(2, 11)
      RSM_SLAB_CASE(2, 12) RSM_SLAB_CASE(2, 13) RSM_SLAB_CASE(2, 14) RSM_SLAB_CASE(2, 15) RSM_SLAB_CASE(2, 16)
      RSM_SLAB_CASE(2, 17)
      default: break;
    }
  } else if (mode == 0) {
    switch (l) {
      RSM_SLAB_CASE(0, 2) RSM_SLAB_CASE(0, 3) RSM_SLAB_CASE(0, 4) RSM_SLAB_CASE(0, 5) RSM_SLAB_CASE(0, 6)
      RSM_SLAB_CASE(0, 7) RSM_SLAB_CASE(0, 8) RSM_SLAB_CASE(0, 9) RSM_SLAB_CASE(0, 10) RSM_SLAB_CASE(0, 11)
      RSM_SLAB_CASE(0, 12)
      default: break;
    }
  }
#undef RSM_SLAB_CASE
  return cudaErrorNotSupported;
}

cudaError_t launch_gram_slab(int mode, int l, int variant, const SlabPlan& S, cudaStream_t s) {
  return slab_dispatch(mode, l, variant, &S, s, nullptr);
}

int gram_slab_regs(int mode, int l, int variant) {
  int regs = -1;
  if (slab_dispatch(mode, l, variant, nullptr, nullptr, &regs) != cudaSuccess) cudaGetLastError();
  return regs;
}

}  // namespace rsm
