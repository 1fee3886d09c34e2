// Stage a8 (the per-row normal equations of eq. solve.barU), FP32 form, on the
// 5th-generation tensor cores.
//
// For every row i the solve needs N_i = sum_{j in K_i} v_j v_j^T (packed, P =
// r(r+1)/2 entries), b_i = sum_{j in K_i} y_ij v_j and |K_i|.  N_i and |K_i|
// are one dense product over all rows:
//     [N_flat | |K|] (m x (P+1)) = W (m x n, 0/1) x Kw (n x (P+1)),
// Kw[j] = (v_ja v_jb for a <= b, 1).  W is exact in TF32, so Kw is split into
// a TF32 head and an FP32 tail (Kw = hi + lo, the tail's own truncation leaves
// ~2^-22 relative) and the product runs as two tcgen05.mma kind::tf32 passes
// accumulating in FP32 in tensor memory.  b_i (r values) runs on the CUDA cores
// in the same pass over Y (r FMAs per known entry).
//
// A CTA owns 128 rows (the MMA M); it walks the columns in chunks of 32 with a
// two-stage ring in shared memory: the threads build the chunk's W tile from
// the mask words (one thread per row) and copy the chunk's pre-laid-out B tiles
// (Kw hi / lo) while the tensor core works on the previous chunk; one thread
// issues the MMAs and commits them to the stage's mbarrier, which the threads
// wait on before refilling that stage.  Operands use the canonical K-major
// layout without swizzle: 8-row x 16-byte core matrices, 128 bytes each,
// 8-row groups 128 B apart (SBO), K-adjacent core matrices LBO apart.
//
// Every mbarrier wait is bounded; on expiry the CTA flags the problem
// (counters[6]), waits (bounded) for its last commit, frees its tensor memory
// and returns.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "refine.cuh"

namespace rsm {

namespace {

constexpr int kRows = 128;      // MMA M: rows per CTA
constexpr int kChunkK = 32;     // columns per stage
constexpr int kThreads = 128;
constexpr int kMaxStages = 3;  // shared-memory ring: chunk c + 1 is copied in while chunk c is built
constexpr uint32_t kWaitLimit = 1u << 26;  // polls of one mbarrier wait before giving up


// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait for completion `parity` of the barrier; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's lane (warp w reads lanes 32 w .. 32 w + 31).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D tiled TMA load of the box at coordinates (x, y) (x innermost) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The descriptors were written to global memory through the generic proxy (by an earlier kernel).
__device__ __forceinline__ void tensormap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// Barrier 1 over the 128 row threads (the copy warp does not take part); the
// second form returns whether pred held in any of them.
__device__ __forceinline__ void rows_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ bool rows_sync_or(bool pred) {
  uint32_t out;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 128, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(out)
      : "r"((uint32_t)pred)
      : "memory");
  return out != 0;
}

}  // namespace

// Bytes of one stage: W tile, Kw hi and lo tiles, the chunk's V (RB per column), mask words.
__host__ __device__ constexpr size_t tc_stage_bytes(int npad, int rb) {
  return (size_t)kRows * kChunkK * 4 + (size_t)2 * npad * kChunkK * 4 + (size_t)kChunkK * rb * 4 + kChunkK * 4 * 4;
}

// Columns of tensor memory for an N of npad (a power of two, at least 32).
__host__ __device__ inline int tc_tmem_cols(int npad) {
  int c = 32;
  while (c < npad) c <<= 1;
  return c;
}

// B operand image of every chunk, in the shared-memory layout (K-major, no
// swizzle): chunk c holds Kw hi then Kw lo for columns 32 c .. 32 c + 31,
// entry (q, jj) at (jj / 4) (npad 16) + (q / 8) 128 + (q % 8) 16 + (jj % 4) 4
// bytes; then V in FP32 (n_pad x RB).  Kw column q < P: v_a v_b (pair q), q = P: 1.
__global__ void __launch_bounds__(256) k_build_B_tc(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ off,
                                                   int nprob) {
  pdl_enter();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= off[nprob]) return;
  const int p = find_problem(off, nprob, g);
  const ProbDesc& d = descs[p];
  const int r = d.r, P = r * (r + 1) / 2, npad = d.tc_npad, rb = d.tc_rb;
  const int n_pad = (int)((d.n + kChunkK - 1) / kChunkK) * kChunkK;
  const int e = (int)(g - off[p]);  // over n_pad x (npad + rb)
  const int j = e / (npad + rb), q = e % (npad + rb);
  float* img = reinterpret_cast<float*>(d.Kmat);
  if (q < npad) {
    double v = 0.0;
    if (j < d.n) {
      if (q < P) {
        int a = 0, rem = q;
        while (rem >= r - a) {
          rem -= r - a;
          ++a;
        }
        const int b = a + rem;
        v = d.V[(int64_t)a * d.ldv + j] * d.V[(int64_t)b * d.ldv + j];
      } else if (q == P) {
        v = 1.0;
      }
    }
    const float x = (float)v;
    const float hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);  // TF32 head (low 13 bits cleared)
    const float lo = x - hi;
    const int c = j / kChunkK, jj = j % kChunkK;
    float* base = img + (size_t)c * 2 * npad * kChunkK;
    const int o = (jj >> 2) * (npad * 4) + (q >> 3) * 32 + (q & 7) * 4 + (jj & 3);  // in floats
    base[o] = hi;
    base[npad * kChunkK + o] = lo;
  } else {
    const int a = q - npad;
    float* vf = img + (size_t)n_pad * 2 * npad;
    vf[(size_t)j * rb + a] = (j < d.n && a < r) ? (float)d.V[(int64_t)a * d.ldv + j] : 0.f;
  }
}

// Epilogue of the tensor-core normal equations, threads 0..127 (thread = row
// i0 + tid): read [N_i | |K_i|] out of tensor memory; for r <= 8 solve the r x r
// system right here, else hand N_i, b_i and |K_i| to the FP64 table.  scratch:
// 128 x 37 floats of shared memory that no copy or MMA still touches.
template <int RB>
__device__ __forceinline__ void tc_epilogue(const ProbDesc& d, int p, uint32_t tmem, unsigned char* scratch,
                                            uint32_t row, bool row_in, const float (&bacc)[RB],
                                            unsigned long long* __restrict__ fail_list,
                                            unsigned long long* __restrict__ fail_count) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = d.r, P = r * (r + 1) / 2, npad = d.tc_npad;
  if (RB == 8) {
    // r <= 8: solve the r x r system of this row right here.  N_i and b_i come
    // out of the FP32 accumulation; the Cholesky factorisation and the two
    // triangular solves run in FP64.  N_i goes through shared memory (the stages
    // are idle now) so the packed index can depend on r.
    float* nsm = reinterpret_cast<float*>(scratch) + tid * 37;
    float cnt = 0.f;
    for (int cb = 0; cb < npad; cb += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int q = cb + k;
        if (q < P) nsm[q] = v[k];
        if (q == P) cnt = v[k];
      }
    }
    double L[36], u[8];
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (a >= r) break;
#pragma unroll
      for (int b = 0; b <= a; ++b) L[a * (a + 1) / 2 + b] = (double)nsm[b * r - b * (b - 1) / 2 + (a - b)];
      tr += L[a * (a + 1) / 2 + a];
    }
    // a pivot below 1e-6 trace(N_i) is not resolved by the FP32-accumulated N_i:
    // such rows take the minimum-norm path
    bool ok = cnt >= (float)r;
    double rdiag[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j >= r || !ok) break;
      double v = L[j * (j + 1) / 2 + j];
#pragma unroll
      for (int t = 0; t < j; ++t) v = fma(-L[j * (j + 1) / 2 + t], L[j * (j + 1) / 2 + t], v);
      if (!(v > 1e-6 * tr)) {
        ok = false;
        break;
      }
      const double iv = rsqrt64(v);
      rdiag[j] = iv;
      L[j * (j + 1) / 2 + j] = v * iv;
#pragma unroll
      for (int k = j + 1; k < 8; ++k) {
        if (k >= r) break;
        double w = L[k * (k + 1) / 2 + j];
#pragma unroll
        for (int t = 0; t < j; ++t) w = fma(-L[k * (k + 1) / 2 + t], L[j * (j + 1) / 2 + t], w);
        L[k * (k + 1) / 2 + j] = w * iv;
      }
    }
    if (row_in) {
      if (ok) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {  // C y = b
          if (a >= r) break;
          double v = (double)bacc[a];
#pragma unroll
          for (int t = 0; t < a; ++t) v = fma(-L[a * (a + 1) / 2 + t], u[t], v);
          u[a] = v * rdiag[a];
        }
#pragma unroll
        for (int a = 7; a >= 0; --a) {  // C^T u = y
          if (a >= r) continue;
          double v = u[a];
#pragma unroll
          for (int t = a + 1; t < 8; ++t)
            if (t < r) v = fma(-L[t * (t + 1) / 2 + a], u[t], v);
          u[a] = v * rdiag[a];
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < r) d.U[(int64_t)a * d.ldu + row] = u[a];
        // the factor, for the refinement step of the residual pass
        float* lf = d.Lf + (size_t)row * P;
#pragma unroll
        for (int q = 0; q < 36; ++q)
          if (q < P) lf[q] = (float)L[q];
      } else {
        d.Lf[(size_t)row * P] = -1.f;  // no refinement: the minimum-norm path owns this row
        // too few known entries or a (numerically) singular N_i: hand the row to the
        // minimum-norm path with its data in the FP64 table
        double* out = d.NB + (size_t)row * d.q_pad;
        for (int q = 0; q < P; ++q) out[q] = (double)nsm[q];
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < r) out[P + a] = (double)bacc[a];
        out[P + r] = (double)cnt;
        if (cnt < (float)r) atomicAdd(&d.counters[4], 1ull);
        const unsigned long long slot = atomicAdd(fail_count, 1ull);
        fail_list[slot] = ((unsigned long long)p << 32) | (unsigned long long)row;
      }
    }
  } else {
    // tensor-memory loads are warp-wide: every lane loads, only rows < m store
    double* out = d.NB + (size_t)(row_in ? row : 0) * d.q_pad;
    for (int cb = 0; cb < npad; cb += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (row_in) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int q = cb + k;
          if (q < P)
            out[q] = (double)v[k];
          else if (q == P)
            out[P + r] = (double)v[k];  // |K_i|
        }
      }
    }
    if (row_in) {
#pragma unroll
      for (int a = 0; a < RB; ++a)
        if (a < r) out[P + a] = (double)bacc[a];
    }
  }
}

template <int RB>
__global__ void __launch_bounds__(kThreads) k_normal_tc(const ProbDesc* __restrict__ descs,
                                                       const int64_t* __restrict__ off, int nprob,
                                                       unsigned long long* __restrict__ fail_list,
                                                       unsigned long long* __restrict__ fail_count, int nstage) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long bars[kMaxStages];
  __shared__ uint32_t tmem_slot;
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npad = d.tc_npad;
  const int ncols = tc_tmem_cols(npad);
  const uint32_t m = (uint32_t)d.m, n = (uint32_t)d.n;
  const uint32_t i0 = (uint32_t)(blockIdx.x - off[p]) * kRows;
  const uint32_t row = i0 + tid;
  const bool row_in = row < m;
  const int nchunk = (int)((n + kChunkK - 1) / kChunkK);
  const size_t a_bytes = (size_t)kRows * kChunkK * 4, b_bytes = (size_t)npad * kChunkK * 4;
  const size_t stage_bytes = tc_stage_bytes(npad, RB);
  const float* img = reinterpret_cast<const float*>(d.Kmat);
  const float* vf = img + (size_t)nchunk * kChunkK * 2 * npad;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < nstage; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = idesc_tf32(npad);
  const uint32_t ldy = (uint32_t)d.ldy, ldb = (uint32_t)d.ldb;
  const float* Y = static_cast<const float*>(d.Y);

  float bacc[RB];
#pragma unroll
  for (int a = 0; a < RB; ++a) bacc[a] = 0.f;
  float ypre[kChunkK];
  auto load_y = [&](int c) {
#pragma unroll
    for (int jj = 0; jj < kChunkK; ++jj) {
      const uint32_t j = (uint32_t)c * kChunkK + jj;
      ypre[jj] = (row_in && j < n) ? __ldg(Y + (j * ldy + row)) : 0.f;
    }
  };
  // the mask words, Kw tiles and V of a chunk go straight to their stage by cp.async
  auto issue_copies = [&](int c) {
    unsigned char* st = tc_smem + (size_t)(c % nstage) * stage_bytes;
    const uint32_t bs = smem_u32(st + a_bytes), vs = smem_u32(st + a_bytes + 2 * b_bytes);
    const uint32_t ws = smem_u32(st + a_bytes + 2 * b_bytes + (size_t)kChunkK * RB * 4);
    const uint32_t j = (uint32_t)c * kChunkK + (tid >> 2);  // word tid % 4 of column tid / 4
    const uint32_t* wsrc = j < n ? d.bits + (j * ldb + (i0 >> 5) + (tid & 3)) : d.bits;
    cp_async4(ws + 4u * tid, wsrc, j < n ? 4u : 0u);
    const float4* src = reinterpret_cast<const float4*>(img + (size_t)c * 2 * npad * kChunkK);
    for (int e = tid; e < 2 * npad * kChunkK / 4; e += kThreads) cp_async16(bs + 16u * e, src + e);
    const float4* vsrc = reinterpret_cast<const float4*>(vf + (size_t)c * kChunkK * RB);
    for (int e = tid; e < kChunkK * RB / 4; e += kThreads) cp_async16(vs + 16u * e, vsrc + e);
    cp_async_commit();
  };
  load_y(0);
  if (nchunk > 0) issue_copies(0);
  bool failed = false;
  for (int c = 0; c < nchunk; ++c) {
    const int s = c % nstage;
    unsigned char* st = tc_smem + (size_t)s * stage_bytes;
    float* As = reinterpret_cast<float*>(st);
    float* Bs = reinterpret_cast<float*>(st + a_bytes);
    float* Vs = reinterpret_cast<float*>(st + a_bytes + 2 * b_bytes);
    uint32_t* Ws = reinterpret_cast<uint32_t*>(st + a_bytes + 2 * b_bytes + (size_t)kChunkK * RB * 4);
    if (c + 1 < nchunk) {
      // stage of chunk c + 1 was last read by the MMAs of chunk c + 1 - nstage
      if (c + 1 >= nstage && !failed)
        failed = !mbar_wait(smem_u32(&bars[(c + 1) % nstage]), (uint32_t)((c + 1 - nstage) / nstage) & 1u);
      issue_copies(c + 1);
      cp_async_wait<1>();  // this thread's copies of chunk c have landed
    } else {
      cp_async_wait<0>();
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    // W tile (thread = row): 8 core-matrix columns of 4 values; and b_i on the CUDA cores
    {
      float w[kChunkK];
#pragma unroll
      for (int jj = 0; jj < kChunkK; ++jj) w[jj] = (float)((Ws[jj * 4 + (tid >> 5)] >> lane) & 1u);
      float4* arow = reinterpret_cast<float4*>(As) + (tid >> 3) * 8 + (tid & 7);
#pragma unroll
      for (int kc = 0; kc < kChunkK / 4; ++kc)
        arow[kc * (kRows * 4 / 4)] = make_float4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
#pragma unroll
      for (int jj = 0; jj < kChunkK; ++jj) {
        const float yw = w[jj] != 0.f ? ypre[jj] : 0.f;
        const float4* vrow = reinterpret_cast<const float4*>(Vs + jj * RB);
#pragma unroll
        for (int a4 = 0; a4 < RB / 4; ++a4) {
          const float4 v = vrow[a4];
          bacc[4 * a4] = fmaf(yw, v.x, bacc[4 * a4]);
          bacc[4 * a4 + 1] = fmaf(yw, v.y, bacc[4 * a4 + 1]);
          bacc[4 * a4 + 2] = fmaf(yw, v.z, bacc[4 * a4 + 2]);
          bacc[4 * a4 + 3] = fmaf(yw, v.w, bacc[4 * a4 + 3]);
        }
      }
    }
    if (c + 1 < nchunk) load_y(c + 1);
    proxy_fence();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const uint32_t a_lbo = kRows * 16, b_lbo = (uint32_t)npad * 16;
#pragma unroll
      for (int ks = 0; ks < kChunkK / 8; ++ks) {  // K = 8 per instruction: two core matrices along K
        const uint64_t ad = smem_desc(a0 + ks * 2 * a_lbo, a_lbo, 128);
        const uint64_t bh = smem_desc(b0 + ks * 2 * b_lbo, b_lbo, 128);
        const uint64_t bl = smem_desc(b0 + (uint32_t)b_bytes + ks * 2 * b_lbo, b_lbo, 128);
        tc_mma_tf32(tmem, ad, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
        tc_mma_tf32(tmem, ad, bl, idesc, 1u);
      }
      tc_commit(smem_u32(&bars[s]));
    }
  }
  // the last commit covers every MMA issued before it
  if (nchunk > 0 && !failed) {
    const int c = nchunk - 1;
    if (!mbar_wait(smem_u32(&bars[c % nstage]), (uint32_t)(c / nstage) & 1u)) failed = true;
  }
  cp_async_wait<0>();  // nothing of this thread's may still be landing when the CTA ends
  failed = __syncthreads_or(failed) != 0;  // the same decision in every thread
  tc_fence_after();
  if (failed) {
    if (tid == 0) atomicAdd(&d.counters[6], 1ull);
  } else {
    tc_epilogue<RB>(d, p, tmem, tc_smem, row, row_in, bacc, fail_list, fail_count);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// The same product with TMA: a copy warp streams each chunk's Y tile (128 rows
// x 32 columns, tensor map over the caller's column-major Y), its mask words
// (tensor map over the packed mask) and its B images (bulk copies) into a ring
// of stages, each completing one mbarrier by transaction count; the 128 row
// threads wait on it, read their row's 32 values and mask bits, accumulate b_i,
// then write the W tile over the Y tile they have read (K-major core matrices),
// and thread 0 issues the MMAs, whose commit frees the stage for the copy warp.
// Stage layout: [Y tile, then W tile: 16 KB | Kw hi, lo | V (32 x RB) | mask 4 x 32 words].
__host__ __device__ constexpr size_t tma_stage_bytes(int npad, int rb) {
  return (size_t)kRows * kChunkK * 4 + (size_t)2 * npad * kChunkK * 4 + (size_t)kChunkK * rb * 4 + kChunkK * 4 * 4;
}
constexpr int kTmaThreads = kRows + 32;

template <int RB>
__global__ void __launch_bounds__(kTmaThreads) k_normal_tma(const ProbDesc* __restrict__ descs,
                                                           const int64_t* __restrict__ off, int nprob,
                                                           unsigned long long* __restrict__ fail_list,
                                                           unsigned long long* __restrict__ fail_count, int nstage) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char tma_smem_raw[];
  __shared__ __align__(8) unsigned long long full[kMaxStages], empty[kMaxStages];
  __shared__ uint32_t tmem_slot;
  // TMA destinations: 128-byte aligned
  unsigned char* smem = tma_smem_raw + ((128u - (smem_u32(tma_smem_raw) & 127u)) & 127u);
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npad = d.tc_npad;
  const int ncols = tc_tmem_cols(npad);
  const uint32_t m = (uint32_t)d.m, n = (uint32_t)d.n;
  const uint32_t i0 = (uint32_t)(blockIdx.x - off[p]) * kRows;
  const uint32_t row = i0 + (uint32_t)tid;
  const bool row_in = tid < kRows && row < m;
  const int nchunk = (int)((n + kChunkK - 1) / kChunkK);
  const uint32_t a_bytes = kRows * kChunkK * 4, b_bytes = (uint32_t)npad * kChunkK * 4;
  const uint32_t v_bytes = kChunkK * RB * 4, w_bytes = kChunkK * 4 * 4;
  const uint32_t stage_bytes = (uint32_t)tma_stage_bytes(npad, RB);
  const float* img = reinterpret_cast<const float*>(d.Kmat);
  const float* vf = img + (size_t)nchunk * kChunkK * 2 * npad;
  const unsigned char* tmaps = static_cast<const unsigned char*>(d.tmap);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < nstage; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool failed = false;
  float bacc[RB];
#pragma unroll
  for (int a = 0; a < RB; ++a) bacc[a] = 0.f;

  if (warp == kRows / 32) {
    // copy warp: one lane issues every copy of every chunk
    if (lane == 0) {
      tensormap_acquire(tmaps);
      tensormap_acquire(tmaps + 128);
      int issued = 0;
      for (int c = 0; c < nchunk; ++c) {
        const int s = c % nstage;
        // stage s was last read by the MMAs of chunk c - nstage
        if (c >= nstage && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(c / nstage - 1) & 1u)) {
          failed = true;
          break;
        }
        const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
        const uint32_t bar = smem_u32(&full[s]);
        mbar_expect_tx(bar, a_bytes + 2 * b_bytes + v_bytes + w_bytes);
        tma_load_2d(st, tmaps, (int)i0, c * kChunkK, bar);
        bulk_load(st + a_bytes, img + (size_t)c * 2 * npad * kChunkK, 2 * b_bytes, bar);
        bulk_load(st + a_bytes + 2 * b_bytes, vf + (size_t)c * kChunkK * RB, v_bytes, bar);
        tma_load_2d(st + a_bytes + 2 * b_bytes + v_bytes, tmaps + 128, (int)(i0 >> 5), c * kChunkK, bar);
        issued = c + 1;
      }
      // nothing may still be landing when the CTA ends: wait (bounded) for the
      // last use of every stage (already complete unless something failed)
      for (int c = issued - 1; c >= 0 && c >= issued - nstage; --c)
        mbar_wait(smem_u32(&full[c % nstage]), (uint32_t)(c / nstage) & 1u);
    }
  } else {
    for (int c = 0; c < nchunk; ++c) {
      const int s = c % nstage;
      const bool ok = mbar_wait(smem_u32(&full[s]), (uint32_t)(c / nstage) & 1u);
      if (rows_sync_or(!ok)) {
        failed = true;
        break;
      }
      unsigned char* st = smem + (size_t)s * stage_bytes;
      float* As = reinterpret_cast<float*>(st);
      const float* Vs = reinterpret_cast<const float*>(st + a_bytes + 2 * b_bytes);
      const uint32_t* Ws = reinterpret_cast<const uint32_t*>(st + a_bytes + 2 * b_bytes + v_bytes);
      float w[kChunkK];
      {
        float y[kChunkK];
#pragma unroll
        for (int jj = 0; jj < kChunkK; ++jj) {
          y[jj] = As[jj * kRows + tid];  // the TMA box: 32 columns of 128 rows
          w[jj] = (float)((Ws[jj * 4 + (tid >> 5)] >> lane) & 1u);
        }
#pragma unroll
        for (int jj = 0; jj < kChunkK; ++jj) {
          const float yw = w[jj] != 0.f ? y[jj] : 0.f;
          const float4* vrow = reinterpret_cast<const float4*>(Vs + jj * RB);
#pragma unroll
          for (int a4 = 0; a4 < RB / 4; ++a4) {
            const float4 v = vrow[a4];
            bacc[4 * a4] = fmaf(yw, v.x, bacc[4 * a4]);
            bacc[4 * a4 + 1] = fmaf(yw, v.y, bacc[4 * a4 + 1]);
            bacc[4 * a4 + 2] = fmaf(yw, v.z, bacc[4 * a4 + 2]);
            bacc[4 * a4 + 3] = fmaf(yw, v.w, bacc[4 * a4 + 3]);
          }
        }
      }
      rows_sync();  // every row thread has read the Y tile: overwrite it with the W tile
      float4* arow = reinterpret_cast<float4*>(As) + (tid >> 3) * 8 + (tid & 7);
#pragma unroll
      for (int kc = 0; kc < kChunkK / 4; ++kc)
        arow[kc * (kRows * 4 / 4)] = make_float4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
      proxy_fence();
      rows_sync();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(As), b0 = a0 + a_bytes;
        const uint32_t a_lbo = kRows * 16, b_lbo = (uint32_t)npad * 16;
        const uint32_t idesc = idesc_tf32(npad);
#pragma unroll
        for (int ks = 0; ks < kChunkK / 8; ++ks) {
          const uint64_t ad = smem_desc(a0 + ks * 2 * a_lbo, a_lbo, 128);
          const uint64_t bh = smem_desc(b0 + ks * 2 * b_lbo, b_lbo, 128);
          const uint64_t bl = smem_desc(b0 + b_bytes + ks * 2 * b_lbo, b_lbo, 128);
          tc_mma_tf32(tmem, ad, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
          tc_mma_tf32(tmem, ad, bl, idesc, 1u);
        }
        tc_commit(smem_u32(&empty[s]));
      }
    }
    // the last commit covers every MMA issued before it
    if (tid == 0 && nchunk > 0 && !failed) {
      const int c = nchunk - 1;
      if (!mbar_wait(smem_u32(&empty[c % nstage]), (uint32_t)(c / nstage) & 1u)) failed = true;
    }
  }
  failed = __syncthreads_or(failed) != 0;  // the same decision in every thread
  tc_fence_after();
  if (failed) {
    if (tid == 0) atomicAdd(&d.counters[6], 1ull);
  } else if (tid < kRows) {
    tc_epilogue<RB>(d, p, tmem, smem, row, row_in, bacc, fail_list, fail_count);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ------------------------------------------------------------------ a9: the residual pass, TMA-fed
// e numerator sum_{known} (y_ij - u_i . v_j)^2 and, with `refine`, the
// refinement step of U (refine_row) for the FP32 form with r <= 8.  A CTA
// takes the same 128-row tile as k_normal_tma (thread = row, so c_i = V_K^T r0
// stays in the thread): the copy warp streams each 32-column chunk's Y tile
// and mask words (the same tensor maps) and the chunk's V rows (bulk copy of
// the FP32 V image) into a ring of stages; the row threads wait on the stage's
// mbarrier, accumulate, and release the stage through a second mbarrier (one
// arrival per warp).  Per chunk the FP32 sum of squares is added into an FP64
// running sum; the CTA's sum goes to its two slots of the 64-row partials.
__host__ __device__ constexpr size_t res_stage_bytes(int rb) {
  return (size_t)kRows * kChunkK * 4 + (size_t)kChunkK * rb * 4 + kChunkK * 4 * 4;
}
constexpr int kResStages = 4;

template <int RB>
__global__ void __launch_bounds__(kTmaThreads, 3) k_residual_tma(const ProbDesc* __restrict__ descs,
                                                             const int64_t* __restrict__ off,
                                                             const int64_t* __restrict__ resv_off, int nprob,
                                                             double* __restrict__ partial, int refine) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char res_smem_raw[];
  __shared__ __align__(8) unsigned long long full[kResStages], empty[kResStages];
  __shared__ double red[kRows / 32];
  unsigned char* smem = res_smem_raw + ((128u - (smem_u32(res_smem_raw) & 127u)) & 127u);
  const int p = find_problem(off, nprob, blockIdx.x);
  const ProbDesc& d = descs[p];
  // a tensor-core problem without the vectorised residual (the scalar kernel has
  // it), or with r > 8 (the 2-row kernel at RM = 16 has it)
  if (!d.resv || d.r > 8) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t m = (uint32_t)d.m, n = (uint32_t)d.n;
  const uint32_t tile = (uint32_t)(blockIdx.x - off[p]);
  const uint32_t i0 = tile * kRows;
  const uint32_t row = i0 + (uint32_t)tid;
  const bool row_in = tid < kRows && row < m;
  const int nchunk = (int)((n + kChunkK - 1) / kChunkK);
  const uint32_t y_bytes = kRows * kChunkK * 4, v_bytes = kChunkK * RB * 4, w_bytes = kChunkK * 4 * 4;
  const uint32_t stage_bytes = (uint32_t)res_stage_bytes(RB);
  const unsigned char* tmaps = static_cast<const unsigned char*>(d.tmap);
  if (tid == 0) {
    for (int k = 0; k < kResStages; ++k) {
      mbar_init(smem_u32(&full[k]), 1);
      mbar_init(smem_u32(&empty[k]), kRows / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool failed = false;
  double dacc = 0.0;
  if (warp == kRows / 32) {
    if (lane == 0) {  // copy warp
      tensormap_acquire(tmaps);
      tensormap_acquire(tmaps + 128);
      int issued = 0;
      for (int c = 0; c < nchunk; ++c) {
        const int s = c % kResStages;
        if (c >= kResStages && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(c / kResStages - 1) & 1u)) {
          failed = true;
          break;
        }
        const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
        const uint32_t bar = smem_u32(&full[s]);
        mbar_expect_tx(bar, y_bytes + v_bytes + w_bytes);
        tma_load_2d(st, tmaps, (int)i0, c * kChunkK, bar);
        bulk_load(st + y_bytes, d.vf32 + (size_t)c * kChunkK * RB, v_bytes, bar);
        tma_load_2d(st + y_bytes + v_bytes, tmaps + 128, (int)(i0 >> 5), c * kChunkK, bar);
        issued = c + 1;
      }
      for (int c = issued - 1; c >= 0 && c >= issued - kResStages; --c)
        mbar_wait(smem_u32(&full[c % kResStages]), (uint32_t)(c / kResStages) & 1u);
    }
  } else {
    const int r = d.r;
    float u[8], cacc[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      u[a] = (row_in && a < r) ? (float)d.U[(int64_t)a * d.ldu + row] : 0.f;
      cacc[a] = 0.f;
    }
    for (int c = 0; c < nchunk; ++c) {
      const int s = c % kResStages;
      if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(c / kResStages) & 1u)) {
        failed = true;
        break;
      }
      const unsigned char* st = smem + (size_t)s * stage_bytes;
      const float* Ys = reinterpret_cast<const float*>(st);
      const float* Vs = reinterpret_cast<const float*>(st + y_bytes);
      const uint32_t* Ws = reinterpret_cast<const uint32_t*>(st + y_bytes + v_bytes);
      float ch = 0.f;
#pragma unroll 8
      for (int jj = 0; jj < kChunkK; ++jj) {
        const float y = Ys[jj * kRows + tid];
        const bool known = row_in && ((Ws[jj * 4 + (tid >> 5)] >> lane) & 1u);
        const float4 va = *reinterpret_cast<const float4*>(Vs + jj * RB);
        const float4 vb = *reinterpret_cast<const float4*>(Vs + jj * RB + 4);
        const float v[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        float pr = 0.f;
#pragma unroll
        for (int a = 0; a < 8; ++a) pr = fmaf(u[a], v[a], pr);
        const float diff = known ? y - pr : 0.f;
        ch = fmaf(diff, diff, ch);
#pragma unroll
        for (int a = 0; a < 8; ++a) cacc[a] = fmaf(diff, v[a], cacc[a]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
      dacc += (double)ch;
    }
    if (!failed && refine && row_in) dacc -= refine_row<8>(d, row, u, cacc);
  }
  failed = __syncthreads_or(failed) != 0;
  if (failed) {
    if (tid == 0) atomicAdd(&d.counters[6], 1ull);
    dacc = 0.0;
  }
  if (tid < kRows) {
#pragma unroll
    for (int o = 16; o; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if (lane == 0) red[warp] = dacc;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int k = 0; k < kRows / 32; ++k) t += red[k];
    const int64_t slot = resv_off[p] + 2 * (int64_t)tile;  // the 64-row slots of this tile
    partial[slot] = t;
    if (slot + 1 < resv_off[p + 1]) partial[slot + 1] = 0.0;
  }
}

cudaError_t launch_residual_tma(const SolvePlan& S, double* partial, int refine, cudaStream_t s) {
  if (S.tc_tiles <= 0) return cudaSuccess;
  const size_t smem = kResStages * res_stage_bytes(S.tc_rb) + 128;
  cudaError_t e;
#define RSM_RTMA(RB)                                                                                              \
  do {                                                                                                            \
    if ((e = cudaFuncSetAttribute(k_residual_tma<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != \
        cudaSuccess) {                                                                                            \
      cudaGetLastError();                                                                                         \
      return e;                                                                                                   \
    }                                                                                                             \
    (void)launch_chained(k_residual_tma<RB>, (unsigned)S.tc_tiles, kTmaThreads, smem, s, S.descs, S.tc_off,        \
                         S.resv_off, S.nprob, partial, refine);                                               \
  } while (0)
  if (S.tc_rb <= 8)
    RSM_RTMA(8);
  else if (S.tc_rb <= 16)
    RSM_RTMA(16);
  else
    RSM_RTMA(24);
#undef RSM_RTMA
  ++g_kernel_launches;
  return cudaGetLastError();
}

bool normal_tc_supported(int r) { return r >= 1 && r <= 21; }

int normal_tc_rb(int r) { return r <= 8 ? 8 : r <= 16 ? 16 : 24; }
int normal_tc_npad(int r) { return ((r * (r + 1) / 2 + 1) + 15) / 16 * 16; }

cudaError_t launch_normal_tc(const SolvePlan& S, int rb_max, int npad_max, cudaStream_t s) {
  const ProbDesc* D = S.descs;
  const int np = S.nprob;
  cudaError_t e;
  if (S.b_total > 0) {
    (void)launch_chained(k_build_B_tc, (unsigned)((S.b_total + 255) / 256), 256, 0, s, D, S.b_off, np);
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (S.tc_tiles <= 0) return cudaSuccess;
  if (S.tc_tma) {
    // two stages, so that three CTAs fit per SM: their warps hide the FP64 epilogue
    // of the others
    const size_t st = tma_stage_bytes(npad_max, rb_max);
    const int stages = 2;
    const size_t smem = stages * st + 128;
#define RSM_TMA(RB)                                                                                             \
  do {                                                                                                          \
    if ((e = cudaFuncSetAttribute(k_normal_tma<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != \
        cudaSuccess) {                                                                                          \
      cudaGetLastError();                                                                                       \
      return e;                                                                                                 \
    }                                                                                                           \
    (void)launch_chained(k_normal_tma<RB>, (unsigned)S.tc_tiles, kTmaThreads, smem, s, D, S.tc_off, np,         \
                         S.fail_list, S.fail_count, stages);                                                  \
  } while (0)
    if (rb_max <= 8)
      RSM_TMA(8);
    else if (rb_max <= 16)
      RSM_TMA(16);
    else
      RSM_TMA(24);
#undef RSM_TMA
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  // three stages when they fit in shared memory (227 KB per CTA), else two
  const int stages = 3 * tc_stage_bytes(npad_max, rb_max) <= 232448 ? 3 : 2;
  const size_t smem = stages * tc_stage_bytes(npad_max, rb_max);
#define RSM_TC(RB)                                                                                             \
  do {                                                                                                         \
    if ((e = cudaFuncSetAttribute(k_normal_tc<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != \
        cudaSuccess) {                                                                                         \
      cudaGetLastError();                                                                                      \
      return e;                                                                                                \
    }                                                                                                          \
    (void)launch_chained(k_normal_tc<RB>, (unsigned)S.tc_tiles, kThreads, smem, s, D, S.tc_off, np, S.fail_list, \
                         S.fail_count, stages);                                                                \
  } while (0)
  if (rb_max <= 8)
    RSM_TC(8);
  else if (rb_max <= 16)
    RSM_TC(16);
  else
    RSM_TC(24);
#undef RSM_TC
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
