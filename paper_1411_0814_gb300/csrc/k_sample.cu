// Stage a1 (mask packing), a2 (column sampling) and the stand-alone row-list
// stage of a3 (the fused selection lives in k_gram.cu).
#include "common.cuh"
#include "kernels.h"

namespace rsm {

// ------------------------------------------------------------------ a1 pack_mask
// Section IV-A: extracting a submatrix needs only logical tests on W, so W is
// packed once into bit words: bit (i mod 32) of word i/32 of column c is
// W[i, c] != 0.  One thread per output word; a CTA covers 256 consecutive words
// of one column.  Blocks are flattened over the problems of the batch.
__device__ __forceinline__ void pack_mask_block(const ProbDesc* __restrict__ descs,
                                                const int64_t* __restrict__ blk_off, int nprob, int64_t block) {
  const int p = find_problem(blk_off, nprob, block);
  const ProbDesc& d = descs[p];
  const int64_t local = block - blk_off[p];
  const int64_t chunks = (d.ldb + 255) / 256;
  const int64_t c = local / chunks;
  const int64_t w = (local % chunks) * 256 + threadIdx.x;
  uint32_t word = 0;
  if (w < d.ldb) {
    const uint8_t* col = d.W + c * d.ldw;
    const int64_t r0 = w * 32;
    if (r0 + 32 <= d.m && ((reinterpret_cast<uintptr_t>(col + r0) & 15) == 0)) {
      const uint4* q = reinterpret_cast<const uint4*>(col + r0);
      uint4 a = __ldg(q), b = __ldg(q + 1);
      uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      // per 4 bytes: 0x01 in each nonzero byte, then the multiply by 0x01020408 moves byte i's bit
      // to bit 24 + i with no other product term reaching bits 24..27
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t ones = __vcmpne4(v[k], 0u) & 0x01010101u;
        word |= ((ones * 0x01020408u) >> 24) << (4 * k);
      }
    } else {
      for (int k = 0; k < 32; ++k)
        if (r0 + k < d.m && col[r0 + k]) word |= 1u << k;
    }
    d.bits[c * d.ldb + w] = word;
  }
  // known-entry count of the problem (eq. def.rho numerator), exact integer sum: one atomic per CTA
  __shared__ unsigned wcnt[8];
  unsigned cnt = __popc(word);
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < 8; ++k) t += wcnt[k];
    if (t) atomicAdd(&d.counters[1], t);
  }
}

__global__ void __launch_bounds__(256) k_pack_mask(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ blk_off,
                                                   int nprob) {
  pack_mask_block(descs, blk_off, nprob, blockIdx.x);
}

// ------------------------------------------------------------------ a2 sample_cols
// Section III, method M1: choose l distinct columns (Section II: a list <k> has
// distinct entries).  Word w of trial t is lane (w mod 4) of Philox4x32-10 with
// key (seed lo, seed hi) and counter (t lo, problem id, w / 4, t hi).  A draw in
// [0, k) is (word * k) >> 32.  RANDOM: Floyd's algorithm, draw d picks x in
// [0, n-l+d] and takes n-l+d instead when x is already chosen.  ADJACENT: a
// start s in [0, n-l] and columns s..s+l-1.  The set is sorted ascending.
// Method M2 (variant 2) draws its k rows the same way over [0, m).
__device__ __forceinline__ void draw_columns(const ProbDesc& d, int64_t t, int32_t* out) {
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  const int l = d.l;
  const int64_t n = d.variant == 2 ? d.m : d.n;
  int32_t c[kMaxL];
  if (d.variant == 1) {
    uint4 w = philox4x32_10(make_uint4((uint32_t)t, d.pid, 0u, (uint32_t)(t >> 32)), k0, k1);
    const int64_t s = (int64_t)__umulhi(w.x, (uint32_t)(n - l + 1));  // (x range) >> 32
    for (int k = 0; k < l; ++k) out[k] = (int32_t)(s + k);
    return;
  }
  uint4 blk = make_uint4(0, 0, 0, 0);
  for (int dd = 0; dd < l; ++dd) {
    if ((dd & 3) == 0)
      blk = philox4x32_10(make_uint4((uint32_t)t, d.pid, (uint32_t)(dd >> 2), (uint32_t)(t >> 32)), k0, k1);
    const uint32_t word = (dd & 3) == 0 ? blk.x : (dd & 3) == 1 ? blk.y : (dd & 3) == 2 ? blk.z : blk.w;
    const int32_t j = (int32_t)(n - l + dd);
    int32_t x = (int32_t)__umulhi(word, (uint32_t)(j + 1));  // multiply-shift draw in [0, j]
    bool taken = false;
    for (int e = 0; e < dd; ++e) taken |= (c[e] == x);
    c[dd] = taken ? (int32_t)j : x;
  }
  for (int a = 1; a < l; ++a) {  // insertion sort, l <= 32
    int32_t v = c[a];
    int b = a - 1;
    while (b >= 0 && c[b] > v) {
      c[b + 1] = c[b];
      --b;
    }
    c[b + 1] = v;
  }
  for (int k = 0; k < l; ++k) out[k] = c[k];
}

// One thread per trial, flattened over the problems of the batch.  Also counts
// how many trials drew each column (an upper bound of every entry of M, used to
// size the fixed-point accumulator).
__device__ __forceinline__ void sample_block(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ trial_off,
                                             int nprob, int64_t block) {
  const int64_t g = block * blockDim.x + threadIdx.x;
  if (g >= trial_off[nprob]) return;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t t = g - trial_off[p];
  int32_t* out = d.cols + t * d.l;
  draw_columns(d, t, out);
  int vmax = 0;
  if (d.variant != 2)  // the row variant counts its columns when it selects them (k_m2_trial)
    for (int k = 0; k < d.l; ++k) vmax = max(vmax, atomicAdd(&d.colcount[out[k]], 1) + 1);
  // one atomic per warp and problem for the largest column count (lanes of a warp may
  // belong to two problems of a batch: reduce among the lanes of the same problem)
  const unsigned same = __match_any_sync(__activemask(), p);
  const int wmax = __reduce_max_sync(same, vmax);
  if ((threadIdx.x & 31) == __ffs(same) - 1) atomicMax(&d.counters[2], (unsigned long long)wmax);
  if (d.debug_cols)
    for (int k = 0; k < d.l; ++k) d.debug_cols[t * d.l + k] = out[k];
}

__global__ void __launch_bounds__(256) k_sample(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ trial_off,
                                                int nprob) {
  sample_block(descs, trial_off, nprob, blockIdx.x);
}

// Stages a1 and a2 in one launch: they are independent, so the sampler's blocks
// (first, a short latency-bound tail of Philox draws) run beside the packing's
// HBM-bound blocks instead of after them.
__global__ void __launch_bounds__(256) k_front(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ blk_off,
                                               const int64_t* __restrict__ trial_off, int nprob, int64_t sample_blocks) {
  if ((int64_t)blockIdx.x < sample_blocks)
    sample_block(descs, trial_off, nprob, blockIdx.x);
  else
    pack_mask_block(descs, blk_off, nprob, (int64_t)blockIdx.x - sample_blocks);
}

// Stand-alone sampler for the stage entry point: trials t0 .. t0+count-1 of one problem.
__global__ void __launch_bounds__(256) k_sample_range(ProbDesc d, int64_t t0, int64_t count, int32_t* cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  draw_columns(d, t0 + i, cols + i * d.l);
}

// ------------------------------------------------------------------ a3 row lists (stage entry)
// Section III, M1: R_t = rows known in every chosen column, ascending.  One CTA
// per trial; each thread ANDs the l mask words of one 32-row group, and a block
// scan places the rows in order.
__global__ void __launch_bounds__(256) k_select_rows(const uint32_t* __restrict__ bits, int64_t ldb, int64_t m,
                                                     const int32_t* __restrict__ cols, int l,
                                                     const int64_t* __restrict__ row_off, int32_t* __restrict__ rows,
                                                     int32_t* __restrict__ row_counts) {
  __shared__ int warp_sums[8];
  __shared__ int32_t cidx[kMaxL];
  const int64_t t = blockIdx.x;
  if (threadIdx.x < l) cidx[threadIdx.x] = cols[t * l + threadIdx.x];
  __syncthreads();
  const int64_t nwords = (m + 31) / 32;
  const int64_t cap = row_off[t + 1] - row_off[t];
  int32_t* out = rows + row_off[t];
  int64_t done = 0;
  for (int64_t w0 = 0; w0 < nwords; w0 += 256) {
    const int64_t w = w0 + threadIdx.x;
    uint32_t mask = 0;
    if (w < nwords) {
      mask = 0xffffffffu;
      for (int k = 0; k < l; ++k) mask &= bits[(int64_t)cidx[k] * ldb + w];
    }
    int total;
    int off = block_exclusive_scan<256>(__popc(mask), warp_sums, &total);
    int64_t rank = done + off;
    while (mask) {
      int b = __ffs(mask) - 1;
      mask &= mask - 1;
      if (rank < cap) out[rank] = (int32_t)(w * 32 + b);
      ++rank;
    }
    done += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) row_counts[t] = (int32_t)done;
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_pack_mask(const ProbDesc* descs, const int64_t* blk_off, int nprob, int64_t nblocks, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  k_pack_mask<<<(unsigned)nblocks, 256, 0, s>>>(descs, blk_off, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_front(const ProbDesc* descs, const int64_t* blk_off, int64_t pack_blocks, const int64_t* trial_off,
                         int64_t trials, int nprob, cudaStream_t s) {
  const int64_t sb = (trials + 255) / 256;
  if (sb + pack_blocks <= 0) return cudaSuccess;
  k_front<<<(unsigned)(sb + pack_blocks), 256, 0, s>>>(descs, blk_off, trial_off, nprob, sb);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_sample(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  k_sample<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(descs, trial_off, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_sample_range(const ProbDesc& d, int64_t t0, int64_t count, int32_t* cols, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_sample_range<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(d, t0, count, cols);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_select_rows(const uint32_t* bits, int64_t ldb, int64_t m, const int32_t* cols, int l, int64_t count,
                               const int64_t* row_off, int32_t* rows, int32_t* row_counts, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_select_rows<<<(unsigned)count, 256, 0, s>>>(bits, ldb, m, cols, l, row_off, rows, row_counts);
  ++g_kernel_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ known-entry count (trial planning)
// out += number of nonzero bytes of the column-major m x n mask W.
__global__ void __launch_bounds__(256) k_count_known(const uint8_t* __restrict__ W, int64_t ldw, int64_t m, int64_t n,
                                                    unsigned long long* __restrict__ out) {
  __shared__ unsigned long long red[8];
  unsigned long long c = 0;
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e - j * m;
    c += W[j * ldw + i] != 0;
  }
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < 8; ++k) t += red[k];
    atomicAdd(out, t);
  }
}

cudaError_t launch_count_known(const uint8_t* W, int64_t ldw, int64_t m, int64_t n, unsigned long long* out,
                               cudaStream_t s) {
  k_count_known<<<1216, 256, 0, s>>>(W, ldw, m, n, out);
  ++g_kernel_launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ coverage (Section III, Theorem 3)
// The known entries visited by the accepted draws of the column variants: for
// trial t and mask word w, the rows of that word known in every chosen column
// (the AND of the l mask words) are visited in each of the chosen columns.
// Grid: x = trial (flattened over the problems that count coverage), y = chunk
// of 256 words.  Only problems with a visited buffer take part.
__global__ void __launch_bounds__(256) k_visit(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ trial_off,
                                              int nprob) {
  const int64_t g = blockIdx.x;
  if (g >= trial_off[nprob]) return;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  if (!d.visited || d.variant == 2) return;  // the row variant records its visits in k_m2_trial
  const int64_t t = g - trial_off[p];
  const int l = d.l;
  if (d.row_counts[t] < l) return;  // rejected draw
  const uint32_t nw = (uint32_t)((d.m + 31) / 32), ldb = (uint32_t)d.ldb;
  const uint32_t w = blockIdx.y * 256u + threadIdx.x;
  if (w >= nw) return;
  const int32_t* cols = d.cols + t * l;
  uint32_t sel = 0xffffffffu;
  for (int k = 0; k < l; ++k) sel &= __ldg(d.bits + ((uint32_t)cols[k] * ldb + w));
  if (sel)
    for (int k = 0; k < l; ++k) atomicOr(d.visited + ((uint32_t)cols[k] * ldb + w), sel);
}

// counters[8] = number of visited entries (all of them known); one CTA per problem.
__global__ void __launch_bounds__(256) k_count_visited(const ProbDesc* __restrict__ descs, int nprob) {
  __shared__ unsigned long long red[8];
  const int p = blockIdx.x;
  if (p >= nprob) return;
  const ProbDesc& d = descs[p];
  if (!d.visited) return;
  const int64_t words = d.n * d.ldb;
  unsigned long long c = 0;
  for (int64_t e = threadIdx.x; e < words; e += 256) c += __popc(d.visited[e]);
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int k = 0; k < 8; ++k) tot += red[k];
    d.counters[8] = tot;
  }
}

cudaError_t launch_coverage(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t trials_total,
                            int64_t max_words, cudaStream_t s) {
  if (trials_total <= 0) return cudaSuccess;
  const unsigned chunks = (unsigned)((max_words + 255) / 256);
  k_visit<<<dim3((unsigned)trials_total, chunks), 256, 0, s>>>(descs, trial_off, nprob);
  ++g_kernel_launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_count_visited<<<nprob, 256, 0, s>>>(descs, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
