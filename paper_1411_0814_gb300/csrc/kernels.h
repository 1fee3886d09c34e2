// Host-side declarations of the kernel launchers (internal to librsm.so).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace rsm {

struct ProbDesc;

// Kernels launched by the calling thread (incremented by every launcher).
extern thread_local int64_t g_kernel_launches;

// Offsets of the eigen stage.  Every table is an exclusive prefix sum of
// nprob + 1 int64 values; dT is the device copy (read by kernels), hT the host
// copy (read by the launcher for grid sizes); both hold the same tables at the
// same positions.
struct EigPlan {
  const ProbDesc* descs;
  int nprob;
  int max_nblk;
  int kx_max;  // largest block width of the batch
  const int64_t* dT;
  const int64_t* hT;
  size_t pad2, step, linv, nk, mx, chunk, part_off, rot, row_tile;  // table positions (step: 2 per step, linv: 3 per step)
  size_t phase;   // task prefix over the 5 max_nblk + 3 kFactorLag segments of the factor launch
  double* part;   // partial Gram sums of the block iteration
  unsigned* sync; // factor launch: claim counter, abort word, per-phase completion counts (zeroed)
  bool fault_wait; // test injection: the factor launch's first wait has nothing to wait for
};

// Table positions read by the factor launch.
struct FactorTables {
  size_t step, linv, phase;
  int nsteps;  // largest block count of the batch
  int lag;     // steps by which the inverse-factor tasks trail the Cholesky tasks in claim order
  unsigned poll_limit;  // polls of one dependency wait before the launch is abandoned
  int fault_wait;       // test injection: the first chain step waits for sync[3], which nothing sets
};
constexpr int kFactorLag = 1;

struct SolvePlan {
  const ProbDesc* descs;
  int nprob;
  int64_t k_total;
  const int64_t* k_off;      // n * q_pad per problem
  int64_t tile_off_host_total;
  const int64_t* tile_off;   // ceil(m / 64) * q_pad / 64 per problem
  int64_t row_total;
  const int64_t* row_off;    // m per problem
  int64_t res_blocks;
  const int64_t* res_off;    // ceil(m / 32) per problem (scalar residual kernel)
  int64_t resv_blocks;
  const int64_t* resv_off;   // ceil(m / 64) per problem (2-row residual kernel); its partials follow the others
  int resv_rmax;             // largest r among those problems (<= 8: TMA-fed or 2-row kernel; else also RM = 16)
  int rmax;                  // largest r of the batch
  unsigned long long* fail_list;   // row_total entries: (problem << 32) | row
  unsigned long long* fail_count;  // zero before the launch
  // tensor-core normal equations (problems with tc set)
  int64_t b_total;
  const int64_t* b_off;      // n_pad * (tc_npad + tc_rb) per problem
  int64_t tc_tiles;
  const int64_t* tc_off;     // ceil(m / 128) per problem
  int tc_rb, tc_npad_max;
  bool tc_tma;               // every tensor-core problem has its TMA descriptors (ProbDesc::tmap)
  bool any_solve;
};
bool normal_tc_supported(int r);
int normal_tc_rb(int r);
int normal_tc_npad(int r);
// The residual pass (a9) with the refinement step of U for the problems with resv set, fed by
// TMA (every tensor-core problem's descriptors present: S.tc_tma); partial holds the resv slots.
cudaError_t launch_residual_tma(const SolvePlan& S, double* partial, int refine, cudaStream_t s);
cudaError_t launch_normal_tc(const SolvePlan& S, int rb_max, int npad_max, cudaStream_t s);

// Row-slab schedule of the fused selection + Gram (k_gram_slab.cu).  Table
// `task_pos` holds nslab prefix tables (nprob + 1 entries each): the trials of
// every problem that has slab s.
struct SlabPlan {
  const ProbDesc* descs;
  int nprob;
  int nslab;
  const int64_t* dT;
  const int64_t* hT;
  size_t task_pos;
};
bool slab_supported(int mode, int l, int y_dtype);
// variant 1: the slab kernel compiled for one CTA per SM fewer (more registers per thread)
cudaError_t launch_gram_slab(int mode, int l, int variant, const SlabPlan& S, cudaStream_t s);
int gram_slab_regs(int mode, int l, int variant);  // registers per thread of that kernel, -1 if none

cudaError_t launch_copy16(const void* src, void* dst, size_t bytes, cudaStream_t s);  // bytes: multiple of 16
cudaError_t launch_zero16(void* dst, size_t bytes, cudaStream_t s);
cudaError_t launch_fp64_math(const double* x, int64_t count, double* out, cudaStream_t s);
cudaError_t launch_readback(const ProbDesc* descs, int nprob, void* host, int stride, cudaStream_t s);
cudaError_t launch_pack_mask(const ProbDesc* descs, const int64_t* blk_off, int nprob, int64_t nblocks, cudaStream_t s);
cudaError_t launch_count_known(const uint8_t* W, int64_t ldw, int64_t m, int64_t n, unsigned long long* out,
                               cudaStream_t s);
cudaError_t launch_coverage(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t trials_total,
                            int64_t max_words, cudaStream_t s);
cudaError_t launch_sample(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total, cudaStream_t s);
// a1 and a2 in one launch (the sampler's blocks first)
cudaError_t launch_front(const ProbDesc* descs, const int64_t* blk_off, int64_t pack_blocks, const int64_t* trial_off,
                         int64_t trials, int nprob, cudaStream_t s);
cudaError_t launch_sample_range(const ProbDesc& d, int64_t t0, int64_t count, int32_t* cols, cudaStream_t s);
cudaError_t launch_select_rows(const uint32_t* bits, int64_t ldb, int64_t m, const int32_t* cols, int l, int64_t count,
                               const int64_t* row_off, int32_t* rows, int32_t* row_counts, cudaStream_t s);
cudaError_t launch_select_gram(int mode, const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total,
                               int lmax, cudaStream_t s);
cudaError_t launch_rows_variant(const ProbDesc* descs, const int64_t* pack_off, int64_t pack_total,
                                const int64_t* trial_off, int64_t trials_total, int nprob, int kmax, int rmax,
                                int64_t nmax, cudaStream_t s);
// list (total entries) and list_count (zeroed): the trials that the two-per-warp kernel hands
// to the one-per-warp kernel; NULL: one trial per warp throughout
cudaError_t launch_minor_scatter(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total, int lmax,
                                 unsigned long long* list, unsigned long long* list_count, cudaStream_t s);
cudaError_t launch_finalize_M(const ProbDesc* descs, const int64_t* ent_off, int nprob, int64_t total, cudaStream_t s);
cudaError_t launch_eig(const EigPlan& P, bool fp64_factor, double shift_rel, int iters, cudaStream_t s);
cudaError_t launch_trace_M(const ProbDesc* descs, int nprob, cudaStream_t s);
cudaError_t launch_solve_u(const SolvePlan& S, int mode, cudaStream_t s);
cudaError_t launch_residual(const SolvePlan& S, int mode, double* partial, cudaStream_t s, bool refine = true);
cudaError_t launch_l1_scatter(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total,
                              cudaStream_t s);
cudaError_t launch_irls_u(const ProbDesc* descs, const int64_t* row_off, int nprob, int64_t total, int rmax,
                          bool fp64, cudaStream_t s);

}  // namespace rsm
