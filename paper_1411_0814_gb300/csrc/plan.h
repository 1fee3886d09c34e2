// Host-side planning of a batch of problems: validation, derived sizes,
// workspace layout and the offset tables the batched kernels read.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rsm.h"
#include "common.cuh"
#include "kernels.h"

namespace rsm {

struct Derived {
  int l = 0, nm = 0, P_l = 0, nblk = 0, kx = 0, q = 0, q_pad = 0;
  int64_t ldb = 0, npad = 0, slab_rows = 0;
  bool solve_u = false;
  bool tc = false;  // normal equations on the tensor cores
  int tc_npad = 0;
};

// Validate a problem and fill its derived sizes.  Returns RSM_OK or
// RSM_ERR_INVALID_ARG / RSM_ERR_NOT_IMPLEMENTED with a message in *why.
int validate_problem(const rsm_problem& p, Derived& dv, std::string* why);

// Gram-stage choices of one problem (picked by rsm_autotune; the defaults
// otherwise): the schedule (0: L2-resident row slabs, 1: one warp per
// submatrix), the slab size in MiB of Y, and the slab kernel's occupancy
// variant (0: the CTAs per SM its registers allow, 1: one fewer).
struct Tune {
  int schedule = 0;
  int slab_mib = 32;
  int variant = 0;
};

// Byte layout of one batch inside a workspace buffer.
struct BatchLayout {
  size_t zero_bytes = 0;   // [0, zero_bytes) must be zeroed before the launch
  size_t total_bytes = 0;  // workspace bytes
  size_t plan_bytes = 0;   // descriptor + offset tables + TMA descriptors (uploaded to the start of the plan buffer)
  size_t tmap_off = 0;     // two 128-byte TMA descriptors per problem, from here
};

// Everything needed to launch one batch, built on the host.
struct Batch {
  int nprob = 0;
  int lmax = 0;
  int gram_mode = 0;
  int solve_mode = 0;
  bool any_solve = false;
  bool tc_tma = false;  // the tensor-core normal equations read Y and the mask by TMA (set at upload)
  std::vector<Derived> dv;
  std::vector<ProbDesc> descs;  // host copies (device pointers filled by bind())
  std::vector<int64_t> tables;  // all int64 offset tables, concatenated
  // positions (in int64 elements) of each table inside `tables`
  size_t o_pack = 0, o_trial = 0, o_ent = 0, o_pad2 = 0, o_step = 0, o_linv = 0, o_nk = 0,
         o_mx = 0, o_chunk = 0, o_part = 0, o_rot = 0, o_rowtile = 0, o_k = 0, o_tile = 0, o_row = 0, o_res = 0,
         o_b = 0, o_tc = 0, o_resv = 0, o_phase = 0;
  int64_t pack_blocks = 0, trials_total = 0, ent_total = 0, pad2_total = 0, nk_total = 0, part_total = 0,
          k_total = 0, tile_total = 0, row_total = 0, res_blocks = 0, b_total = 0, tc_total = 0, resv_blocks = 0;
  int resv_rmax = 0;  // largest r of the problems with the vectorised residual
  int64_t solve_rows = 0;  // rows of all problems that solve for U
  bool any_coverage = false;  // some problem counts its visited entries
  bool l1 = false;            // the L1 forms (all problems of the batch)
  int irls_iters = 0;
  size_t o_urow = 0;          // m per solving problem (IRLS of U)
  int64_t urow_total = 0;
  // method M2 problems: row-packing blocks, their trials, largest k, r and n
  size_t o_prow = 0, o_trial2 = 0;
  int64_t prow_total = 0, trials2_total = 0, nmax2 = 0;
  int kmax2 = 0, rmax2 = 0;
  int64_t max_words = 0;      // largest ceil(m / 32) of the batch
  int tc_rb = 0, tc_npad_max = 0;  // batch-wide V stride and largest N of the tensor-core normal equations
  int max_nblk = 0;
  // per-problem byte offsets inside the workspace
  std::vector<size_t> zero_off, data_off;
  std::vector<size_t> zero_size, data_size;
  size_t part_bytes_off = 0, res_bytes_off = 0, fail_list_off = 0, fail_count_off = 0;
  size_t minor_list_off = 0, minor_count_off = 8;  // trials handed from the two-per-warp minor kernel (count zeroed)
  size_t sync_off = 0, sync_bytes = 0;  // the factor launch's claim counter and phase counts (zeroed)
  int rmax = 0;
  // Row-slab schedule of the Gram: one group per distinct l that the slab
  // kernel supports (a launch per slab per group); problems of other l go
  // through the per-trial kernel (table o_trial_generic).
  struct SlabGroup {
    int l;
    int variant;
    size_t o_slab;  // nslab prefix tables over the problems of this l and variant
  };
  std::vector<SlabGroup> slab_groups;
  int nslab = 0;
  size_t o_trial_generic = 0;
  int64_t generic_total = 0;
  int generic_lmax = 0;
  BatchLayout layout;
};

// Build the batch (sizes, tables, layout).  Problems must be validated first.
// tunes: one per problem, or NULL for the defaults.
void build_batch(const rsm_problem* ps, int count, Batch& b, const Tune* tunes = nullptr);
// Fill the device pointers of b.descs for a workspace at `ws`.
void bind_batch(Batch& b, const rsm_problem* ps, unsigned char* ws);

// Device bytes of one problem's workspace (what rsm_footprint_bytes reports).
size_t problem_footprint(const rsm_problem& p, const Derived& dv);

}  // namespace rsm
