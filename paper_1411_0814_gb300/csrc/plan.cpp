// Host-side planning of a batch of problems (see plan.h).
#include "plan.h"

#ifndef RSM_EIG_EXTRA
#define RSM_EIG_EXTRA 4  // extra vectors of the eigen block iteration beyond r (the gap at r is wide)
#endif

#include <algorithm>

namespace rsm {

namespace {
constexpr int kEigSplit = 32;  // must equal kSplit in k_eig.cu
constexpr int kPrecSplit = 16;  // must equal kPSplit in k_eig.cu
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Sizes {
  size_t macc, counters, colcount, stats, tflag, visited;    // zero region
  size_t bits, cols, rowc, gram, M, Mdf, F1, F2, Dinv, X, MX, R, small, Kmat, NB, Lf, rbits, Bt, Zst;  // data region
};

Sizes sizes_of(const rsm_problem& p, const Derived& dv) {
  Sizes s{};
  const size_t n = (size_t)p.n, m = (size_t)p.m, I = (size_t)p.trials;
  s.macc = align_up(n * n * 8);
  s.counters = align_up(16 * 8);
  s.colcount = align_up(n * 4);
  s.stats = align_up(64 * 8);
  s.tflag = align_up((size_t)3 * dv.nblk * dv.nblk * 4);
  s.visited = p.coverage ? align_up(n * (size_t)dv.ldb * 4) : 0;
  s.bits = align_up(n * (size_t)dv.ldb * 4);
  s.cols = align_up(I * dv.l * 4);
  s.rowc = align_up(I * 4);
  s.gram = align_up(I * dv.P_l * 8);
  s.M = align_up(n * n * 8);
  s.Mdf = align_up(n * n * 8);
  s.F1 = align_up((size_t)dv.npad * dv.npad * 8 * 2);  // the factor, then T = A^-1
  s.F2 = align_up((size_t)dv.npad * dv.npad * 8);
  s.Dinv = align_up((size_t)dv.nblk * 32 * 32 * 8);
  s.X = align_up(n * dv.kx * 8);
  s.MX = s.X;
  s.R = align_up((size_t)kEigSplit * n * dv.kx * 8);
  s.small = align_up((2 * 32 * 32 + 32) * 8);
  // Kmat: the SIMT form's n x q_pad table, or the tensor-core form's B images
  // (n_pad x 2 npad FP32) plus V in FP32 (n_pad x 24 at most)
  const size_t n_pad = (n + 31) / 32 * 32;
  s.Kmat = dv.solve_u ? align_up(std::max(n * dv.q_pad * 8, n_pad * (2 * (size_t)normal_tc_npad(p.r) + 24) * 4)) : 0;
  s.NB = dv.solve_u ? align_up(m * dv.q_pad * 8) : 0;
  // method M2: the row-packed mask and B_t of every trial (the per-trial Gram is not stored)
  const bool rows = p.variant == RSM_ROWS_RANDOM;
  s.gram = rows ? 0 : s.gram;
  s.rbits = rows ? align_up(m * (size_t)((n + 31) / 32) * 4) : 0;
  s.Bt = rows ? align_up(I * (size_t)dv.l * p.r * 8) : 0;
  // the L1 forms keep every trial's minor vectors for the reweighting steps
  s.Zst = p.norm == 1 ? align_up(I * (size_t)dv.l * dv.nm * 8) : 0;
  // the FP32 normal equations keep each row's factor for the refinement step of the residual pass
  s.Lf = dv.solve_u && p.solve_prec == RSM_PREC_F32 ? align_up(m * (size_t)(p.r * (p.r + 1) / 2) * 4) : 0;
  return s;
}

size_t zero_sum(const Sizes& s) { return s.macc + s.counters + s.colcount + s.stats + s.tflag + s.visited; }
size_t data_sum(const Sizes& s) {
  return s.bits + s.cols + s.rowc + s.gram + s.M + s.Mdf + s.F1 + s.F2 + s.Dinv + s.X + s.MX + s.R + s.small + s.Kmat +
         s.NB + s.Lf + s.rbits + s.Bt + s.Zst;
}
size_t part_doubles(const rsm_problem& p, const Derived& dv) {
  return (size_t)((p.n + 63) / 64) * 2 * dv.kx * dv.kx;  // chunks of kChunk = 64 rows (k_eig.cu)
}
// The vectorised residual kernels (2 rows per lane, or the TMA-fed pass for r <=
// 8): FP32 form of FP32 Y whose columns start on 16-byte boundaries, r <= 16
// (the refinement keeps 2 rows x r sums per lane in registers).
bool resv_of(const rsm_problem& p, const Derived& dv) {
  return dv.solve_u && p.solve_prec == RSM_PREC_F32 && p.y_dtype == RSM_F32 && p.ldy % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(p.Y) & 15) == 0 && p.r <= 16 && p.m % 2 == 0;  // pairs of rows stay in Y
}
size_t res_blocks_of(const rsm_problem& p, const Derived& dv) {  // partial sums of the residual
  if (!dv.solve_u) return 0;
  return resv_of(p, dv) ? (size_t)((p.m + 63) / 64) : (size_t)((p.m + 31) / 32);
}
}  // namespace

int validate_problem(const rsm_problem& p, Derived& dv, std::string* why) {
  auto bad = [&](const char* msg) {
    if (why) *why = msg;
    return (int)RSM_ERR_INVALID_ARG;
  };
  if (!p.Y || !p.W || !p.V) return bad("Y, W and V must be device pointers");
  if (p.n < 2 || p.m < p.n) return bad("need 2 <= n <= m");
  if (p.m > 0x7fffffffLL) return bad("m must fit in int32");
  if (p.r < 1 || p.r >= p.n) return bad("need 1 <= r < n");
  dv.l = p.l ? p.l : p.r + 1;
  if (p.variant == RSM_ROWS_RANDOM) {
    // M2: l is the number of rows k; every vector beyond the r largest is kept
    if (dv.l <= p.r || dv.l > p.m || dv.l > kMaxL) return bad("rows variant: need r < k <= min(m, 32)");
    if (p.n_minor != 0) return bad("rows variant: n_minor must be 0 (all c_t - r vectors are used)");
    if (p.debug_Z) return bad("rows variant: debug_Z is not available");
    if (p.n > 8192) {
      if (why) *why = "rows variant: n > 8192 is not supported";
      return (int)RSM_ERR_NOT_IMPLEMENTED;
    }
    dv.nm = 1;
  } else {
    if (dv.l <= p.r || dv.l > p.n || dv.l > kMaxL) return bad("need r < l <= min(n, 32)");
    dv.nm = p.n_minor ? p.n_minor : dv.l - p.r;
    if (dv.nm < 1 || dv.nm > dv.l - p.r) return bad("need 1 <= n_minor <= l - r");
  }
  if (p.trials < 1 || p.trials > (int64_t)1 << 36) return bad("need 1 <= trials <= 2^36");
  if (p.coverage != 0 && p.coverage != 1) return bad("coverage must be 0 or 1");
  if (p.norm != 0 && p.norm != 1 && p.norm != 2) return bad("norm must be 1 (L1) or 2 (L2)");
  if (p.norm == 1 && p.variant == RSM_ROWS_RANDOM) return bad("the L1 forms need a column variant");
  if (p.norm == 1 && p.r > 8) return bad("the L1 forms support r <= 8");
  if (p.irls_iters < 0 || p.irls_iters > 1000 || p.irls_delta_v < 0.0 || p.irls_delta_u < 0.0)
    return bad("irls_iters in 0..1000, irls_delta_v and irls_delta_u >= 0");
  if (p.debug_visited && !p.coverage) return bad("debug_visited needs coverage = 1");
  if (p.ldy < p.m || p.ldw < p.m || p.ldv < p.n) return bad("leading dimensions too small");
  if (p.U && p.ldu < p.m) return bad("ldu < m");
  if (p.y_dtype != RSM_F64 && p.y_dtype != RSM_F32) return bad("y_dtype");
  if (p.variant != RSM_COLS_RANDOM && p.variant != RSM_COLS_ADJACENT && p.variant != RSM_ROWS_RANDOM)
    return bad("variant");
  if (p.gram_prec < RSM_PREC_F64 || p.gram_prec > RSM_PREC_F32) return bad("gram_prec");
  if (p.solve_prec != RSM_PREC_F64 && p.solve_prec != RSM_PREC_F32) {
    if (p.solve_prec == RSM_PREC_F32X2) {
      if (why) *why = "solve_prec F32X2 is not implemented";
      return (int)RSM_ERR_NOT_IMPLEMENTED;
    }
    return bad("solve_prec");
  }
  dv.P_l = dv.l * (dv.l + 1) / 2;
  dv.ldb = (((p.m + 31) / 32) + 3) / 4 * 4;
  // The kernels index Y, W, the packed mask and the n x n work matrices with
  // 32-bit offsets (64-bit integer arithmetic is slow on the device).
  if (p.n > 32768) {
    if (why) *why = "n > 32768 is not supported";
    return (int)RSM_ERR_NOT_IMPLEMENTED;
  }
  const uint64_t lim = (uint64_t)1 << 32;
  if ((uint64_t)p.ldy * (uint64_t)p.n >= lim || (uint64_t)p.ldw * (uint64_t)p.n >= lim ||
      (uint64_t)p.m * 64u >= lim) {
    if (why) *why = "ldy * n, ldw * n and 64 m must stay below 2^32";
    return (int)RSM_ERR_NOT_IMPLEMENTED;
  }
  dv.nblk = (int)((p.n + 31) / 32);
  dv.npad = (int64_t)dv.nblk * 32;
  dv.kx = (int)std::min<int64_t>(std::min<int64_t>(p.n, 32), p.r + RSM_EIG_EXTRA);
  dv.q = p.r * (p.r + 1) / 2 + p.r + 1;
  dv.q_pad = (dv.q + 63) / 64 * 64;
  dv.solve_u = p.U != nullptr;
  return RSM_OK;
}

size_t problem_footprint(const rsm_problem& p, const Derived& dv) {
  Sizes s = sizes_of(p, dv);
  return zero_sum(s) + data_sum(s) + align_up(part_doubles(p, dv) * 8) + align_up(res_blocks_of(p, dv) * 8) +
         align_up(dv.solve_u ? (size_t)p.m * 8 : 0) + kAlign;
}

// Rows per slab of the row-slab Gram: slab_mib MiB of the problem's Y (32 by
// default, so that a slab stays resident in L2 while every trial reads it), at
// least 1024 rows, a multiple of 32 (whole mask words).
int64_t slab_rows_of(const rsm_problem& p, int slab_mib) {
  const int64_t row_bytes = p.n * (p.y_dtype == RSM_F64 ? 8 : 4);
  return std::max<int64_t>(1024, ((int64_t)slab_mib << 20) / std::max<int64_t>(1, row_bytes) / 32 * 32);
}

void build_batch(const rsm_problem* ps, int count, Batch& b, const Tune* tunes) {
  const Tune dflt{};
  auto tune = [&](int i) -> const Tune& { return tunes ? tunes[i] : dflt; };
  b.nprob = count;
  b.dv.resize(count);
  b.descs.assign(count, ProbDesc{});
  b.lmax = 0;
  b.max_nblk = 0;
  b.rmax = 0;
  b.any_solve = false;
  for (int i = 0; i < count; ++i) {
    validate_problem(ps[i], b.dv[i], nullptr);
    b.lmax = std::max(b.lmax, b.dv[i].l);
    b.max_nblk = std::max(b.max_nblk, b.dv[i].nblk);
    b.any_solve |= b.dv[i].solve_u;
    b.rmax = std::max(b.rmax, ps[i].r);
  }
  b.l1 = ps[0].norm == 1;
  b.irls_iters = ps[0].irls_iters ? ps[0].irls_iters : 8;
  b.any_coverage = false;
  b.max_words = 0;
  for (int i = 0; i < count; ++i) {
    b.any_coverage |= ps[i].coverage != 0;
    b.max_words = std::max<int64_t>(b.max_words, (ps[i].m + 31) / 32);
  }
  // normal equations on the tensor cores: FP32 solve of FP32 Y, r small enough for one N tile
  b.tc_rb = 0;
  b.tc_npad_max = 0;
  for (int i = 0; i < count; ++i) {
    Derived& dv = b.dv[i];
    dv.tc = dv.solve_u && ps[i].solve_prec == RSM_PREC_F32 && ps[i].y_dtype == RSM_F32 && normal_tc_supported(ps[i].r);
    dv.tc_npad = dv.tc ? normal_tc_npad(ps[i].r) : 0;
    if (dv.tc) {
      b.tc_rb = std::max(b.tc_rb, normal_tc_rb(ps[i].r));
      b.tc_npad_max = std::max(b.tc_npad_max, dv.tc_npad);
    }
  }
  std::vector<int64_t>& T = b.tables;
  T.clear();
  auto prefix = [&](auto per) -> size_t {  // append an exclusive prefix table, return its position
    size_t pos = T.size();
    int64_t acc = 0;
    for (int i = 0; i < count; ++i) {
      T.push_back(acc);
      acc += per(i);
    }
    T.push_back(acc);
    return pos;
  };
  auto total = [&](size_t pos) { return T[pos + count]; };
  b.o_pack = prefix([&](int i) { return ps[i].n * ((b.dv[i].ldb + 255) / 256); });
  // method M2: row-packed mask (ceil(n/32) words x m rounded to 32, word-major) and its trials
  auto is_rows = [&](int i) { return ps[i].variant == RSM_ROWS_RANDOM; };
  b.o_prow = prefix([&](int i) { return is_rows(i) ? (ps[i].n + 31) / 32 * ((ps[i].m + 31) / 32 * 32) : (int64_t)0; });
  b.prow_total = total(b.o_prow);
  b.o_trial2 = prefix([&](int i) { return is_rows(i) ? ps[i].trials : (int64_t)0; });
  b.trials2_total = total(b.o_trial2);
  b.kmax2 = b.rmax2 = 0;
  b.nmax2 = 0;
  for (int i = 0; i < count; ++i)
    if (is_rows(i)) {
      b.kmax2 = std::max(b.kmax2, b.dv[i].l);
      b.rmax2 = std::max(b.rmax2, ps[i].r);
      b.nmax2 = std::max<int64_t>(b.nmax2, ps[i].n);
    }
  b.pack_blocks = total(b.o_pack);
  b.o_trial = prefix([&](int i) { return ps[i].trials; });
  b.trials_total = total(b.o_trial);
  b.o_ent = prefix([&](int i) { return ps[i].n * ps[i].n; });
  b.ent_total = total(b.o_ent);
  b.o_pad2 = prefix([&](int i) { return b.dv[i].npad * b.dv[i].npad; });
  b.pad2_total = total(b.o_pad2);
  b.o_step = T.size();
  for (int k = 0; k < b.max_nblk; ++k) {  // per step: panel tiles i >= k + 3, trailing tiles of columns >= k + 2
    prefix([&](int i) { return (int64_t)std::max(0, b.dv[i].nblk - k - 3); });
    prefix([&](int i) {
      const int64_t t = std::max(0, b.dv[i].nblk - k - 2);
      return t * (t + 1) / 2;
    });
  }
  b.o_linv = T.size();
  for (int k = 0; k < b.max_nblk; ++k) {  // per step: row k of L^-1, updates of the rows >= k + 2, row k's share of T
    prefix([&](int i) { return (int64_t)(k < b.dv[i].nblk ? k + 1 : 0); });
    prefix([&](int i) { return (int64_t)std::max(0, b.dv[i].nblk - k - 2) * (k + 1); });
    prefix([&](int i) { return (int64_t)(k < b.dv[i].nblk ? (int64_t)(k + 1) * (k + 2) / 2 : 0); });
  }
  // Task prefix over the segments of the factor launch's claim order (after
  // its chain tasks): per step k the panel and the trailing update, then the
  // inverse-factor tasks and the rows of T of step k - kFactorLag; then those
  // of the last kFactorLag steps.
  {
    const size_t n1 = (size_t)count + 1;
    const int K = b.max_nblk, lag = kFactorLag;
    auto tot = [&](size_t pos) { return T[pos + count]; };
    std::vector<int64_t> ph(1, 0);
    auto linv_seg = [&](int kk) {
      for (int c = 0; c < 3; ++c)
        ph.push_back(ph.back() + (kk >= 0 && kk < K ? tot(b.o_linv + (size_t)kk * 3 * n1 + (size_t)c * n1) : 0));
    };
    for (int k = 0; k < K; ++k) {
      for (int c = 0; c < 2; ++c) ph.push_back(ph.back() + tot(b.o_step + (size_t)k * 2 * n1 + (size_t)c * n1));
      linv_seg(k - lag);
    }
    for (int m = 0; m < lag; ++m) linv_seg(K - lag + m);
    b.o_phase = T.size();
    T.insert(T.end(), ph.begin(), ph.end());
  }
  b.o_nk = prefix([&](int i) { return ps[i].n * b.dv[i].kx; });
  b.nk_total = total(b.o_nk);
  b.o_mx = prefix([&](int i) { return (int64_t)kEigSplit * ((ps[i].n + 127) / 128); });
  b.o_chunk = prefix([&](int i) { return (ps[i].n + 63) / 64; });
  b.o_part = prefix([&](int i) { return (int64_t)part_doubles(ps[i], b.dv[i]); });
  b.part_total = total(b.o_part);
  b.o_rot = prefix([&](int i) { return (ps[i].n + 7) / 8; });
  b.o_rowtile = prefix([&](int i) { return (int64_t)kPrecSplit * ((ps[i].n + 15) / 16); });
  b.o_k = prefix([&](int i) { return b.dv[i].solve_u && !b.dv[i].tc ? ps[i].n * b.dv[i].q_pad : 0; });
  b.k_total = total(b.o_k);
  b.o_tile = prefix([&](int i) {
    return b.dv[i].solve_u && !b.dv[i].tc ? ((ps[i].m + 63) / 64) * (b.dv[i].q_pad / 64) : 0;
  });
  b.tile_total = total(b.o_tile);
  b.o_b = prefix([&](int i) {
    return b.dv[i].tc ? (ps[i].n + 31) / 32 * 32 * (int64_t)(b.dv[i].tc_npad + b.tc_rb) : 0;
  });
  b.b_total = total(b.o_b);
  b.o_tc = prefix([&](int i) { return b.dv[i].tc ? (ps[i].m + 127) / 128 : 0; });
  b.tc_total = total(b.o_tc);
  // rows for k_row_solve: the tensor-core form with r <= 8 (batch-wide accumulator width 8)
  // solves its rows in its own epilogue
  b.o_row = prefix([&](int i) { return b.dv[i].solve_u && !(b.dv[i].tc && b.tc_rb == 8) ? ps[i].m : 0; });
  b.row_total = total(b.o_row);
  b.solve_rows = 0;
  for (int i = 0; i < count; ++i)
    if (b.dv[i].solve_u) b.solve_rows += ps[i].m;
  b.o_urow = prefix([&](int i) { return b.dv[i].solve_u ? (ps[i].m + 127) / 128 * 128 : (int64_t)0; });
  b.urow_total = total(b.o_urow);
  b.o_res = prefix([&](int i) { return resv_of(ps[i], b.dv[i]) ? (int64_t)0 : (int64_t)res_blocks_of(ps[i], b.dv[i]); });
  b.res_blocks = total(b.o_res);
  b.o_resv = prefix([&](int i) { return resv_of(ps[i], b.dv[i]) ? (int64_t)res_blocks_of(ps[i], b.dv[i]) : (int64_t)0; });
  b.resv_blocks = total(b.o_resv);
  b.resv_rmax = 0;
  for (int i = 0; i < count; ++i)
    if (resv_of(ps[i], b.dv[i])) b.resv_rmax = std::max(b.resv_rmax, ps[i].r);

  // Row slabs: the slab size of a problem depends on its own n and Y type only,
  // and problems are grouped by l, so a problem's Gram is summed in the same
  // order alone and in any batch (results do not depend on the batch).
  const int mode = ps[0].gram_prec == RSM_PREC_F64 ? 0 : ps[0].gram_prec == RSM_PREC_F32X2 ? 1 : 2;
  b.nslab = 0;
  for (int i = 0; i < count; ++i) {
    b.dv[i].slab_rows = slab_rows_of(ps[i], tune(i).slab_mib);
    b.nslab = std::max<int>(b.nslab, (int)((ps[i].m + b.dv[i].slab_rows - 1) / b.dv[i].slab_rows));
  }
  // problems on the slab schedule, grouped by (l, occupancy variant); the others (the
  // per-submatrix schedule, or a mode the slab kernel does not read) take the generic kernel
  auto on_slab = [&](int i) {
    return !is_rows(i) && tune(i).schedule == 0 && slab_supported(mode, b.dv[i].l, ps[i].y_dtype);
  };
  std::vector<std::pair<int, int>> groups;
  for (int i = 0; i < count; ++i)
    if (on_slab(i)) groups.emplace_back(b.dv[i].l, tune(i).variant ? 1 : 0);
  std::sort(groups.begin(), groups.end());
  groups.erase(std::unique(groups.begin(), groups.end()), groups.end());
  b.slab_groups.clear();
  for (const auto& lv : groups) {
    Batch::SlabGroup g{lv.first, lv.second, T.size()};
    for (int sl = 0; sl < b.nslab; ++sl)
      prefix([&](int i) {
        return on_slab(i) && b.dv[i].l == lv.first && (tune(i).variant ? 1 : 0) == lv.second &&
                       (int64_t)sl * b.dv[i].slab_rows < ps[i].m
                   ? ps[i].trials
                   : (int64_t)0;
      });
    b.slab_groups.push_back(g);
  }
  b.o_trial_generic = prefix([&](int i) { return is_rows(i) || on_slab(i) ? (int64_t)0 : ps[i].trials; });
  b.generic_total = total(b.o_trial_generic);
  b.generic_lmax = 0;
  for (int i = 0; i < count; ++i)
    if (!is_rows(i) && !on_slab(i)) b.generic_lmax = std::max(b.generic_lmax, b.dv[i].l);

  // workspace: all zero regions first, then all data regions, then shared partial buffers
  b.zero_off.resize(count);
  b.data_off.resize(count);
  b.zero_size.resize(count);
  b.data_size.resize(count);
  size_t off = kAlign;  // batch header: the fail-list counter
  b.fail_count_off = 0;
  b.sync_off = off;  // factor launch: claim counter, abort word
  b.sync_bytes = align_up(4 * 4);
  off += b.sync_bytes;
  for (int i = 0; i < count; ++i) {
    Sizes s = sizes_of(ps[i], b.dv[i]);
    b.zero_off[i] = off;
    b.zero_size[i] = zero_sum(s);
    off += b.zero_size[i];
  }
  b.layout.zero_bytes = off;
  for (int i = 0; i < count; ++i) {
    Sizes s = sizes_of(ps[i], b.dv[i]);
    b.data_off[i] = off;
    b.data_size[i] = data_sum(s);
    off += b.data_size[i];
  }
  b.part_bytes_off = off;
  off += align_up((size_t)b.part_total * 8);
  b.res_bytes_off = off;
  off += align_up((size_t)(b.res_blocks + b.resv_blocks) * 8);
  b.fail_list_off = off;
  off += align_up((size_t)b.solve_rows * 8);  // any solved row may take the minimum-norm path
  b.minor_list_off = off;  // any trial may be handed to the one-per-warp minor kernel
  off += align_up((size_t)b.trials_total * 8);
  b.layout.total_bytes = off;
  b.layout.tmap_off = align_up(sizeof(ProbDesc) * count) + align_up(T.size() * 8);
  b.layout.plan_bytes = b.layout.tmap_off + (size_t)256 * count;
  b.gram_mode = ps[0].gram_prec == RSM_PREC_F64 ? 0 : ps[0].gram_prec == RSM_PREC_F32X2 ? 1 : 2;
  b.solve_mode = ps[0].solve_prec == RSM_PREC_F64 ? 0 : 2;
}

void bind_batch(Batch& b, const rsm_problem* ps, unsigned char* ws) {
  for (int i = 0; i < b.nprob; ++i) {
    const rsm_problem& p = ps[i];
    const Derived& dv = b.dv[i];
    Sizes s = sizes_of(p, dv);
    ProbDesc& d = b.descs[i];
    d = ProbDesc{};
    d.m = p.m;
    d.n = p.n;
    d.trials = p.trials;
    d.r = p.r;
    d.l = dv.l;
    d.n_minor = dv.nm;
    d.variant = p.variant;
    d.seed = p.seed;
    d.pid = p.problem_id;
    d.y_dtype = p.y_dtype;
    d.Y = p.Y;
    d.ldy = p.ldy;
    d.W = p.W;
    d.ldw = p.ldw;
    d.ldb = dv.ldb;
    d.U = p.U;
    d.ldu = p.ldu;
    d.V = p.V;
    d.ldv = p.ldv;
    d.debug_Z = p.debug_Z;
    d.debug_M = p.debug_M;
    d.debug_cols = p.debug_cols;
    d.debug_row_counts = p.debug_row_counts;
    d.kx = dv.kx;
    d.slab_rows = dv.slab_rows;
    d.nblk = dv.nblk;
    d.q = dv.q;
    d.q_pad = dv.q_pad;
    unsigned char* z = ws + b.zero_off[i];
    d.macc = reinterpret_cast<unsigned long long*>(z);
    z += s.macc;
    d.counters = reinterpret_cast<unsigned long long*>(z);
    z += s.counters;
    d.colcount = reinterpret_cast<int32_t*>(z);
    z += s.colcount;
    d.stats = reinterpret_cast<double*>(z);
    z += s.stats;
    d.tflag = reinterpret_cast<unsigned*>(z);
    z += s.tflag;
    d.visited = s.visited ? reinterpret_cast<uint32_t*>(z) : nullptr;
    unsigned char* q = ws + b.data_off[i];
    auto take = [&](size_t bytes) {
      unsigned char* r = q;
      q += bytes;
      return r;
    };
    d.bits = reinterpret_cast<uint32_t*>(take(s.bits));
    d.cols = reinterpret_cast<int32_t*>(take(s.cols));
    d.row_counts = reinterpret_cast<int32_t*>(take(s.rowc));
    d.gram = reinterpret_cast<double*>(take(s.gram));
    d.M = reinterpret_cast<double*>(take(s.M));
    d.Mdf = reinterpret_cast<float2*>(take(s.Mdf));
    d.F1 = take(s.F1);
    d.F2 = take(s.F2);
    d.Dinv = take(s.Dinv);
    d.X = reinterpret_cast<double*>(take(s.X));
    d.MX = reinterpret_cast<double*>(take(s.MX));
    d.R = reinterpret_cast<double*>(take(s.R));
    d.small = reinterpret_cast<double*>(take(s.small));
    d.Kmat = s.Kmat ? reinterpret_cast<double*>(take(s.Kmat)) : nullptr;
    d.NB = s.NB ? reinterpret_cast<double*>(take(s.NB)) : nullptr;
    d.Lf = s.Lf ? reinterpret_cast<float*>(take(s.Lf)) : nullptr;
    d.rbits = s.rbits ? reinterpret_cast<uint32_t*>(take(s.rbits)) : nullptr;
    d.ldr = (p.n + 31) / 32;
    d.Bt = s.Bt ? reinterpret_cast<double*>(take(s.Bt)) : nullptr;
    d.Zst = s.Zst ? reinterpret_cast<double*>(take(s.Zst)) : nullptr;
    d.l1 = p.norm == 1 ? 1 : 0;
    d.irls_iters = p.irls_iters ? p.irls_iters : 8;
    d.delta_v = p.irls_delta_v > 0.0 ? p.irls_delta_v : 1e-4;
    d.delta_u = p.irls_delta_u > 0.0 ? p.irls_delta_u : 1e-3;
    d.tc = dv.tc ? 1 : 0;
    d.resv = resv_of(p, dv) ? 1 : 0;
    d.gram_fp32 = p.gram_prec == RSM_PREC_F32 ? 1 : 0;
    d.tc_npad = dv.tc_npad;
    d.tc_rb = b.tc_rb;
    if (d.Kmat) {
      const float* kf = reinterpret_cast<const float*>(d.Kmat);
      if (dv.tc) {  // V follows the B images
        d.vf32 = kf + (size_t)((p.n + 31) / 32 * 32) * 2 * dv.tc_npad;
        d.vf_ld = b.tc_rb;
      } else {  // the FP32 Kmat holds V in columns P .. P + r - 1
        d.vf32 = kf + p.r * (p.r + 1) / 2;
        d.vf_ld = dv.q_pad;
      }
    }
  }
}

}  // namespace rsm
