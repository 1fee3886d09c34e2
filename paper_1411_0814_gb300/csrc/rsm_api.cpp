// C ABI of librsm.so (include/rsm.h): handles, the synchronous and batched
// decompositions, the serving loop and the stage entry points.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rsm.h"
#include "common.cuh"
#include "kernels.h"
#include "plan.h"

using namespace rsm;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace rsm {
thread_local int64_t g_kernel_launches = 0;
void set_last_error(const std::string& msg) { g_last_error = msg; }
}

namespace {

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return RSM_ERR_CUDA;
}

#define RSM_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Makes `device` current for the scope of an entry point and restores the
// caller's current device on exit.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int device) {
    if ((err = cudaGetDevice(&prev)) == cudaSuccess && prev != device) err = cudaSetDevice(device);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr double kShiftRel32 = 3e-4;   // tau / (trace(M) / n) with the FP32 factor
constexpr double kShiftRel64 = 1e-11;  // tau / (trace(M) / n) with the FP64 factor
#ifndef RSM_EIG_ITERS32
#define RSM_EIG_ITERS32 3
#endif
#ifndef RSM_EIG_ITERS64
#define RSM_EIG_ITERS64 6
#endif
// most preconditioned steps with the FP32 factor (stops when converged; the
// paper-scale problem and the batched problems stop after two with the
// predicted-step rule, and every step left costs its launches even when they
// return at once: ~8 us alone, ~0.3 ms in a batch of 64 problems); a problem
// not converged by then takes the FP64 factor
constexpr int kEigIters32 = RSM_EIG_ITERS32;
constexpr int kEigIters64 = RSM_EIG_ITERS64;  // most steps with the FP64 factor (near-exact shift-invert)
constexpr int64_t kSmallN = 256;       // at or below this n the FP64 factor is cheap: use it directly
constexpr double kEigErrTol = 1e-11;   // a-posteriori bound that accepts the FP32-factor result
constexpr double kRankTol = 1e-12;  // lambda_{r+1} <= kRankTol * trace(M): underdetermined

// A device buffer that only grows.
struct DevBuf {
  void* ptr = nullptr;
  size_t size = 0;
  int reserve(size_t bytes) {
    if (bytes <= size) return RSM_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    size = 0;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RSM_ERR_NO_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    size = bytes;
    return RSM_OK;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    size = 0;
  }
};

struct PinBuf {
  void* ptr = nullptr;
  size_t size = 0;
  int reserve(size_t bytes) {
    if (bytes <= size) return RSM_OK;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    size = 0;
    cudaError_t e = cudaMallocHost(&ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
    size = bytes;
    return RSM_OK;
  }
  void release() {
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    size = 0;
  }
};

// Everything one in-flight decomposition (or batch) uses: a stream, a
// workspace, a plan buffer, pinned readback space and stage events.
struct Slot {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevBuf ws, plan;
  PinBuf host;
  cudaEvent_t ev[10] = {};
  cudaEvent_t ev_order = nullptr;  // recorded on the legacy default stream before a call on an owned stream
  bool fault_wait = false;  // RSM_FAULT_DEVICE_WAIT for the batches this slot runs
  int init(cudaStream_t external) {
    if (external) {
      stream = external;
    } else {
      RSM_CUDA(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
      own_stream = true;
    }
    for (auto& e : ev) RSM_CUDA(cudaEventCreate(&e));
    RSM_CUDA(cudaEventCreateWithFlags(&ev_order, cudaEventDisableTiming));
    return RSM_OK;
  }
  void destroy() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (ev_order) cudaEventDestroy(ev_order);
    ev_order = nullptr;
    ws.release();
    plan.release();
    host.release();
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

struct Request {
  uint64_t ticket = 0;
  rsm_problem prob{};
  size_t footprint = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  cudaEvent_t ready = nullptr;  // recorded on the submitter's stream: the inputs are complete after it
  rsm_result res{};
  std::chrono::steady_clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct rsm_handle {
  rsm_config cfg{};
  int device = 0;
  Slot main;  // rsm_decompose / rsm_decompose_batch
  std::mutex api_mu;  // serialises the synchronous entry points
  // serving
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::vector<Slot> slots;
  std::vector<std::thread> workers;
  size_t budget = 0, in_use = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  uint32_t fault = 0;
  // Gram-stage choices found by rsm_autotune, by problem shape (tune_key)
  std::mutex tune_mu;
  std::map<std::vector<int64_t>, std::pair<Tune, rsm_tune>> tuned;
};

namespace {

// Problems that share this key share the Gram stage's best choices: the Gram
// precision, the type of Y, the submatrix width l, n, and m to the next power of two.
std::vector<int64_t> tune_key(const rsm_problem& p) {
  const int64_t l = p.l ? p.l : p.r + 1;
  int64_t mb = 0;
  while (((int64_t)1 << mb) < p.m) ++mb;
  return {p.gram_prec, p.y_dtype, l, p.n, mb};
}

}  // namespace

namespace {

// Zero what the factor launch needs zeroed before it runs again: the claim
// counter and abort word, every problem's tile states and factor-failure flag.
int reset_eig_state(Batch& b, Slot& slot) {
  RSM_CUDA(cudaMemsetAsync(static_cast<unsigned char*>(slot.ws.ptr) + b.sync_off, 0, b.sync_bytes, slot.stream));
  for (int i = 0; i < b.nprob; ++i) {
    RSM_CUDA(cudaMemsetAsync(b.descs[i].counters + 3, 0, 8, slot.stream));
    RSM_CUDA(cudaMemsetAsync(b.descs[i].tflag, 0, (size_t)3 * b.dv[i].nblk * b.dv[i].nblk * 4, slot.stream));
  }
  return RSM_OK;
}

// Launch every stage of one batch on slot.stream.  The workspace and plan
// buffers of the slot must already hold the batch.  Does not synchronise.
int launch_batch(Batch& b, Slot& slot, bool fp64_factor, double shift_rel, bool do_front) {
  cudaStream_t s = slot.stream;
  unsigned char* plan = static_cast<unsigned char*>(slot.plan.ptr);
  const ProbDesc* D = reinterpret_cast<const ProbDesc*>(plan);
  const int64_t* T = reinterpret_cast<const int64_t*>(plan + ((sizeof(ProbDesc) * b.nprob + 255) / 256 * 256));
  const int np = b.nprob;
  cudaError_t e;
  if (do_front) {
    // mask packing and column sampling in one launch: the pack_mask stage time
    // covers both and the sample_cols stage is empty
    if ((e = launch_front(D, T + b.o_pack, b.pack_blocks, T + b.o_trial, b.trials_total, np, s)) != cudaSuccess)
      return cuda_fail(e, "pack_mask + sample");
    RSM_CUDA(cudaEventRecord(slot.ev[2], s));
    RSM_CUDA(cudaEventRecord(slot.ev[3], s));
    for (const auto& g : b.slab_groups) {
      SlabPlan sp{D, np, b.nslab, T, b.tables.data(), g.o_slab};
      if ((e = launch_gram_slab(b.gram_mode, g.l, g.variant, sp, s)) != cudaSuccess) return cuda_fail(e, "gram_slab");
    }
    if (b.generic_total > 0 &&
        (e = launch_select_gram(b.gram_mode, D, T + b.o_trial_generic, np, b.generic_total, b.generic_lmax, s)) !=
            cudaSuccess)
      return cuda_fail(e, "select_gram");
    RSM_CUDA(cudaEventRecord(slot.ev[4], s));
    if (b.any_coverage &&
        (e = launch_coverage(D, T + b.o_trial, np, b.trials_total, b.max_words, s)) != cudaSuccess)
      return cuda_fail(e, "coverage");
    if (b.trials2_total > 0 &&
        (e = launch_rows_variant(D, T + b.o_prow, b.prow_total, T + b.o_trial2, b.trials2_total, np, b.kmax2,
                                 b.rmax2, b.nmax2, s)) != cudaSuccess)
      return cuda_fail(e, "rows variant");
    unsigned char* wsb = static_cast<unsigned char*>(slot.ws.ptr);
    if ((e = launch_minor_scatter(D, T + b.o_trial, np, b.trials_total, b.lmax,
                                  reinterpret_cast<unsigned long long*>(wsb + b.minor_list_off),
                                  reinterpret_cast<unsigned long long*>(wsb + b.minor_count_off), s)) != cudaSuccess)
      return cuda_fail(e, "minor_scatter");
    if ((e = launch_finalize_M(D, T + b.o_ent, np, b.ent_total, s)) != cudaSuccess) return cuda_fail(e, "finalize_M");
    if (b.l1 && (e = launch_trace_M(D, np, s)) != cudaSuccess) return cuda_fail(e, "trace_M");
    RSM_CUDA(cudaEventRecord(slot.ev[5], s));
  }
  EigPlan ep{};
  ep.descs = D;
  ep.nprob = np;
  ep.max_nblk = b.max_nblk;
  ep.kx_max = 0;
  for (int i = 0; i < b.nprob; ++i) ep.kx_max = std::max(ep.kx_max, b.dv[i].kx);
  ep.dT = T;
  ep.hT = b.tables.data();
  ep.pad2 = b.o_pad2;
  ep.step = b.o_step;
  ep.linv = b.o_linv;
  ep.nk = b.o_nk;
  ep.mx = b.o_mx;
  ep.chunk = b.o_chunk;
  ep.part_off = b.o_part;
  ep.rot = b.o_rot;
  ep.row_tile = b.o_rowtile;
  ep.part = reinterpret_cast<double*>(static_cast<unsigned char*>(slot.ws.ptr) + b.part_bytes_off);
  ep.phase = b.o_phase;
  ep.sync = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(slot.ws.ptr) + b.sync_off);
  ep.fault_wait = slot.fault_wait;
  if ((e = launch_eig(ep, fp64_factor, shift_rel, fp64_factor ? kEigIters64 : kEigIters32, s)) != cudaSuccess)
    return cuda_fail(e, "eig");
  if (b.l1) {
    // the L1 form of V-hat: reweight the stored minor vectors by the current V,
    // rebuild M_w and solve it again, irls_iters times (k_robust.cu)
    for (int it = 0; it < b.irls_iters; ++it) {
      for (int i = 0; i < np; ++i)
        RSM_CUDA(cudaMemsetAsync(b.descs[i].macc, 0, (size_t)b.descs[i].n * b.descs[i].n * 8, s));
      if ((e = launch_l1_scatter(D, T + b.o_trial, np, b.trials_total, s)) != cudaSuccess)
        return cuda_fail(e, "l1_scatter");
      if ((e = launch_finalize_M(D, T + b.o_ent, np, b.ent_total, s)) != cudaSuccess)
        return cuda_fail(e, "finalize_M");
      if ((e = launch_trace_M(D, np, s)) != cudaSuccess) return cuda_fail(e, "trace_M");
      int st = reset_eig_state(b, slot);
      if (st != RSM_OK) return st;
      if ((e = launch_eig(ep, fp64_factor, shift_rel, fp64_factor ? kEigIters64 : kEigIters32, s)) != cudaSuccess)
        return cuda_fail(e, "eig");
    }
  }
  RSM_CUDA(cudaEventRecord(slot.ev[6], s));
  if (b.any_solve) {
    SolvePlan sp{};
    sp.descs = D;
    sp.nprob = np;
    sp.k_total = b.k_total;
    sp.k_off = T + b.o_k;
    sp.tile_off_host_total = b.tile_total;
    sp.tile_off = T + b.o_tile;
    sp.row_total = b.row_total;
    sp.row_off = T + b.o_row;
    sp.res_blocks = b.res_blocks;
    sp.res_off = T + b.o_res;
    sp.rmax = b.rmax;
    sp.b_total = b.b_total;
    sp.b_off = T + b.o_b;
    sp.tc_tiles = b.tc_total;
    sp.tc_off = T + b.o_tc;
    sp.tc_rb = b.tc_rb;
    sp.tc_npad_max = b.tc_npad_max;
    sp.tc_tma = b.tc_tma;
    sp.resv_blocks = b.resv_blocks;
    sp.resv_rmax = b.resv_rmax;
    sp.resv_off = T + b.o_resv;
    sp.any_solve = b.any_solve;
    sp.fail_list = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(slot.ws.ptr) + b.fail_list_off);
    sp.fail_count = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(slot.ws.ptr) + b.fail_count_off);
    if ((e = launch_solve_u(sp, b.solve_mode, s)) != cudaSuccess) return cuda_fail(e, "solve_u");
    RSM_CUDA(cudaEventRecord(slot.ev[7], s));
    double* partial = reinterpret_cast<double*>(static_cast<unsigned char*>(slot.ws.ptr) + b.res_bytes_off);
    if ((e = launch_residual(sp, b.solve_mode, partial, s)) != cudaSuccess) return cuda_fail(e, "residual");
    if (b.l1) {
      // the L1 rows: reweighting steps from the L2 rows (their e sets the scale of
      // delta), then e of the final U and V without the L2 refinement step
      for (int it = 0; it < b.irls_iters; ++it)
        if ((e = launch_irls_u(D, T + b.o_urow, np, b.urow_total, b.rmax, b.solve_mode == 0, s)) != cudaSuccess)
          return cuda_fail(e, "irls_u");
      if ((e = launch_residual(sp, b.solve_mode, partial, s, false)) != cudaSuccess) return cuda_fail(e, "residual");
    }
  } else {
    RSM_CUDA(cudaEventRecord(slot.ev[7], s));
  }
  RSM_CUDA(cudaEventRecord(slot.ev[8], s));
  return RSM_OK;
}

// Host readback area per problem: counters (16 x u64) + stats (64 doubles).
constexpr size_t kCountersBytes = 16 * 8;
constexpr size_t kReadback = kCountersBytes + 64 * 8;

int enqueue_readback(Batch& b, Slot& slot) {
  const ProbDesc* D = reinterpret_cast<const ProbDesc*>(slot.plan.ptr);
  // gather into a device staging area behind the plan, then one small copy to the host
  unsigned char* staging = static_cast<unsigned char*>(slot.plan.ptr) + b.layout.plan_bytes;
  RSM_CUDA(launch_readback(D, b.nprob, staging, kReadback, slot.stream));
  RSM_CUDA(cudaMemcpyAsync(slot.host.ptr, staging, (size_t)b.nprob * kReadback, cudaMemcpyDeviceToHost, slot.stream));
  return RSM_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library); NULL when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// TMA descriptors of a tensor-core problem (out: 256 bytes, 64-byte aligned):
// its FP32 Y (m x n column-major, boxes of 128 rows x 32 columns) and its packed
// mask (ldb words x n, boxes of 4 words x 32 columns).  False when the layout
// does not allow it (Y or ldy not 16-byte aligned) or the encoder refuses.
bool encode_tc_maps(const ProbDesc& d, void* out) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || d.y_dtype != RSM_F32) return false;
  if ((reinterpret_cast<uintptr_t>(d.Y) & 15) || ((d.ldy * 4) & 15) || (reinterpret_cast<uintptr_t>(d.bits) & 15))
    return false;
  CUtensorMap* maps = static_cast<CUtensorMap*>(out);
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t ydim[2] = {(cuuint64_t)d.m, (cuuint64_t)d.n};
  const cuuint64_t ystride[1] = {(cuuint64_t)d.ldy * 4};
  const cuuint32_t ybox[2] = {128, 32};
  if (enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(d.Y), ydim, ystride, ybox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t wdim[2] = {(cuuint64_t)d.ldb, (cuuint64_t)d.n};
  const cuuint64_t wstride[1] = {(cuuint64_t)d.ldb * 4};
  const cuuint32_t wbox[2] = {4, 32};
  return enc(&maps[1], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, d.bits, wdim, wstride, wbox, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Prepare slot buffers, upload the plan, zero the accumulators, launch, read
// back and fill results.  Synchronises slot.stream.
// given_M (count == 1 only): the caller's n x n M (device); the stages before
// the eigensolve are skipped and M is copied into the workspace instead.
int run_batch(rsm_handle* h, Slot& slot, const rsm_problem* ps, int count, rsm_result* res,
              const double* given_M = nullptr, const Tune* force = nullptr) {
  slot.fault_wait = (h->fault & RSM_FAULT_DEVICE_WAIT) != 0;
  std::vector<Tune> tunes(count);
  if (force) {
    tunes.assign(count, *force);
  } else {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    for (int i = 0; i < count && !h->tuned.empty(); ++i) {
      auto it = h->tuned.find(tune_key(ps[i]));
      if (it != h->tuned.end()) tunes[i] = it->second.first;
    }
  }
  Batch b;
  build_batch(ps, count, b, tunes.data());
  int st = slot.ws.reserve(b.layout.total_bytes);
  if (st != RSM_OK) return st;
  if ((st = slot.plan.reserve(b.layout.plan_bytes + (size_t)count * kReadback)) != RSM_OK) return st;
  if ((st = slot.host.reserve(std::max(b.layout.plan_bytes, (size_t)count * kReadback))) != RSM_OK) return st;
  bind_batch(b, ps, static_cast<unsigned char*>(slot.ws.ptr));
  if (given_M) b.descs[0].m_given = 1;
  // plan upload through the pinned buffer
  unsigned char* hp = static_cast<unsigned char*>(slot.host.ptr);
  const size_t dsz = (sizeof(ProbDesc) * count + 255) / 256 * 256;
  // TMA descriptors of the tensor-core normal equations: all problems have them, or the batch
  // takes the kernel without TMA
  b.tc_tma = b.tc_total > 0;
  for (int i = 0; i < count; ++i) {
    ProbDesc& d = b.descs[i];
    d.tmap = nullptr;
    if (!d.tc) continue;
    if (encode_tc_maps(d, hp + b.layout.tmap_off + (size_t)256 * i))
      d.tmap = static_cast<unsigned char*>(slot.plan.ptr) + b.layout.tmap_off + (size_t)256 * i;
    else
      b.tc_tma = false;
  }
  std::memcpy(hp, b.descs.data(), sizeof(ProbDesc) * count);
  std::memcpy(hp + dsz, b.tables.data(), b.tables.size() * 8);
  const int64_t launches0 = g_kernel_launches;
  RSM_CUDA(cudaEventRecord(slot.ev[0], slot.stream));
  // plan upload and zeroing by kernels, not by the copy engines (see k_util.cu)
  RSM_CUDA(launch_copy16(hp, slot.plan.ptr, b.layout.plan_bytes, slot.stream));
  RSM_CUDA(launch_zero16(slot.ws.ptr, (b.layout.zero_bytes + 15) / 16 * 16, slot.stream));
  RSM_CUDA(cudaEventRecord(slot.ev[1], slot.stream));
  int64_t max_n = 0;
  for (int i = 0; i < count; ++i) max_n = std::max<int64_t>(max_n, ps[i].n);
  bool fp64 = max_n <= kSmallN;
  double shift = fp64 ? kShiftRel64 : kShiftRel32;
  if (given_M) {
    const ProbDesc* D = reinterpret_cast<const ProbDesc*>(slot.plan.ptr);
    RSM_CUDA(cudaMemcpyAsync(b.descs[0].M, given_M, (size_t)ps[0].n * ps[0].n * 8, cudaMemcpyDeviceToDevice,
                             slot.stream));
    RSM_CUDA(launch_trace_M(D, 1, slot.stream));
    for (int k = 2; k <= 5; ++k) RSM_CUDA(cudaEventRecord(slot.ev[k], slot.stream));
  }
  if ((st = launch_batch(b, slot, fp64, shift, given_M == nullptr)) != RSM_OK) return st;
  if ((st = enqueue_readback(b, slot)) != RSM_OK) return st;
  RSM_CUDA(cudaStreamSynchronize(slot.stream));
  // Accept the result when the factorisation succeeded and the a-posteriori
  // eigenvector bound (residual norm over the eigen-gap) is small; otherwise
  // redo the eigen stage with the FP64 factor (and then larger shifts).
  bool timed_out = false;  // a bounded device-side wait ran out (counters[6])
  for (int attempt = 0; attempt < 3; ++attempt) {
    bool redo = false;
    for (int i = 0; i < count; ++i) {
      const unsigned long long* c = reinterpret_cast<const unsigned long long*>(hp + (size_t)i * kReadback);
      const double* stats = reinterpret_cast<const double*>(hp + (size_t)i * kReadback + kCountersBytes);
      const int r = ps[i].r;
      const double gap = stats[r] - stats[r - 1];
      const double trace = given_M || b.l1 ? stats[kStatTrace]
                           : ps[i].variant == RSM_ROWS_RANDOM ? (double)c[7]
                                                              : (double)c[0] * b.dv[i].nm;
      const bool determined = (given_M || c[0] > 0) && stats[r] > kRankTol * trace;
      const double est = stats[34] / (gap > 0.0 ? gap : 1e-300);
      if (c[3] != 0 || (!fp64 && determined && !(est <= kEigErrTol))) redo = true;
      if (c[6] != 0) timed_out = true;
    }
    if (!redo || timed_out) break;
    if (fp64)
      shift *= 100.0;
    else {
      fp64 = true;
      shift = kShiftRel64;
    }
    for (int i = 0; i < count; ++i) RSM_CUDA(cudaMemsetAsync(b.descs[i].counters + 3, 0, 16, slot.stream));
    RSM_CUDA(cudaMemsetAsync(static_cast<unsigned char*>(slot.ws.ptr) + b.fail_count_off, 0, 8, slot.stream));
    RSM_CUDA(cudaMemsetAsync(static_cast<unsigned char*>(slot.ws.ptr) + b.sync_off, 0, b.sync_bytes, slot.stream));
    for (int i = 0; i < count; ++i)
      RSM_CUDA(cudaMemsetAsync(b.descs[i].tflag, 0, (size_t)3 * b.dv[i].nblk * b.dv[i].nblk * 4, slot.stream));
    if ((st = launch_batch(b, slot, fp64, shift, false)) != RSM_OK) return st;
    if ((st = enqueue_readback(b, slot)) != RSM_OK) return st;
    RSM_CUDA(cudaStreamSynchronize(slot.stream));
  }
  float ms[9] = {0};
  for (int k = 0; k < 8; ++k) cudaEventElapsedTime(&ms[k], slot.ev[k], slot.ev[k + 1]);
  cudaEventElapsedTime(&ms[8], slot.ev[0], slot.ev[8]);
  const int64_t launches = g_kernel_launches - launches0;
  int first_bad = RSM_OK;
  for (int i = 0; i < count; ++i) {
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(hp + (size_t)i * kReadback);
    const double* stats = reinterpret_cast<const double*>(hp + (size_t)i * kReadback + kCountersBytes);
    rsm_result r{};
    r.accepted_trials = (int64_t)c[0];
    r.rows_underdetermined = (int64_t)c[4];
    r.rows_selected = (int64_t)c[5];
    r.kernel_launches = launches;
    r.eig_factor_bits = fp64 ? 64 : 32;
    r.eig_iterations = (int32_t)stats[43];
    r.n_eig = b.dv[i].kx;
    for (int k = 0; k < 32; ++k) r.eig_M[k] = k < r.n_eig ? stats[k] : 0.0;
    r.eig_residual = stats[34];
    const double trace = given_M || b.l1 ? stats[kStatTrace]
                         : ps[i].variant == RSM_ROWS_RANDOM ? (double)c[7]
                                                            : (double)c[0] * b.dv[i].nm;
    r.e_known_rms = b.dv[i].solve_u ? stats[33] : NAN;
    int status = RSM_OK;
    if (c[6] != 0)
      status = RSM_ERR_TIMEOUT;
    else if ((!given_M && c[0] == 0) || !(r.eig_M[ps[i].r] > kRankTol * trace))
      status = RSM_ERR_UNDERDETERMINED;
    else if (c[3] != 0)
      status = RSM_ERR_UNDERDETERMINED;
    else if (c[4] > 0)
      status = RSM_ERR_ROWS_UNDERDETERMINED;
    r.status = status;
    r.trials = ps[i].trials;
    r.coverage = ps[i].coverage && c[1] > 0 ? (double)c[8] / (double)c[1] : NAN;
    if (ps[i].debug_visited)
      RSM_CUDA(cudaMemcpyAsync(ps[i].debug_visited, b.descs[i].visited, (size_t)ps[i].n * b.dv[i].ldb * 4,
                               cudaMemcpyDeviceToDevice, slot.stream));
    for (int k = 0; k < 9; ++k) r.stage_ms[k] = ms[k];
    if (res) res[i] = r;
    if (status != RSM_OK && first_bad == RSM_OK) first_bad = status;
  }
  bool copies = false;
  for (int i = 0; i < count; ++i) copies |= ps[i].debug_visited != nullptr;
  if (copies) RSM_CUDA(cudaStreamSynchronize(slot.stream));
  (void)h;
  return first_bad;
}

int validate_all(const rsm_problem* ps, int count) {
  for (int i = 0; i < count; ++i) {
    Derived dv;
    std::string why;
    int st = validate_problem(ps[i], dv, &why);
    if (st != RSM_OK) return fail(st, "problem " + std::to_string(i) + ": " + why);
    if (ps[i].gram_prec != ps[0].gram_prec || ps[i].solve_prec != ps[0].solve_prec)
      return fail(RSM_ERR_INVALID_ARG, "all problems of a batch must share gram_prec and solve_prec");
    if ((ps[i].norm == 1) != (ps[0].norm == 1) || ps[i].irls_iters != ps[0].irls_iters)
      return fail(RSM_ERR_INVALID_ARG, "all problems of a batch must share norm and irls_iters");
  }
  return RSM_OK;
}

// Problems with trials == 0: count their known entries on the device (one small
// kernel each, one synchronisation), then draw the number of submatrices that
// visits each known entry with probability >= epsilon (rsm_plan_trials).  `out`
// stays empty when every problem gives its trial count.
int plan_missing_trials(rsm_handle* h, const rsm_problem* ps, int count, std::vector<rsm_problem>& out) {
  bool any = false;
  for (int i = 0; i < count; ++i) any |= ps[i].trials == 0;
  if (!any) return RSM_OK;
  out.assign(ps, ps + count);
  Slot& slot = h->main;
  int st = slot.plan.reserve((size_t)count * 8);
  if (st != RSM_OK) return st;
  if ((st = slot.host.reserve((size_t)count * 8)) != RSM_OK) return st;
  unsigned long long* dcnt = static_cast<unsigned long long*>(slot.plan.ptr);
  RSM_CUDA(cudaMemsetAsync(dcnt, 0, (size_t)count * 8, slot.stream));
  for (int i = 0; i < count; ++i) {
    const rsm_problem& p = ps[i];
    if (p.trials != 0) continue;
    if (!(p.epsilon > 0.0 && p.epsilon < 1.0))
      return fail(RSM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": trials == 0 needs 0 < epsilon < 1");
    if (p.debug_cols || p.debug_row_counts || p.debug_Z)
      return fail(RSM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": planned trials exclude per-trial debug outputs");
    if (!p.W || p.m < 1 || p.n < 1 || p.ldw < p.m)
      return fail(RSM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": W, m, n, ldw");
    RSM_CUDA(launch_count_known(p.W, p.ldw, p.m, p.n, dcnt + i, slot.stream));
  }
  RSM_CUDA(cudaMemcpyAsync(slot.host.ptr, dcnt, (size_t)count * 8, cudaMemcpyDeviceToHost, slot.stream));
  RSM_CUDA(cudaStreamSynchronize(slot.stream));
  const unsigned long long* known = static_cast<const unsigned long long*>(slot.host.ptr);
  for (int i = 0; i < count; ++i) {
    if (ps[i].trials != 0) continue;
    const rsm_problem& p = ps[i];
    const double rho = (double)known[i] / ((double)p.m * (double)p.n);
    const int32_t size = p.l ? p.l : p.r + 1;
    rsm_trial_plan plan{};
    if (rho <= 0.0 || rsm_plan_trials(p.m, p.n, rho, p.r, size, p.variant, p.epsilon, &plan) != RSM_OK ||
        !(plan.trials < 68719476736.0))
      return fail(RSM_ERR_INVALID_ARG, "problem " + std::to_string(i) + ": no trial count reaches epsilon");
    out[i].trials = std::max<int64_t>(1, (int64_t)std::ceil(plan.trials));
  }
  return RSM_OK;
}

}  // namespace

extern "C" {

const char* rsm_version(void) { return "rsm-gb300 0.1.0 (sm_103a)"; }

size_t rsm_struct_size(int32_t which) {
  switch (which) {
    case 0: return sizeof(rsm_config);
    case 1: return sizeof(rsm_problem);
    case 2: return sizeof(rsm_result);
    default: return 0;
  }
}

const char* rsm_status_string(int32_t s) {
  switch (s) {
    case RSM_OK: return "ok";
    case RSM_ERR_INVALID_ARG: return "invalid argument";
    case RSM_ERR_NO_MEMORY: return "out of device memory or above the HBM budget";
    case RSM_ERR_UNDERDETERMINED: return "underdetermined: M has more than r null directions";
    case RSM_ERR_ROWS_UNDERDETERMINED: return "some rows have fewer than r known entries";
    case RSM_ERR_TIMEOUT: return "timed out";
    case RSM_ERR_CANCELLED: return "cancelled";
    case RSM_ERR_CUDA: return "CUDA error";
    case RSM_ERR_NOT_IMPLEMENTED: return "not implemented";
    case RSM_PENDING: return "pending";
    case RSM_ERR_QUEUE_FULL: return "admission queue full";
    default: return "unknown status";
  }
}

const char* rsm_last_error(void) { return g_last_error.c_str(); }

size_t rsm_footprint_bytes(const rsm_problem* p) {
  if (!p) return 0;
  Derived dv;
  if (validate_problem(*p, dv, nullptr) != RSM_OK) return 0;
  return problem_footprint(*p, dv);
}

int32_t rsm_create(const rsm_config* config, rsm_handle** out) {
  if (!out) return fail(RSM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  rsm_config cfg{};
  if (config) cfg = *config;
  int ndev = 0;
  RSM_CUDA(cudaGetDeviceCount(&ndev));
  if (cfg.device < 0 || cfg.device >= ndev) return fail(RSM_ERR_INVALID_ARG, "device ordinal out of range");
  RSM_CUDA(cudaSetDevice(cfg.device));
  if (cfg.max_slots <= 0) cfg.max_slots = 4;
  if (cfg.max_slots > 64) return fail(RSM_ERR_INVALID_ARG, "max_slots > 64");
  if (cfg.wait_timeout_ns == 0) cfg.wait_timeout_ns = 10ull * 1000 * 1000 * 1000;
  auto h = std::make_unique<rsm_handle>();
  h->cfg = cfg;
  h->device = cfg.device;
  h->fault = cfg.fault_inject;
  size_t free_b = 0, total_b = 0;
  RSM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  h->budget = cfg.hbm_budget_bytes ? cfg.hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
  int st = h->main.init(static_cast<cudaStream_t>(cfg.stream));
  if (st != RSM_OK) return st;
  *out = h.release();
  return RSM_OK;
}

int32_t rsm_decompose_batch(rsm_handle* h, const rsm_problem* ps_in, int32_t count, rsm_result* res) {
  if (!h || !ps_in || count < 1) return fail(RSM_ERR_INVALID_ARG, "handle, problems and count >= 1 are required");
  std::lock_guard<std::mutex> lk(h->api_mu);
  DeviceGuard dg(h->device);
  RSM_CUDA(dg.err);
  bool planning = false;
  for (int i = 0; i < count; ++i) planning |= ps_in[i].trials == 0;
  if (!planning) {
    int st = validate_all(ps_in, count);
    if (st != RSM_OK) return st;
  }
  if (h->main.own_stream) {
    // the handle's own stream does not order with the caller's work: start
    // after everything enqueued on the legacy default stream so far (which in
    // turn waits for the caller's blocking streams)
    RSM_CUDA(cudaEventRecord(h->main.ev_order, nullptr));
    RSM_CUDA(cudaStreamWaitEvent(h->main.stream, h->main.ev_order, 0));
  }
  std::vector<rsm_problem> planned;
  const rsm_problem* ps = ps_in;
  int st = plan_missing_trials(h, ps_in, count, planned);
  if (st != RSM_OK) return st;
  if (!planned.empty()) {
    ps = planned.data();
    if ((st = validate_all(ps, count)) != RSM_OK) return st;
  }
  size_t need = 0;
  for (int i = 0; i < count; ++i) need += rsm_footprint_bytes(&ps[i]);
  if (need > h->budget) return fail(RSM_ERR_NO_MEMORY, "batch footprint above the handle's HBM budget");
  if (h->fault & RSM_FAULT_ALLOC) {
    h->fault &= ~RSM_FAULT_ALLOC;
    return fail(RSM_ERR_NO_MEMORY, "injected allocation failure");
  }
  return run_batch(h, h->main, ps, count, res);
}

int32_t rsm_decompose(rsm_handle* h, const rsm_problem* p, rsm_result* res) {
  rsm_result tmp{};
  int st = rsm_decompose_batch(h, p, 1, &tmp);
  if (res) *res = tmp;
  if (st == RSM_OK || st == RSM_ERR_UNDERDETERMINED || st == RSM_ERR_ROWS_UNDERDETERMINED) return tmp.status;
  if (res) res->status = st;
  return st;
}

// ---------------------------------------------------------------- autotuning

int32_t rsm_autotune(rsm_handle* h, const rsm_problem* p_in, int32_t reps, rsm_tune* out) {
  if (!h || !p_in) return fail(RSM_ERR_INVALID_ARG, "handle and problem are required");
  if (reps == 0) reps = 3;
  if (reps < 1 || reps > 100) return fail(RSM_ERR_INVALID_ARG, "reps must be 1..100 (0 -> 3)");
  if (p_in->variant == RSM_ROWS_RANDOM)
    return fail(RSM_ERR_INVALID_ARG, "the rows variant has no Gram schedule to tune");
  std::lock_guard<std::mutex> lk(h->api_mu);
  DeviceGuard dg(h->device);
  RSM_CUDA(dg.err);
  if (h->main.own_stream) {
    RSM_CUDA(cudaEventRecord(h->main.ev_order, nullptr));
    RSM_CUDA(cudaStreamWaitEvent(h->main.stream, h->main.ev_order, 0));
  }
  std::vector<rsm_problem> planned;
  int st = plan_missing_trials(h, p_in, 1, planned);
  if (st != RSM_OK) return st;
  rsm_problem p = planned.empty() ? *p_in : planned[0];
  p.U = nullptr;  // the Gram stage is what is timed: stop after V
  p.debug_cols = nullptr;
  p.debug_row_counts = nullptr;
  p.debug_Z = nullptr;
  p.debug_visited = nullptr;
  if ((st = validate_all(&p, 1)) != RSM_OK) return st;
  const size_t need = rsm_footprint_bytes(&p);
  if (need > h->budget) return fail(RSM_ERR_NO_MEMORY, "problem footprint above the handle's HBM budget");
  // candidates: the default first, then every slab size and occupancy, then one warp per submatrix
  const int mode = p.gram_prec == RSM_PREC_F64 ? 0 : p.gram_prec == RSM_PREC_F32X2 ? 1 : 2;
  const int l = p.l ? p.l : p.r + 1;
  // (the occupancy variant only where its build differs: more registers per thread)
  std::vector<Tune> cand{Tune{}};
  if (slab_supported(mode, l, p.y_dtype)) {
    const bool occ = gram_slab_regs(mode, l, 1) != gram_slab_regs(mode, l, 0);
    for (int mib : {8, 16, 32, 64})
      for (int v = 0; v <= (occ ? 1 : 0); ++v)
        if (!(mib == 32 && v == 0)) cand.push_back(Tune{0, mib, v});
  }
  cand.push_back(Tune{1, 32, 0});
  // between timed runs, a write larger than L2 evicts the previous run's Y, as a
  // stream of calls on different problems would
  constexpr size_t kFlush = (size_t)256 << 20;
  DevBuf flush;
  struct Release {
    DevBuf& b;
    ~Release() { b.release(); }
  } release_flush{flush};
  const bool flushing = need + kFlush <= h->budget && flush.reserve(kFlush) == RSM_OK;
  std::vector<double> best_ms(cand.size(), INFINITY);
  for (size_t c = 0; c < cand.size(); ++c) {
    for (int k = 0; k <= reps; ++k) {  // k == 0: untimed warm-up
      if (flushing) RSM_CUDA(launch_zero16(flush.ptr, kFlush, h->main.stream));
      rsm_result r{};
      st = run_batch(h, h->main, &p, 1, &r, nullptr, &cand[c]);
      if (st != RSM_OK && st != RSM_ERR_UNDERDETERMINED && st != RSM_ERR_ROWS_UNDERDETERMINED) return st;
      if (k > 0) best_ms[c] = std::min(best_ms[c], (double)r.stage_ms[3]);
    }
  }
  size_t best = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (best_ms[c] < best_ms[best]) best = c;
  rsm_tune t{};
  t.schedule = cand[best].schedule;
  t.slab_mib = cand[best].slab_mib;
  t.variant = cand[best].variant;
  t.candidates = (int32_t)cand.size();
  t.gram_ms = best_ms[best];
  t.default_ms = best_ms[0];
  {
    std::lock_guard<std::mutex> tl(h->tune_mu);
    h->tuned[tune_key(p)] = {cand[best], t};
  }
  if (out) *out = t;
  return RSM_OK;
}

int32_t rsm_autotune_lookup(rsm_handle* h, const rsm_problem* p, rsm_tune* out) {
  if (!h || !p) return -RSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> tl(h->tune_mu);
  auto it = h->tuned.find(tune_key(*p));
  if (it == h->tuned.end()) return 0;
  if (out) *out = it->second.second;
  return 1;
}

int32_t rsm_autotune_clear(rsm_handle* h) {
  if (!h) return fail(RSM_ERR_INVALID_ARG, "handle is NULL");
  std::lock_guard<std::mutex> tl(h->tune_mu);
  h->tuned.clear();
  return RSM_OK;
}

int32_t rsm_autotune_save(rsm_handle* h, const char* path) {
  if (!h || !path) return fail(RSM_ERR_INVALID_ARG, "handle and path are required");
  std::lock_guard<std::mutex> tl(h->tune_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(RSM_ERR_INVALID_ARG, std::string("cannot write ") + path);
  std::fprintf(f, "# rsm autotune v1: gram_prec y_dtype l n log2m schedule slab_mib variant gram_ms default_ms\n");
  for (const auto& kv : h->tuned) {
    const auto& k = kv.first;
    const rsm_tune& t = kv.second.second;
    std::fprintf(f, "%lld %lld %lld %lld %lld %d %d %d %.6g %.6g\n", (long long)k[0], (long long)k[1],
                 (long long)k[2], (long long)k[3], (long long)k[4], t.schedule, t.slab_mib, t.variant, t.gram_ms,
                 t.default_ms);
  }
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  return ok ? RSM_OK : fail(RSM_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

int32_t rsm_autotune_load(rsm_handle* h, const char* path) {
  if (!h || !path) return fail(RSM_ERR_INVALID_ARG, "handle and path are required");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(RSM_ERR_INVALID_ARG, std::string("cannot read ") + path);
  std::map<std::vector<int64_t>, std::pair<Tune, rsm_tune>> got;
  char line[512];
  int lineno = 0;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n') continue;
    long long k[5];
    int sc, mib, v;
    double g, d;
    const bool ok = std::sscanf(line, "%lld %lld %lld %lld %lld %d %d %d %lf %lf", &k[0], &k[1], &k[2], &k[3], &k[4],
                                &sc, &mib, &v, &g, &d) == 10 &&
                    (sc == 0 || sc == 1) && (mib == 8 || mib == 16 || mib == 32 || mib == 64) && (v == 0 || v == 1) &&
                    k[2] >= 2 && k[3] >= 2 && k[4] >= 0 && k[4] < 63;
    if (!ok) {
      std::fclose(f);
      return fail(RSM_ERR_INVALID_ARG, std::string(path) + ":" + std::to_string(lineno) + ": malformed entry");
    }
    rsm_tune t{};
    t.schedule = sc;
    t.slab_mib = mib;
    t.variant = v;
    t.gram_ms = g;
    t.default_ms = d;
    got[{k[0], k[1], k[2], k[3], k[4]}] = {Tune{sc, mib, v}, t};
  }
  std::fclose(f);
  std::lock_guard<std::mutex> tl(h->tune_mu);
  for (auto& kv : got) h->tuned[kv.first] = kv.second;
  return RSM_OK;
}

// ---------------------------------------------------------------- serving

namespace {

// Continuous batching: a free slot admits the oldest queued request whose
// footprint fits the free budget, then every further queued request of the same
// precisions that still fits (oldest first, up to kServeBatch), and runs them as one batch on its own
// stream.  Other slots keep admitting while this batch is on the GPU, so the
// work of requests that arrive while others run overlaps on the device.
constexpr int kServeBatch = 16;

void worker_loop(rsm_handle* h, int slot_id) {
  cudaSetDevice(h->device);
  Slot& slot = h->slots[slot_id];
  for (;;) {
    std::vector<std::shared_ptr<Request>> reqs;
    {
      std::unique_lock<std::mutex> lk(h->mu);
      for (;;) {
        if (h->stopping) return;
        if (!(h->fault & RSM_FAULT_STALL) && !h->queue.empty()) {
          for (auto it = h->queue.begin(); it != h->queue.end() && (int)reqs.size() < kServeBatch;) {
            auto& r = h->reqs[*it];
            const bool same_prec = reqs.empty() || (r->prob.gram_prec == reqs[0]->prob.gram_prec &&
                                                    r->prob.solve_prec == reqs[0]->prob.solve_prec &&
                                                    (r->prob.norm == 1) == (reqs[0]->prob.norm == 1) &&
                                                    r->prob.irls_iters == reqs[0]->prob.irls_iters);
            if (same_prec && r->footprint + h->in_use <= h->budget) {
              h->in_use += r->footprint;
              r->state = 1;
              r->t_start = std::chrono::steady_clock::now();
              reqs.push_back(r);
              it = h->queue.erase(it);
            } else {
              ++it;
            }
          }
          if (!reqs.empty()) break;
        }
        h->cv.wait(lk);
      }
    }
    const int count = (int)reqs.size();
    // each request's inputs are complete once the work its submitter had
    // enqueued before rsm_submit has run
    for (auto& r : reqs)
      if (r->ready) {
        cudaStreamWaitEvent(slot.stream, r->ready, 0);
        cudaEventDestroy(r->ready);
        r->ready = nullptr;
      }
    std::vector<rsm_problem> probs(count);
    std::vector<rsm_result> res(count);
    for (int i = 0; i < count; ++i) probs[i] = reqs[i]->prob;
    const int st = run_batch(h, slot, probs.data(), count, res.data());
    {
      std::lock_guard<std::mutex> lk(h->mu);
      const auto t_end = std::chrono::steady_clock::now();
      for (int i = 0; i < count; ++i) {
        auto& req = reqs[i];
        if (st != RSM_OK && st != RSM_ERR_UNDERDETERMINED && st != RSM_ERR_ROWS_UNDERDETERMINED) res[i].status = st;
        req->t_end = t_end;
        res[i].queue_ms = std::chrono::duration<double, std::milli>(req->t_start - req->t_submit).count();
        res[i].run_ms = std::chrono::duration<double, std::milli>(req->t_end - req->t_start).count();
        req->res = res[i];
        req->state = 2;
        h->in_use -= req->footprint;
      }
    }
    h->cv.notify_all();
    h->done_cv.notify_all();
  }
}

int ensure_workers(rsm_handle* h) {
  if (!h->workers.empty()) return RSM_OK;
  h->slots.resize(h->cfg.max_slots);
  for (auto& s : h->slots) {
    int st = s.init(nullptr);
    if (st != RSM_OK) return st;
  }
  for (int i = 0; i < h->cfg.max_slots; ++i) h->workers.emplace_back(worker_loop, h, i);
  return RSM_OK;
}

}  // namespace

int32_t rsm_submit_on(rsm_handle* h, const rsm_problem* p, void* stream, uint64_t* ticket) {
  if (!h || !p || !ticket) return fail(RSM_ERR_INVALID_ARG, "handle, problem and ticket are required");
  int st = validate_all(p, 1);
  if (st != RSM_OK) return st;
  const size_t fp = rsm_footprint_bytes(p);
  std::lock_guard<std::mutex> lk(h->mu);
  if (fp > h->budget || (h->fault & RSM_FAULT_ADMISSION))
    return fail(RSM_ERR_NO_MEMORY, "footprint above the handle's HBM budget: never admissible");
  if (h->queue.size() >= 4096) return fail(RSM_ERR_QUEUE_FULL, "admission queue full");
  DeviceGuard dg(h->device);
  RSM_CUDA(dg.err);
  st = ensure_workers(h);
  if (st != RSM_OK) return st;
  cudaEvent_t ready = nullptr;
  RSM_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  cudaError_t er = cudaEventRecord(ready, static_cast<cudaStream_t>(stream));
  if (er != cudaSuccess) {
    cudaEventDestroy(ready);
    return cuda_fail(er, "cudaEventRecord on the submitting stream");
  }
  auto r = std::make_shared<Request>();
  r->ready = ready;
  r->ticket = h->next_ticket++;
  r->prob = *p;
  r->footprint = fp;
  r->t_submit = std::chrono::steady_clock::now();
  h->reqs[r->ticket] = r;
  h->queue.push_back(r->ticket);
  *ticket = r->ticket;
  h->cv.notify_all();
  return RSM_OK;
}

int32_t rsm_submit(rsm_handle* h, const rsm_problem* p, uint64_t* ticket) {
  return rsm_submit_on(h, p, nullptr, ticket);
}

int32_t rsm_poll(rsm_handle* h, uint64_t ticket, rsm_result* res) {
  if (!h) return fail(RSM_ERR_INVALID_ARG, "handle is NULL");
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return fail(RSM_ERR_INVALID_ARG, "unknown ticket");
  if (it->second->state != 2) return RSM_PENDING;
  if (res) *res = it->second->res;
  return it->second->res.status;
}

int32_t rsm_wait(rsm_handle* h, uint64_t ticket, uint64_t timeout_ns, rsm_result* res) {
  if (!h) return fail(RSM_ERR_INVALID_ARG, "handle is NULL");
  if (timeout_ns == 0) timeout_ns = h->cfg.wait_timeout_ns;
  std::unique_lock<std::mutex> lk(h->mu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return fail(RSM_ERR_INVALID_ARG, "unknown ticket");
  auto req = it->second;
  const bool done = h->done_cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [&] { return req->state == 2; });
  if (!done) return fail(RSM_ERR_TIMEOUT, "request still pending after the wait limit");
  if (res) *res = req->res;
  return req->res.status;
}

int32_t rsm_cancel(rsm_handle* h, uint64_t ticket) {
  if (!h) return fail(RSM_ERR_INVALID_ARG, "handle is NULL");
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return fail(RSM_ERR_INVALID_ARG, "unknown ticket");
  auto& r = it->second;
  if (r->state != 0) return fail(RSM_ERR_INVALID_ARG, "request already started");
  h->queue.erase(std::remove(h->queue.begin(), h->queue.end(), ticket), h->queue.end());
  if (r->ready) {
    cudaEventDestroy(r->ready);
    r->ready = nullptr;
  }
  r->state = 2;
  r->res = rsm_result{};
  r->res.status = RSM_ERR_CANCELLED;
  h->done_cv.notify_all();
  return RSM_OK;
}

int32_t rsm_release(rsm_handle* h, uint64_t ticket) {
  if (!h) return fail(RSM_ERR_INVALID_ARG, "handle is NULL");
  std::lock_guard<std::mutex> lk(h->mu);
  auto it = h->reqs.find(ticket);
  if (it == h->reqs.end()) return fail(RSM_ERR_INVALID_ARG, "unknown ticket");
  if (it->second->state != 2) return fail(RSM_ERR_INVALID_ARG, "request not finished");
  h->reqs.erase(it);
  return RSM_OK;
}

void rsm_destroy(rsm_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  {
    std::unique_lock<std::mutex> lk(h->mu);
    // let running requests finish (bounded by the wait limit), drop queued ones
    for (uint64_t t : h->queue) {
      auto it = h->reqs.find(t);
      if (it != h->reqs.end() && it->second->ready) {
        cudaEventDestroy(it->second->ready);
        it->second->ready = nullptr;
      }
    }
    h->queue.clear();
    h->done_cv.wait_for(lk, std::chrono::nanoseconds(h->cfg.wait_timeout_ns), [&] {
      for (auto& kv : h->reqs)
        if (kv.second->state == 1) return false;
      return true;
    });
    h->stopping = true;
  }
  h->cv.notify_all();
  for (auto& t : h->workers) t.join();
  for (auto& s : h->slots) s.destroy();
  h->main.destroy();
  delete h;
}

// ---------------------------------------------------------------- stage entry points

int32_t rsm_pack_mask(const uint8_t* W, int64_t ldw, int64_t m, int64_t n, uint32_t* bits, int64_t ldb, void* stream) {
  if (!W || !bits || m < 1 || n < 1 || ldw < m || ldb < (m + 31) / 32)
    return fail(RSM_ERR_INVALID_ARG, "pack_mask: bad pointer or size");
  ProbDesc d{};
  d.m = m;
  d.n = n;
  d.W = W;
  d.ldw = ldw;
  d.bits = bits;
  d.ldb = ldb;
  unsigned long long* cnt = nullptr;
  int64_t* offs = nullptr;
  ProbDesc* dd = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // small transient device copies of the descriptor and offsets
  RSM_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dd), sizeof(ProbDesc) + 64, s));
  offs = reinterpret_cast<int64_t*>(reinterpret_cast<unsigned char*>(dd) + sizeof(ProbDesc));
  cnt = reinterpret_cast<unsigned long long*>(offs + 2);
  d.counters = cnt - 1;  // counters[1] is the known-entry count
  const int64_t nblocks = n * ((ldb + 255) / 256);
  int64_t h_off[2] = {0, nblocks};
  RSM_CUDA(cudaMemcpyAsync(dd, &d, sizeof(ProbDesc), cudaMemcpyHostToDevice, s));
  RSM_CUDA(cudaMemcpyAsync(offs, h_off, sizeof(h_off), cudaMemcpyHostToDevice, s));
  RSM_CUDA(cudaMemsetAsync(cnt, 0, 8, s));
  cudaError_t e = launch_pack_mask(dd, offs, 1, nblocks, s);
  RSM_CUDA(cudaFreeAsync(dd, s));
  if (e != cudaSuccess) return cuda_fail(e, "pack_mask");
  return RSM_OK;
}

int32_t rsm_sample_columns(int64_t n, int32_t l, int64_t t0, int64_t count, uint64_t seed, uint32_t problem_id,
                           int32_t variant, int32_t* cols, void* stream) {
  if (!cols || n < 1 || l < 1 || l > n || l > kMaxL || t0 < 0 || count < 0 ||
      (variant != RSM_COLS_RANDOM && variant != RSM_COLS_ADJACENT))
    return fail(RSM_ERR_INVALID_ARG, "sample_columns: bad argument");
  ProbDesc d{};
  d.n = n;
  d.l = l;
  d.seed = seed;
  d.pid = problem_id;
  d.variant = variant;
  cudaError_t e = launch_sample_range(d, t0, count, cols, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "sample_columns");
  return RSM_OK;
}

int32_t rsm_select_rows(const uint32_t* bits, int64_t ldb, int64_t m, const int32_t* cols, int32_t l, int64_t count,
                        const int64_t* row_offsets, int32_t* rows, int32_t* row_counts, void* stream) {
  if (!bits || !cols || !row_offsets || !rows || !row_counts || m < 1 || l < 1 || l > kMaxL || count < 0 ||
      ldb < (m + 31) / 32)
    return fail(RSM_ERR_INVALID_ARG, "select_rows: bad argument");
  cudaError_t e = launch_select_rows(bits, ldb, m, cols, l, count, row_offsets, rows, row_counts,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "select_rows");
  return RSM_OK;
}

int32_t rsm_eig_smallest(rsm_handle* h, const double* M, int64_t n, int32_t r, double* V, int64_t ldv,
                         rsm_result* res) {
  if (!h || !M || !V) return fail(RSM_ERR_INVALID_ARG, "eig_smallest: handle, M and V are required");
  if (n < 2 || n > 32768 || r < 1 || r >= n || r >= kMaxL || ldv < n)
    return fail(RSM_ERR_INVALID_ARG, "eig_smallest: need 2 <= n <= 32768, 1 <= r < min(n, 32), ldv >= n");
  rsm_problem p{};
  p.m = n;
  p.n = n;
  p.r = r;
  p.l = r + 1;
  p.trials = 1;
  p.Y = M;  // never read: the stages that read Y and W are skipped
  p.W = reinterpret_cast<const uint8_t*>(M);
  p.ldy = p.ldw = n;
  p.V = V;
  p.ldv = ldv;
  p.y_dtype = RSM_F64;
  p.gram_prec = p.solve_prec = RSM_PREC_F64;
  Derived dv;
  std::string why;
  int st = validate_problem(p, dv, &why);
  if (st != RSM_OK) return fail(st, "eig_smallest: " + why);
  std::lock_guard<std::mutex> lk(h->api_mu);
  DeviceGuard dg(h->device);
  RSM_CUDA(dg.err);
  if (rsm_footprint_bytes(&p) > h->budget) return fail(RSM_ERR_NO_MEMORY, "footprint above the handle's HBM budget");
  if (h->main.own_stream) {
    RSM_CUDA(cudaEventRecord(h->main.ev_order, nullptr));
    RSM_CUDA(cudaStreamWaitEvent(h->main.stream, h->main.ev_order, 0));
  }
  rsm_result tmp{};
  st = run_batch(h, h->main, &p, 1, &tmp, M);
  tmp.accepted_trials = 0;
  tmp.rows_selected = 0;
  if (res) *res = tmp;
  if (st == RSM_OK || st == RSM_ERR_UNDERDETERMINED) return tmp.status;
  if (res) res->status = st;
  return st;
}

int32_t rsm_check_fp64_math(const double* x, int64_t count, double* out, void* stream) {
  if (!x || !out || count < 0) return fail(RSM_ERR_INVALID_ARG, "check_fp64_math: bad argument");
  cudaError_t e = launch_fp64_math(x, count, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "check_fp64_math");
  return RSM_OK;
}

}  // extern "C"
