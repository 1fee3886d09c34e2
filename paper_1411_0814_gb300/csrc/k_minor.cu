// Stages a5 + a6: minor eigenvectors of each trial's Gram and their exact,
// order-independent accumulation into M.
//
// a5: the right singular vectors of A_t for its l - r smallest singular values
// (Section III) are the eigenvectors of G_t = A_t^T A_t for its smallest
// eigenvalues.  One warp per trial: FP32 Jacobi (jacobi.cuh) for the eigenbasis,
// then FP64 Newton refinement of the minor subspace (see k_minor_scatter).
//
// a6: M = Xi Xi^T = sum_t sum_j xi xi^T with xi = e(zeta) (eq. get_xi, eq. XI).
// Trial t adds the projector Z_t Z_t^T (l x l) to M[C_t, C_t].  Contributions
// are rounded to 64-bit fixed point (2^-f, f chosen so no sum can overflow)
// and added with integer atomics: integer addition is associative, so the
// result is bit-identical for any order of the trials.
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "jacobi.cuh"
#include "kernels.h"
#include "small_df.cuh"

namespace rsm {

constexpr int kMinorWarps = 4;
constexpr int kNewtonSteps = 4;

// Relative gap across the minor split below which a trial takes the FP64
// polish path instead of Newton steps from the FP32 Jacobi basis.  FP64 Gram:
// 1e-4 (four steps reach FP64 from an FP32 basis off by u32 / 1e-4).  FP32
// Gram: its own rounding defines the minor subspace only to ~u32 ||G|| / gap,
// and the single Newton step from the FP32 basis leaves ~(u32 ||G|| / gap)^2,
// below that limit for any gap above u32 ||G||; 1e-5 keeps a wide margin.
__device__ __forceinline__ float split_tol(const ProbDesc& d) { return d.gram_fp32 ? 1e-5f : 1e-4f; }

// Shared memory per warp (row stride ls = lmax + 1): G (FP64), the FP32 copy
// and FP32 eigenvectors, Z and a second FP64 work matrix, three FP64 vectors.
__host__ __device__ inline size_t minor_smem_per_warp(int lmax) {
  const int ls = lmax + 1;
  return sizeof(double) * (size_t)lmax * ls + 2 * sizeof(float) * (size_t)lmax * ls +
         sizeof(double) * (2 * (size_t)lmax * ls + 3 * (size_t)ls);
}

// Newton refinement of the n_minor columns of Z (l x n_minor, FP64) against the
// complement eigenvectors of the FP32 basis Qf (eigenvalues on Sf's diagonal).
// Qd (l x l, stride ls) and lam (l) are FP64 copies of the FP32 eigenvectors and
// eigenvalues, made once per trial so the steps convert nothing.  The steps stop
// early once every correction is below `stop` (z has unit norm), 1e-17, or
// after max_steps.  An FP32 Gram takes a single step: its own rounding (~1e-7
// relative) already bounds how well its minor vectors are defined, and one
// step from the FP32 basis (error ~1e-7) leaves ~1e-14 (times ||G|| / gap).
// W = 32: one warp per trial; W = 16: one half warp per trial (lane = lane in the half).
template <int W = 32>
__device__ inline void newton_refine(const double* Gs, const double* Qd, const double* lam, double* Z, double* rv,
                                     double* cv, int l, int nm, int ls, const int* is_minor, double fro, double stop,
                                     int max_steps) {
  const int lane = threadIdx.x & (W - 1);
  const unsigned gmask = W == 32 ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
  for (int step = 0; step < max_steps; ++step) {
    double cmax = 0.0;
    for (int j = 0; j < nm; ++j) {
      double gz = 0.0, za = 0.0;
      if (lane < l) {
        za = Z[lane * nm + j];
        for (int b = 0; b < l; ++b) gz = fma(Gs[lane * ls + b], Z[b * nm + j], gz);
      }
      double th = za * gz;
#pragma unroll
      for (int o = W / 2; o; o >>= 1) th += __shfl_xor_sync(gmask, th, o);
      if (lane < l) rv[lane] = gz - th * za;
      __syncwarp(gmask);
      // block form: drop the part of r inside span(Z); only the part that leaves
      // the current minor subspace is corrected against the complement
      for (int k = 0; k < nm; ++k) {
        double zr = lane < l ? Z[lane * nm + k] * rv[lane] : 0.0;
#pragma unroll
        for (int o = W / 2; o; o >>= 1) zr += __shfl_xor_sync(gmask, zr, o);
        if (lane < l) rv[lane] -= zr * Z[lane * nm + k];
        __syncwarp(gmask);
      }
      if (lane < l) {
        double c = 0.0;
        if (!is_minor[lane]) {
          double qr = 0.0;
          for (int a = 0; a < l; ++a) qr = fma(Qd[a * ls + lane], rv[a], qr);
          c = qr * rcp64(lam[lane] - th);
        }
        cv[lane] = c;
        cmax = fmax(cmax, fabs(c));
      }
      __syncwarp(gmask);
      if (lane < l) {
        double zn = Z[lane * nm + j];
        for (int i = 0; i < l; ++i) zn = fma(-cv[i], Qd[lane * ls + i], zn);
        Z[lane * nm + j] = zn;
      }
      __syncwarp(gmask);
    }
#pragma unroll
    for (int o = W / 2; o; o >>= 1) cmax = fmax(cmax, __shfl_xor_sync(gmask, cmax, o));
    for (int j = 0; j < nm; ++j) {  // Gram-Schmidt (twice) in FP64
      for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < j; ++k) {
          double pr = lane < l ? Z[lane * nm + k] * Z[lane * nm + j] : 0.0;
#pragma unroll
          for (int o = W / 2; o; o >>= 1) pr += __shfl_xor_sync(gmask, pr, o);
          if (lane < l) Z[lane * nm + j] -= pr * Z[lane * nm + k];
          __syncwarp(gmask);
        }
      double nn = lane < l ? Z[lane * nm + j] * Z[lane * nm + j] : 0.0;
#pragma unroll
      for (int o = W / 2; o; o >>= 1) nn += __shfl_xor_sync(gmask, nn, o);
      const double inv = rsqrt64(nn);
      if (lane < l) Z[lane * nm + j] *= inv;
      __syncwarp(gmask);
    }
    if (cmax < stop) break;
  }
}

// a5: the FP32 Jacobi eigenbasis Q of G (accurate to FP32 rounding) separates
// the n_minor smallest eigenvalues from the rest; the minor subspace is then
// refined in FP64 by Newton corrections against the complement of Q:
//   z <- z - sum_{i not minor} q_i (q_i^T r') / (lambda_i - theta),
//   theta = z^T G z,  r = G z - theta z,  r' = r - Z Z^T r,
// followed by Gram-Schmidt.  Removing the part of r inside span(Z) (block
// Newton) keeps the fixed point exact when several minor vectors are kept.  The fixed point is an exact eigenvector of the
// FP64 Gram whatever the FP32 rounding of Q, and the error squares per step.
// One trial (global index g) by one warp; `counted`: the accepted-trial count
// already holds it (a trial handed over by k_minor_half).
__device__ __forceinline__ void minor_trial(const ProbDesc* __restrict__ descs, const int64_t* __restrict__ trial_off,
                                            int nprob, int lmax, int64_t g, bool counted, unsigned char* smraw) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.variant == 2) return;  // the row variant has its own kernels (k_rows.cu)
  const int64_t t = g - trial_off[p];
  const int l = d.l;
  const int ls = lmax + 1;
  unsigned char* base = smraw + (size_t)wid * minor_smem_per_warp(lmax);
  double* Gs = reinterpret_cast<double*>(base);
  float* Sf = reinterpret_cast<float*>(Gs + (size_t)lmax * ls);
  float* Qf = Sf + (size_t)lmax * ls;
  double* Z = reinterpret_cast<double*>(Qf + (size_t)lmax * ls);
  double* Wd = Z + (size_t)lmax * ls;  // FP64 work matrix of the fallback path
  double* gv = Wd + (size_t)lmax * ls;
  double* rv = gv + ls;
  double* cv = rv + ls;
  __shared__ JacobiScratchT<float> js[kMinorWarps];
  __shared__ JacobiScratchT<double> jsd[kMinorWarps];
  __shared__ int pick[kMinorWarps][kMaxL];
  __shared__ int is_minor[kMinorWarps][kMaxL];

  const int count = d.row_counts[t];
  if (count < l) {  // rejected trial (fewer than l rows, i.e. not more than r)
    if (d.debug_Z)
      for (int i = lane; i < l * d.n_minor; i += 32) d.debug_Z[t * l * d.n_minor + i] = 0.0;
    if (d.Zst)
      for (int i = lane; i < l * d.n_minor; i += 32) d.Zst[t * l * d.n_minor + i] = 0.0;
    return;
  }
  if (lane == 0 && !counted) atomicAdd(&d.counters[0], 1ull);

  // packed Gram -> full symmetric FP64 matrix and its FP32 copy
  const int P = l * (l + 1) / 2;
  const double* G = d.gram + t * P;
  for (int q = lane; q < P; q += 32) {
    int a = 0, rem = q;
    while (rem >= l - a) {
      rem -= l - a;
      ++a;
    }
    const int b = a + rem;
    const double v = G[q];
    Gs[a * ls + b] = v;
    Gs[b * ls + a] = v;
    Sf[a * ls + b] = (float)v;
    Sf[b * ls + a] = (float)v;
  }
  __syncwarp();
  const double fro = warp_frobenius(Gs, l, ls);
  warp_jacobi<float>(Sf, Qf, l, ls, js[wid], (float)(4.0 * FLT_EPSILON * fro));

  // the n_minor smallest eigenvalues (ties broken by index)
  const int nm = d.n_minor;
  const SmallDiv dnm((uint32_t)nm), dl((uint32_t)l);  // quotients by nm and l without integer division
  if (lane == 0) {
    for (int i = 0; i < l; ++i) is_minor[wid][i] = 0;
    for (int j = 0; j < nm; ++j) {
      int best = -1;
      for (int i = 0; i < l; ++i)
        if (!is_minor[wid][i] && (best < 0 || Sf[i * ls + i] < Sf[best * ls + best])) best = i;
      is_minor[wid][best] = 1;
      pick[wid][j] = best;
    }
  }
  __syncwarp();
  // Newton converges from the FP32 basis when every complement eigenvalue is at
  // least split_tol ||G|| away from the minor ones.  Otherwise (a nearly
  // degenerate pair across the split) the trial takes the FP32 Jacobi + FP64
  // polish path instead.
  float gap_min = 3.0e38f;
  if (lane < l && !is_minor[wid][lane])
    for (int j = 0; j < nm; ++j) gap_min = fminf(gap_min, fabsf(Sf[lane * ls + lane] - Sf[pick[wid][j] * ls + pick[wid][j]]));
#pragma unroll
  for (int o = 16; o; o >>= 1) gap_min = fminf(gap_min, __shfl_xor_sync(0xffffffffu, gap_min, o));
  const bool polish = gap_min < split_tol(d) * (float)fro;
  if (polish) {
    // eigen-decomposition of the FP64 Gram: eigenvalues on Gs's diagonal, vectors in Z (stride ls)
    warp_eig_mixed(Gs, Z, Sf, Qf, Wd, l, ls, js[wid], jsd[wid]);
    if (lane == 0) {
      for (int i = 0; i < l; ++i) is_minor[wid][i] = 0;
      for (int j = 0; j < nm; ++j) {
        int best = -1;
        for (int i = 0; i < l; ++i)
          if (!is_minor[wid][i] && (best < 0 || Gs[i * ls + i] < Gs[best * ls + best])) best = i;
        is_minor[wid][best] = 1;
        pick[wid][j] = best;
      }
    }
    __syncwarp();
    // compact the picked columns into Wd as the l x n_minor minor basis
    for (int it = lane; it < l * nm; it += 32) {
      const int a = dnm.q(it), j = dnm.r(it);
      Wd[a * nm + j] = Z[a * ls + pick[wid][j]];
    }
    __syncwarp();
    for (int it = lane; it < l * nm; it += 32) Z[it] = Wd[it];
    __syncwarp();
  } else {
    for (int it = lane; it < l * nm; it += 32) {
      const int a = dnm.q(it), j = dnm.r(it);
      Z[a * nm + j] = (double)Qf[a * ls + pick[wid][j]];
    }
    for (int it = lane; it < l * l; it += 32) Wd[dl.q(it) * ls + dl.r(it)] = (double)Qf[dl.q(it) * ls + dl.r(it)];
    if (lane < l) gv[lane] = (double)Sf[lane * ls + lane];
    __syncwarp();
    newton_refine(Gs, Wd, gv, Z, rv, cv, l, nm, ls, is_minor[wid], fro, 1e-17, d.gram_fp32 ? 1 : kNewtonSteps);
  }

  if (d.debug_Z)
    for (int it = lane; it < l * nm; it += 32) d.debug_Z[t * l * nm + it] = Z[it];
  if (d.Zst)  // kept for the reweighting steps of the L1 form
    for (int it = lane; it < l * nm; it += 32) d.Zst[t * l * nm + it] = Z[it];

  // scatter Z Z^T into M[C_t, C_t] in fixed point
  const int f = macc_frac_bits(d.counters[2]);
  const double scale = ldexp(1.0, f);
  const int32_t* C = d.cols + t * l;
  for (int it = lane; it < l * l; it += 32) {
    const int a = dl.q(it), b = dl.r(it);
    double pr = 0.0;
    for (int j = 0; j < nm; ++j) pr = fma(Z[a * nm + j], Z[b * nm + j], pr);
    const long long v = llrint(pr * scale);
    if (v) atomicAdd(&d.macc[(uint32_t)C[a] * (uint32_t)d.n + (uint32_t)C[b]], (unsigned long long)v);
  }
}

__global__ void __launch_bounds__(32 * kMinorWarps) k_minor_scatter(const ProbDesc* __restrict__ descs,
                                                                   const int64_t* __restrict__ trial_off, int nprob,
                                                                   int lmax) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  const int64_t g = (int64_t)blockIdx.x * kMinorWarps + (threadIdx.x >> 5);
  if (g >= trial_off[nprob]) return;
  minor_trial(descs, trial_off, nprob, lmax, g, false, smraw);
}

// The trials k_minor_half handed over (l > 16): one warp per listed trial,
// grid-stride.
__global__ void __launch_bounds__(32 * kMinorWarps) k_minor_listed(const ProbDesc* __restrict__ descs,
                                                                  const int64_t* __restrict__ trial_off, int nprob,
                                                                  int lmax, const unsigned long long* __restrict__ list,
                                                                  const unsigned long long* __restrict__ list_count) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  const unsigned long long count = *list_count;
  for (unsigned long long k = (unsigned long long)blockIdx.x * kMinorWarps + (threadIdx.x >> 5); k < count;
       k += (unsigned long long)gridDim.x * kMinorWarps)
    minor_trial(descs, trial_off, nprob, lmax, (int64_t)list[k], true, smraw);
}

// a5 + a6 with two trials per warp: each half warp takes one trial with
// l <= 16, its Gram's rows in the registers of its lanes (lane i < l: row i).
// FP32 Jacobi in registers (small_df.cuh, circle ordering on KP = l rounded up
// to even, so a trial's rotations depend on its own l only and its result is
// the same in any batch), the n_minor smallest eigenvalues, then the same FP64
// block-Newton refinement and fixed-point scatter as minor_trial with 16 lanes.
// A trial whose split is nearly degenerate (a complement eigenvalue within
// split_tol ||G|| of a minor one) refines that cluster as a block and splits it
// by a small FP64 Rayleigh-Ritz step, in the same half warp; a trial with
// l > 16 is appended to `list` for k_minor_listed.
// Cyclic Jacobi of the small symmetric FP64 matrix C (nc x nc, row stride
// ls) by one thread (nc is the size of a nearly degenerate cluster, usually 2):
// eigenvalues on C's diagonal, eigenvectors into V (columns).
__device__ inline void serial_jacobi64(double* C, double* V, int nc, int ls) {
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) V[i * ls + j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 16; ++sweep) {
    bool any = false;
    for (int p = 0; p < nc; ++p)
      for (int q = p + 1; q < nc; ++q) {
        const double apq = C[p * ls + q], app = C[p * ls + p], aqq = C[q * ls + q];
        if (apq == 0.0 || fabs(apq) <= 1e-17 * (fabs(app) + fabs(aqq))) continue;
        any = true;
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < nc; ++k) {  // columns p, q
          const double x = C[k * ls + p], y = C[k * ls + q];
          C[k * ls + p] = c * x - s * y;
          C[k * ls + q] = s * x + c * y;
          const double vx = V[k * ls + p], vy = V[k * ls + q];
          V[k * ls + p] = c * vx - s * vy;
          V[k * ls + q] = s * vx + c * vy;
        }
        for (int k = 0; k < nc; ++k) {  // rows p, q
          const double x = C[p * ls + k], y = C[q * ls + k];
          C[p * ls + k] = c * x - s * y;
          C[q * ls + k] = s * x + c * y;
        }
        C[p * ls + q] = C[q * ls + p] = 0.0;
      }
    if (!any) break;
  }
}

template <int KP>
__device__ __forceinline__ void minor_half_body(const ProbDesc& d, int64_t t, int64_t g, int ls, unsigned char* base,
                                                int* pick, int* is_minor, unsigned long long* __restrict__ list,
                                                unsigned long long* __restrict__ list_count) {
  const int wl = threadIdx.x & 31, hl = wl & 15;
  const unsigned hmask = 0xffffu << (wl & 16);
  const int l = d.l, nm = d.n_minor;
  const int lsz = ls - 1;  // the slot's matrices are lsz x lsz with row stride ls
  double* Gs = reinterpret_cast<double*>(base);
  float* Sf = reinterpret_cast<float*>(Gs + (size_t)lsz * ls);  // eigenvalues on the diagonal
  float* Qf = Sf + (size_t)lsz * ls;
  double* Z = reinterpret_cast<double*>(Qf + (size_t)lsz * ls);
  double* Wd = Z + (size_t)lsz * ls;
  double* gv = Wd + (size_t)lsz * ls;
  double* rv = gv + ls;
  double* cv = rv + ls;
  const int P = l * (l + 1) / 2;
  const double* G = d.gram + t * P;
  for (int q = hl; q < P; q += 16) {
    int a = 0, rem = q;
    while (rem >= l - a) {
      rem -= l - a;
      ++a;
    }
    const int b = a + rem;
    const double v = G[q];
    Gs[a * ls + b] = v;
    Gs[b * ls + a] = v;
  }
  __syncwarp(hmask);
  float a[KP], v[KP];
  float f = 0.f;
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    a[j] = (hl < l && j < l) ? (float)Gs[hl * ls + j] : 0.f;
    v[j] = (j == hl) ? 1.f : 0.f;
    f += a[j] * a[j];
  }
#pragma unroll
  for (int o = 8; o; o >>= 1) f += __shfl_xor_sync(hmask, f, o);
  const float fro = sqrtf(f);
  reg_jacobi<KP, 16>(a, v, 4.f * FLT_EPSILON * fro, 40);
  const float lam = reg_pick<KP>(a, hl);
  if (hl < l) {
    Sf[hl * ls + hl] = lam;
#pragma unroll
    for (int j = 0; j < KP; ++j)
      if (j < l) Qf[hl * ls + j] = v[j];
  }
  __syncwarp(hmask);
  // the n_minor smallest eigenvalues (ties broken by index)
  const SmallDiv dnm((uint32_t)nm), dl((uint32_t)l);  // quotients by nm and l without integer division
  if (hl == 0) {
    for (int i = 0; i < l; ++i) is_minor[i] = 0;
    for (int j = 0; j < nm; ++j) {
      int best = -1;
      for (int i = 0; i < l; ++i)
        if (!is_minor[i] && (best < 0 || Sf[i * ls + i] < Sf[best * ls + best])) best = i;
      is_minor[best] = 1;
      pick[j] = best;
    }
  }
  __syncwarp(hmask);
  float gap_min = 3.0e38f;
  if (hl < l && !is_minor[hl])
    for (int j = 0; j < nm; ++j) gap_min = fminf(gap_min, fabsf(lam - Sf[pick[j] * ls + pick[j]]));
#pragma unroll
  for (int o = 8; o; o >>= 1) gap_min = fminf(gap_min, __shfl_xor_sync(hmask, gap_min, o));
  if (gap_min < split_tol(d) * fro) {
    // Nearly degenerate across the split: the cluster of the minor eigenvectors
    // and the complement ones within split_tol ||G|| of them is refined as one
    // block by the FP64 Newton steps (its gaps to the rest are wide), then a
    // Rayleigh-Ritz step inside it (FP64, nc x nc) gives the n_minor vectors.
    const float tol = split_tol(d) * fro;
    if (hl == 0) {  // the cluster: is_minor marks it, pick lists it
      int nc = 0;
      for (int i = 0; i < l; ++i) {
        bool in = is_minor[i] != 0;
        for (int j = 0; j < nm && !in; ++j) in = fabsf(Sf[i * ls + i] - Sf[pick[j] * ls + pick[j]]) < tol;
        is_minor[i] = in ? 1 : 0;
      }
      for (int i = 0; i < l; ++i)
        if (is_minor[i]) pick[nc++] = i;
      gv[ls - 1] = (double)nc;  // (the last entry of ev is beyond l)
    }
    __syncwarp(hmask);
    const int nc = (int)gv[ls - 1];
    const SmallDiv dnc((uint32_t)nc);
    for (int it = hl; it < l * nc; it += 16) {
      const int aa = dnc.q(it), j = dnc.r(it);
      Z[aa * nc + j] = (double)Qf[aa * ls + pick[j]];
    }
    for (int it = hl; it < l * l; it += 16) Wd[dl.q(it) * ls + dl.r(it)] = (double)Qf[dl.q(it) * ls + dl.r(it)];
    if (hl < l) gv[hl] = (double)lam;
    __syncwarp(hmask);
    newton_refine<16>(Gs, Wd, gv, Z, rv, cv, l, nc, ls, is_minor, (double)fro, 1e-17, kNewtonSteps);
    // Rayleigh-Ritz inside the cluster: T = G Z (l x nc, into Wd), C = Z^T T (into the space of Sf and Qf)
    double* T = Wd;
    double* Cm = reinterpret_cast<double*>(Sf);  // Sf and Qf are no longer needed: lsz x ls doubles
    double* Vc = Wd;                             // after C is formed, T's space
    for (int it = hl; it < l * nc; it += 16) {
      const int aa = dnc.q(it), j = dnc.r(it);
      double acc = 0.0;
      for (int b = 0; b < l; ++b) acc = fma(Gs[aa * ls + b], Z[b * nc + j], acc);
      T[aa * nc + j] = acc;
    }
    __syncwarp(hmask);
    for (int it = hl; it < nc * nc; it += 16) {
      const int i = dnc.q(it), j = dnc.r(it);
      double acc = 0.0;
      for (int b = 0; b < l; ++b) acc = fma(Z[b * nc + i], T[b * nc + j], acc);
      Cm[i * ls + j] = acc;
    }
    __syncwarp(hmask);
    if (hl == 0) {
      for (int i = 0; i < nc; ++i)  // symmetrise
        for (int j = i + 1; j < nc; ++j) Cm[i * ls + j] = Cm[j * ls + i] = 0.5 * (Cm[i * ls + j] + Cm[j * ls + i]);
      serial_jacobi64(Cm, Vc, nc, ls);
      for (int i = 0; i < nc; ++i) is_minor[i] = 0;  // now: which cluster vectors are minor
      for (int j = 0; j < nm; ++j) {
        int best = -1;
        for (int i = 0; i < nc; ++i)
          if (!is_minor[i] && (best < 0 || Cm[i * ls + i] < Cm[best * ls + best])) best = i;
        is_minor[best] = 1;
        pick[j] = best;
      }
    }
    __syncwarp(hmask);
    for (int it = hl; it < l * nm; it += 16) {  // Z (l x n_minor) = Z_cluster Vc[:, picked], into C's space
      const int aa = dnm.q(it), j = dnm.r(it);
      double acc = 0.0;
      for (int c = 0; c < nc; ++c) acc = fma(Z[aa * nc + c], Vc[c * ls + pick[j]], acc);
      Cm[aa * nm + j] = acc;
    }
    __syncwarp(hmask);
    for (int it = hl; it < l * nm; it += 16) Z[it] = Cm[it];
    __syncwarp(hmask);
  } else {
    for (int it = hl; it < l * nm; it += 16) {
      const int aa = dnm.q(it), j = dnm.r(it);
      Z[aa * nm + j] = (double)Qf[aa * ls + pick[j]];
    }
    for (int it = hl; it < l * l; it += 16) Wd[dl.q(it) * ls + dl.r(it)] = (double)Qf[dl.q(it) * ls + dl.r(it)];
    if (hl < l) gv[hl] = (double)lam;
    __syncwarp(hmask);
    newton_refine<16>(Gs, Wd, gv, Z, rv, cv, l, nm, ls, is_minor, (double)fro, 1e-17, d.gram_fp32 ? 1 : kNewtonSteps);
  }
  if (d.debug_Z)
    for (int it = hl; it < l * nm; it += 16) d.debug_Z[t * l * nm + it] = Z[it];
  if (d.Zst)
    for (int it = hl; it < l * nm; it += 16) d.Zst[t * l * nm + it] = Z[it];
  const int fb = macc_frac_bits(d.counters[2]);
  const double scale = ldexp(1.0, fb);
  const int32_t* C = d.cols + t * l;
  for (int it = hl; it < l * l; it += 16) {
    const int aa = dl.q(it), b = dl.r(it);
    double pr = 0.0;
    for (int j = 0; j < nm; ++j) pr = fma(Z[aa * nm + j], Z[b * nm + j], pr);
    const long long val = llrint(pr * scale);
    if (val) atomicAdd(&d.macc[(uint32_t)C[aa] * (uint32_t)d.n + (uint32_t)C[b]], (unsigned long long)val);
  }
}

constexpr int kHalfMaxL = 16;  // largest l of the two-per-warp kernel

// Eight CTAs per SM (64 registers): the kernel is issue-bound, and the warps
// of the extra CTAs hide more of each other's latency than the few spilled
// registers cost (0.31 -> 0.27 ms at 20000 trials of l = 9, against six CTAs
// at 80 registers).
__global__ void __launch_bounds__(32 * kMinorWarps, 8) k_minor_half(const ProbDesc* __restrict__ descs,
                                                                   const int64_t* __restrict__ trial_off, int nprob,
                                                                   int ls, unsigned long long* __restrict__ list,
                                                                   unsigned long long* __restrict__ list_count) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int pick[2 * kMinorWarps][kHalfMaxL];
  __shared__ int is_minor[2 * kMinorWarps][kHalfMaxL];
  const int wl = threadIdx.x & 31, hl = wl & 15, slot = threadIdx.x >> 4;
  const int64_t g = (int64_t)blockIdx.x * 2 * kMinorWarps + slot;
  if (g >= trial_off[nprob]) return;  // the half's lanes leave together
  const int p = find_problem(trial_off, nprob, g);
  const ProbDesc& d = descs[p];
  if (d.variant == 2) return;  // the row variant has its own kernels (k_rows.cu)
  const int64_t t = g - trial_off[p];
  const int l = d.l, nm = d.n_minor;
  const int count = d.row_counts[t];
  if (count < l) {  // rejected trial (fewer than l rows, i.e. not more than r)
    if (d.debug_Z)
      for (int i = hl; i < l * nm; i += 16) d.debug_Z[t * l * nm + i] = 0.0;
    if (d.Zst)
      for (int i = hl; i < l * nm; i += 16) d.Zst[t * l * nm + i] = 0.0;
    return;
  }
  if (hl == 0) atomicAdd(&d.counters[0], 1ull);
  if (l > kHalfMaxL) {  // one warp per trial
    if (hl == 0) list[atomicAdd(list_count, 1ull)] = (unsigned long long)g;
    return;
  }
  unsigned char* base = smraw + (size_t)slot * minor_smem_per_warp(ls - 1);
  int* pk = pick[slot];
  int* im = is_minor[slot];
  switch (l <= 4 ? 4 : (l + 1) & ~1) {
    case 4: minor_half_body<4>(d, t, g, ls, base, pk, im, list, list_count); break;
    case 6: minor_half_body<6>(d, t, g, ls, base, pk, im, list, list_count); break;
    case 8: minor_half_body<8>(d, t, g, ls, base, pk, im, list, list_count); break;
    case 10: minor_half_body<10>(d, t, g, ls, base, pk, im, list, list_count); break;
    case 12: minor_half_body<12>(d, t, g, ls, base, pk, im, list, list_count); break;
    case 14: minor_half_body<14>(d, t, g, ls, base, pk, im, list, list_count); break;
    default: minor_half_body<16>(d, t, g, ls, base, pk, im, list, list_count); break;
  }
}

// M = macc * 2^-f (two's-complement words read as signed).  Grid over all
// entries of all problems.
__global__ void __launch_bounds__(256) k_finalize_M(const ProbDesc* __restrict__ descs,
                                                  const int64_t* __restrict__ ent_off, int nprob) {
  pdl_enter();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ent_off[nprob]) return;
  const int p = find_problem(ent_off, nprob, g);
  const ProbDesc& d = descs[p];
  const int64_t e = g - ent_off[p];
  const int f = macc_frac_bits(d.counters[2]);
  const double v = ldexp((double)(long long)d.macc[e], -f);
  d.M[e] = v;
  if (d.debug_M) d.debug_M[e] = v;
}

cudaError_t launch_minor_scatter(const ProbDesc* descs, const int64_t* trial_off, int nprob, int64_t total, int lmax,
                                 unsigned long long* list, unsigned long long* list_count, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  if (list && list_count) {
    // two trials per warp (l <= 16), then the handed-over trials one per warp
    const int lh = std::min(lmax, kHalfMaxL);
    const size_t dynh = 2 * kMinorWarps * minor_smem_per_warp(lh) + 16;
    cudaError_t e = cudaFuncSetAttribute(k_minor_half, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynh);
    if (e != cudaSuccess) return e;
    (void)launch_chained(k_minor_half, (unsigned)((total + 2 * kMinorWarps - 1) / (2 * kMinorWarps)), 32 * kMinorWarps,
                         dynh, s, descs, trial_off, nprob, lh + 1, list, list_count);
    ++g_kernel_launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t dyn = kMinorWarps * minor_smem_per_warp(lmax) + 16;
    if ((e = cudaFuncSetAttribute(k_minor_listed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)) !=
        cudaSuccess)
      return e;
    // grid-stride over the list with enough CTAs to fill the GPU when every trial is listed
    const int64_t grid = std::min<int64_t>((total + kMinorWarps - 1) / kMinorWarps, 1024);
    (void)launch_chained(k_minor_listed, (unsigned)grid, 32 * kMinorWarps, dyn, s, descs, trial_off, nprob, lmax, list,
                         list_count);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  const size_t dyn = kMinorWarps * minor_smem_per_warp(lmax) + 16;
  cudaError_t e = cudaFuncSetAttribute(k_minor_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  (void)launch_chained(k_minor_scatter, (unsigned)((total + kMinorWarps - 1) / kMinorWarps), 32 * kMinorWarps, dyn, s,
                       descs, trial_off, nprob, lmax);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_finalize_M(const ProbDesc* descs, const int64_t* ent_off, int nprob, int64_t total, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  (void)launch_chained(k_finalize_M, (unsigned)((total + 255) / 256), 256, 0, s, descs, ent_off, nprob);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace rsm
