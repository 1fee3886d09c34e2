// One-warp cyclic Jacobi eigensolver for a small symmetric matrix in shared
// memory (FP64).  Textbook two-sided Jacobi (symmetric Schur decomposition,
// Golub & Van Loan, "Matrix Computations", Sec. 8.5): a rotation in plane
// (p, q) with tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c annihilates a_pq.  The parallel
// round-robin ordering applies the k/2 disjoint rotations of a round together.
// A rotation is skipped when |a_pq| <= eps sqrt(|a_pp a_qq|); the sweeps stop
// when a whole sweep skips every rotation.
#pragma once

#include <cfloat>

namespace rsm {

struct JacobiScratch {
  int p[16], q[16];
  double c[16], s[16];
};

// S: k x k symmetric (row stride ls), overwritten by its eigenvalues on the
// diagonal; Vm: k x k (row stride ls) receives the eigenvectors as columns.
// k <= 32.  All 32 lanes of the warp must call it.
__device__ inline void warp_jacobi(double* S, double* Vm, int k, int ls, JacobiScratch& js, int max_sweeps = 40) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < k * k; i += 32) {
    const int a = i / k, b = i % k;
    Vm[a * ls + b] = (a == b) ? 1.0 : 0.0;
  }
  __syncwarp();
  const int ne = (k + 1) & ~1;
  const int np = ne / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    for (int round = 0; round < ne - 1; ++round) {
      if (lane < np) {
        const int s0 = lane, s1 = ne - 1 - lane;
        int a = (s0 == 0) ? 0 : ((s0 - 1 + round) % (ne - 1)) + 1;
        int b = (s1 == 0) ? 0 : ((s1 - 1 + round) % (ne - 1)) + 1;
        if (a > b) {
          const int tmp = a;
          a = b;
          b = tmp;
        }
        double c = 1.0, s = 0.0;
        if (b < k) {
          const double apq = S[a * ls + b];
          const double app = S[a * ls + a], aqq = S[b * ls + b];
          if (fabs(apq) > DBL_EPSILON * sqrt(fabs(app) * fabs(aqq)) && fabs(apq) > 1e-300) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        } else {
          b = a;
        }
        js.p[lane] = a;
        js.q[lane] = b;
        js.c[lane] = c;
        js.s[lane] = s;
      }
      __syncwarp();
      const bool rot = lane < np && js.s[lane] != 0.0;
      any |= __any_sync(0xffffffffu, rot);
      for (int it = lane; it < np * k; it += 32) {  // columns p, q of S and Vm
        const int r = it / k, i = it % k;
        const double s = js.s[r];
        if (s == 0.0) continue;
        const double c = js.c[r];
        const int a = js.p[r], b = js.q[r];
        const double xp = S[i * ls + a], xq = S[i * ls + b];
        S[i * ls + a] = c * xp - s * xq;
        S[i * ls + b] = s * xp + c * xq;
        const double vp = Vm[i * ls + a], vq = Vm[i * ls + b];
        Vm[i * ls + a] = c * vp - s * vq;
        Vm[i * ls + b] = s * vp + c * vq;
      }
      __syncwarp();
      for (int it = lane; it < np * k; it += 32) {  // rows p, q of S
        const int r = it / k, j = it % k;
        const double s = js.s[r];
        if (s == 0.0) continue;
        const double c = js.c[r];
        const int a = js.p[r], b = js.q[r];
        const double xp = S[a * ls + j], xq = S[b * ls + j];
        S[a * ls + j] = c * xp - s * xq;
        S[b * ls + j] = s * xp + c * xq;
      }
      __syncwarp();
      if (rot) {
        const int a = js.p[lane], b = js.q[lane];
        S[a * ls + b] = 0.0;
        S[b * ls + a] = 0.0;
      }
      __syncwarp();
    }
    if (!any) break;
  }
}

}  // namespace rsm
