// Trial-count planner (Section III, Lemma 1 and Theorem 3): how many submatrix
// draws make every known entry of Y visited with probability at least epsilon,
// assuming the known entries are spread homogeneously with density rho.
//
// A trial visits a given known entry with probability P (the first line of the
// proof of Theorem 3): the submatrix has i rows (M1: i ~ Bin(m, rho^l), l
// columns) or i columns (M2: i ~ Bin(n, rho^k), k rows); it is used when
// i >= l (M1) or i > r (M2) and then visits i l (or k i) of the m n rho known
// entries.  So, with X ~ Bin(N, p),
//   M1: P = l / (m n rho) E[X 1{X >= l}],   N = m, p = rho^l
//   M2: P = k / (m n rho) E[X 1{X > r}],    N = n, p = rho^k
// and E[X 1{X >= a}] = N p P(Bin(N - 1, p) >= a - 1).  I independent trials
// miss the entry with probability (1 - P)^I, so I = ln(1 / (1 - eps)) / P trials
// are needed (eq. I.bnd uses ln(1 - x) <= -x, so this is also the bound's form).
// Theorem 3 replaces P by a closed-form lower bound through Lemma 1's
// C_{N,p}(k) >= P(X < k); that bound is reported too (for M1 with the same
// steps: i >= l replaced by l, the tail P(X >= l) = 1 - P(X < l) by 1 - C_{m, rho^l}(l + 1)).
// Reading of Lemma 1: its bracket C(k) <= . <= C(k + 1) is of the printed sum
// over i = 0 .. k, P(X <= k); Theorem 3's P(X < r + 1) <= C(r + 2) holds either way.
#include <cmath>

#include "../../include/rsm.h"

namespace {

// P(Bin(N, p) <= K), summed in the log domain (K is small here: r or l).
double binom_cdf(int64_t N, double p, int64_t K) {
  if (K < 0) return 0.0;
  if (K >= N) return 1.0;
  if (p <= 0.0) return 1.0;
  if (p >= 1.0) return 0.0;
  const double lp = std::log(p), lq = std::log1p(-p), lnf = std::lgamma((double)N + 1.0);
  double s = 0.0;
  for (int64_t i = 0; i <= K; ++i)
    s += std::exp(lnf - std::lgamma((double)i + 1.0) - std::lgamma((double)(N - i) + 1.0) + i * lp + (N - i) * lq);
  return s < 1.0 ? s : 1.0;
}

// Lemma 1: C_{N,p}(k), with C(0) = (1 - p)^N, C(N) = 1 - p^N, 1 for k > N.
double lemma1_C(int64_t N, double p, int64_t k) {
  if (k <= 0) return std::pow(1.0 - p, (double)N);
  if (k == N) return 1.0 - std::pow(p, (double)N);
  if (k > N) return 1.0;
  const double x = (double)k / (double)N;
  const double phi = x * std::log(x / p) + (1.0 - x) * std::log((1.0 - x) / (1.0 - p));
  const double z = (x > p ? 1.0 : (x < p ? -1.0 : 0.0)) * std::sqrt(2.0 * (double)N * (phi > 0.0 ? phi : 0.0));
  return 0.5 * std::erfc(-z / std::sqrt(2.0));
}

}  // namespace

extern "C" int32_t rsm_plan_trials(int64_t m, int64_t n, double rho, int32_t r, int32_t size, int32_t variant,
                                   double epsilon, rsm_trial_plan* out) {
  if (!out || m < 1 || n < 1 || !(rho > 0.0 && rho <= 1.0) || r < 1 || size <= r || !(epsilon > 0.0 && epsilon < 1.0))
    return RSM_ERR_INVALID_ARG;
  if (variant == RSM_ROWS_RANDOM ? size > m : size > n) return RSM_ERR_INVALID_ARG;
  const double known = (double)m * (double)n * rho;
  const double need = std::log(1.0 / (1.0 - epsilon));
  double P, P_low;
  if (variant == RSM_ROWS_RANDOM) {  // M2: k = size rows, i ~ Bin(n, rho^k) columns, used when i > r
    const int64_t k = size;
    const double p = std::pow(rho, (double)k);
    P = (double)k * (double)n * p / known * (1.0 - binom_cdf(n - 1, p, r - 1));
    P_low = (double)k * (double)(r + 1) / known * (1.0 - lemma1_C(n, p, r + 2));
  } else {  // M1: l = size columns, i ~ Bin(m, rho^l) rows, used when i >= l
    const int64_t l = size;
    const double p = std::pow(rho, (double)l);
    P = (double)l * (double)m * p / known * (1.0 - binom_cdf(m - 1, p, l - 2));
    P_low = (double)l * (double)l / known * (1.0 - lemma1_C(m, p, l + 1));
  }
  out->p_visit = P;
  out->p_visit_theorem3 = P_low;
  out->trials = P > 0.0 ? need / P : INFINITY;
  out->trials_theorem3 = P_low > 0.0 ? need / P_low : INFINITY;
  return RSM_OK;
}
