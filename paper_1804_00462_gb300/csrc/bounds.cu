// Bounds of Sec. IV on the SOR-SVD approximation A_hat (rank k, l = k + p,
// q power iterations), evaluated on the host for a given spectrum:
//
//   Theorem 4 (deterministic lower bound, with the power method):
//     sigma_j(.) >= sigma_j / sqrt(1 + x (sigma_{k+1} / sigma_j)^{4q+4}),
//     x = (||Omega2||_2 ||Omega1^+||_2)^2, j = 1..k;
//   Theorem 5 (deterministic error bound, 2- and F-norm):
//     ||A - A_hat|| <= e_k + sqrt(alpha^2 x / (1 + beta^2 x))
//                          + sqrt(eta^2 x / (1 + tau^2 x)),
//     g = (sigma_{k+1}/sigma_k)^{2q}, alpha = sqrt(k) sigma_{k+1}^2/sigma_k g,
//     beta = sigma_{k+1}^2 / (sigma_1 sigma_k) g, eta = (sigma_k/sigma_{k+1})
//     alpha, tau = (sigma_k/sigma_{k+1}) beta; e_k = sigma_{k+1} (2-norm) or
//     sqrt(sum_{j>k} sigma_j^2) (F-norm);
//   Theorem 6 (lower bound on the expected singular values):
//     E sigma_j(.) >= sigma_j / sqrt(1 + nu^2 (sigma_{k+1}/sigma_j)^{4q+4});
//   Theorem 7 (upper bound on the expected error):
//     E ||A - A_hat|| <= e_k + (1 + gamma) sqrt(k) nu sigma_{k+1} gamma^{2q},
//     gamma = sigma_{k+1} / sigma_k,
//   with nu = (sqrt(n - l + p) + sqrt(l) + 7) (4 e sqrt(l) / (p + 1)).
//
// Omega1 = V1^T Omega and Omega2 = V2^T Omega split the test matrix along the
// first k right singular vectors and the rest (with the oversampling p of
// l = k + p as the analysis parameter, so sigma_{l-p+1} = sigma_{k+1}).
// Readings: Theorem 5's tau for q > 0 is (sigma_k / sigma_{k+1}) beta (the
// form that reduces to the q = 0 value and is dimensionless), and Theorem
// 4's deterministic bound holds for sigma_j(A Q2 Q2^T), which is what its
// proof establishes.
#include "../../include/sorsvd.h"

#include <math.h>

namespace {

constexpr double kE = 2.718281828459045;

double nu_of(int64_t n, int k, int p) {
  const int l = k + p;
  const double nu1 = sqrt((double)(n - l + p)) + sqrt((double)l) + 7.0;
  const double nu2 = 4.0 * kE * sqrt((double)l) / (double)(p + 1);
  return nu1 * nu2;
}

}  // namespace

extern "C" int sorsvd_bounds(const double* sigma, int r, int64_t n, int k, int p, int q, double omega2_norm,
                             double omega1_pinv_norm, sorsvd_bounds_out* out, double* thm4_lower,
                             double* thm6_lower) {
  if (!sigma || !out || k < 1 || p < 0 || q < 0 || r < k + 1 || n < (int64_t)(k + p)) return SORSVD_ERR_ARG;
  for (int j = 0; j < r; ++j)
    if (!(sigma[j] >= 0.0) || (j > 0 && sigma[j] > sigma[j - 1])) return SORSVD_ERR_ARG;
  if (!(sigma[k - 1] > 0.0)) return SORSVD_ERR_ARG;
  const double s1 = sigma[0], sk = sigma[k - 1], sl = sigma[k];
  double tail2 = 0.0;
  for (int j = k; j < r; ++j) tail2 += sigma[j] * sigma[j];
  out->ey_2 = sl;
  out->ey_fro = sqrt(tail2);
  // Theorems 6 and 7 (expected case): the spectrum alone
  const double nu = nu_of(n, k, p);
  const double gam = sl / sk;
  const double extra7 = (1.0 + gam) * sqrt((double)k) * nu * sl * pow(gam, 2.0 * q);
  out->thm7_upper_2 = out->ey_2 + extra7;
  out->thm7_upper_fro = out->ey_fro + extra7;
  if (thm6_lower)
    for (int j = 0; j < k; ++j)
      thm6_lower[j] = sigma[j] / sqrt(1.0 + nu * nu * pow(sl / sigma[j], 4.0 * q + 4.0));
  // Theorems 4 and 5 (deterministic): need ||Omega2||_2 and ||Omega1^+||_2
  const bool det = omega2_norm >= 0.0 && omega1_pinv_norm >= 0.0;
  if (!det) {
    out->thm5_upper_2 = NAN;
    out->thm5_upper_fro = NAN;
    if (thm4_lower)
      for (int j = 0; j < k; ++j) thm4_lower[j] = NAN;
    return SORSVD_OK;
  }
  const double x = (omega2_norm * omega1_pinv_norm) * (omega2_norm * omega1_pinv_norm);
  const double g = pow(sl / sk, 2.0 * q);
  const double alpha = sqrt((double)k) * sl * sl / sk * g;
  const double beta = sl * sl / (s1 * sk) * g;
  // eta = (sigma_k / sigma_{k+1}) alpha and tau = (sigma_k / sigma_{k+1}) beta,
  // written without the division (sigma_{k+1} may be 0)
  const double eta = sqrt((double)k) * sl * g;
  const double tau = sl / s1 * g;
  const double extra5 = sqrt(alpha * alpha * x / (1.0 + beta * beta * x)) + sqrt(eta * eta * x / (1.0 + tau * tau * x));
  out->thm5_upper_2 = out->ey_2 + extra5;
  out->thm5_upper_fro = out->ey_fro + extra5;
  if (thm4_lower)
    for (int j = 0; j < k; ++j) thm4_lower[j] = sigma[j] / sqrt(1.0 + x * pow(sl / sigma[j], 4.0 * q + 4.0));
  return SORSVD_OK;
}
