// Fermi-Dirac occupations of the Ritz states (host code, no device work).
//
// f_nk = 1 / (1 + exp((eps_nk - mu) / kT)), one electron per two-component
// spinor state; mu is the root of N(mu) = sum_k w_k sum_n f_nk = N_e (the
// electron-count constraint imposed through the Lagrange multiplier mu in
// Sec. II; Fermi-Dirac smearing as used throughout Sec. V).  N(mu) is
// continuous and strictly increasing, so mu is found by bisection on a bracket
// widened until it holds the root; the result is deterministic.
#include <cmath>
#include <vector>

#include "gbchfsi.h"

namespace {

double fermi(double x) {   // 1 / (1 + e^x) without overflow
  if (x > 0) {
    const double e = std::exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + std::exp(x));
}

double count(const double* eps, const std::vector<double>& w, int nk, int ns, double mu,
             double kT) {
  double n = 0.0;
  for (int k = 0; k < nk; ++k) {
    double nk_sum = 0.0;
    for (int i = 0; i < ns; ++i) nk_sum += fermi((eps[(size_t)k * ns + i] - mu) / kT);
    n += w[k] * nk_sum;
  }
  return n;
}

}  // namespace

extern "C" gbc_status gbc_fermi_occupations(const double* eps, const double* kweights, int nk,
                                            int nstates, double nelec, double kT, double* occ,
                                            double* mu_out) {
  if (!eps || !occ || nk < 1 || nstates < 1) return GBC_EINVAL;
  if (!(kT > 0.0) || !std::isfinite(kT) || !std::isfinite(nelec)) return GBC_EINVAL;
  std::vector<double> w(nk, 1.0 / nk);
  double wsum = 0.0;
  for (int k = 0; k < nk; ++k) {
    if (kweights) w[k] = kweights[k];
    if (!(w[k] >= 0.0) || !std::isfinite(w[k])) return GBC_EINVAL;
    wsum += w[k];
  }
  if (!(nelec > 0.0) || !(nelec < wsum * nstates)) return GBC_EINVAL;
  double emin = eps[0], emax = eps[0];
  for (size_t i = 0; i < (size_t)nk * nstates; ++i) {
    if (!std::isfinite(eps[i])) return GBC_EINVAL;
    emin = std::fmin(emin, eps[i]);
    emax = std::fmax(emax, eps[i]);
  }
  double lo = emin - 60.0 * kT, hi = emax + 60.0 * kT;
  int widen = 0;
  while (count(eps, w, nk, nstates, lo, kT) > nelec || count(eps, w, nk, nstates, hi, kT) < nelec) {
    if (++widen > 200) return GBC_ETIMEOUT;
    lo -= 60.0 * kT;
    hi += 60.0 * kT;
  }
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;   // adjacent doubles
    if (count(eps, w, nk, nstates, mid, kT) < nelec)
      lo = mid;
    else
      hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  for (size_t i = 0; i < (size_t)nk * nstates; ++i) occ[i] = fermi((eps[i] - mu) / kT);
  if (mu_out) *mu_out = mu;
  return GBC_OK;
}
