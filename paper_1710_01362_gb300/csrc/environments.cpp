// Grouping of vibrational modes into environments (host, FP64): weighted k-means of the
// modes' normalised coupling patterns (Results, "Interface to TTNS": modes with similar
// patterns Wbar_n are grouped by k-means clustering with k-means++ seeding, and each group
// becomes one chain environment of Eq. 2).
//
// Pattern and strength of mode n: lambda_n = ||W_n||_F, Wbar_n = W_n / lambda_n; W and -W are one
// coupling direction, so the clustering is sign-invariant: a mode meets centre c aligned by
// s = sign(<x, c>) (+1 at zero), at the distance ||x||^2 + ||c||^2 - 2 |<x, c>|.  Features: Re
// and Im of Wbar_n (2 n_el^2 reals), weights lambda_n^2.  Lloyd iterations from the given
// initial centres (the caller's k-means++ draw): nearest centre (ties to the lower index),
// centres to the weighted means of their sign-aligned modes (an empty cluster keeps its
// centre), until no assignment changes.  Environment i: Wbar_i = centre_i / ||centre_i||_F,
// and mode n of it couples with lambda_n = Re <Wbar_i, W_n>_F.
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "../../include/ttns.h"

namespace ttns {
void set_last_error(const std::string& msg);
}

extern "C" ttns_status ttns_cluster_modes(int n_modes, int n_el, const double* W, int k, const int* init, int max_iter,
                                          int* assign, double* W_bar, double* lambda, int* iterations) {
  using cplx = std::complex<double>;
  if (n_modes < 1 || n_el < 1 || n_el > 64 || k < 1 || k > n_modes || max_iter < 1 || !W || !init || !assign ||
      !W_bar || !lambda) {
    ttns::set_last_error("ttns_cluster_modes: bad arguments");
    return TTNS_E_INVALID;
  }
  for (int c = 0; c < k; ++c)
    if (init[c] < 0 || init[c] >= n_modes) {
      ttns::set_last_error("ttns_cluster_modes: initial centre index out of range");
      return TTNS_E_INVALID;
    }
  const int m2 = n_el * n_el, F = 2 * m2;
  std::vector<double> X((size_t)n_modes * F), w(n_modes);
  for (int n = 0; n < n_modes; ++n) {
    const double* Wn = W + (size_t)2 * m2 * n;
    double ss = 0.0;
    for (int q = 0; q < m2; ++q) ss += Wn[2 * q] * Wn[2 * q] + Wn[2 * q + 1] * Wn[2 * q + 1];
    const double lam = std::sqrt(ss);
    w[n] = ss;
    for (int q = 0; q < m2; ++q) {
      X[(size_t)n * F + q] = lam > 0.0 ? Wn[2 * q] / lam : 0.0;
      X[(size_t)n * F + m2 + q] = lam > 0.0 ? Wn[2 * q + 1] / lam : 0.0;
    }
  }
  std::vector<double> C((size_t)k * F);
  for (int c = 0; c < k; ++c)
    for (int f = 0; f < F; ++f) C[(size_t)c * F + f] = X[(size_t)init[c] * F + f];
  std::vector<int> a(n_modes, -1);
  std::vector<double> sg(n_modes, 1.0), xx(n_modes, 0.0);
  for (int n = 0; n < n_modes; ++n)
    for (int f = 0; f < F; ++f) xx[n] += X[(size_t)n * F + f] * X[(size_t)n * F + f];
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    bool changed = false;
    std::vector<double> cc(k, 0.0);
    for (int c = 0; c < k; ++c)
      for (int f = 0; f < F; ++f) cc[c] += C[(size_t)c * F + f] * C[(size_t)c * F + f];
    for (int n = 0; n < n_modes; ++n) {
      int best = 0;
      double bd = 0.0, bdot = 0.0;
      for (int c = 0; c < k; ++c) {
        double dot = 0.0;
        for (int f = 0; f < F; ++f) dot += X[(size_t)n * F + f] * C[(size_t)c * F + f];
        const double d = xx[n] + cc[c] - 2.0 * std::fabs(dot);
        if (c == 0 || d < bd) { bd = d; best = c; bdot = dot; }
      }
      if (best != a[n]) changed = true;
      a[n] = best;
      sg[n] = bdot >= 0.0 ? 1.0 : -1.0;
    }
    for (int c = 0; c < k; ++c) {
      double ws = 0.0;
      std::vector<double> acc(F, 0.0);
      for (int n = 0; n < n_modes; ++n)
        if (a[n] == c) {
          ws += w[n];
          for (int f = 0; f < F; ++f) acc[f] += w[n] * sg[n] * X[(size_t)n * F + f];
        }
      if (ws > 0.0)
        for (int f = 0; f < F; ++f) C[(size_t)c * F + f] = acc[f] / ws;
    }
    if (!changed) break;
  }
  if (it > max_iter) it = max_iter;
  for (int c = 0; c < k; ++c) {
    double ss = 0.0;
    for (int f = 0; f < F; ++f) ss += C[(size_t)c * F + f] * C[(size_t)c * F + f];
    const double nrm = std::sqrt(ss);
    for (int q = 0; q < m2; ++q) {
      W_bar[(size_t)2 * m2 * c + 2 * q] = nrm > 0.0 ? C[(size_t)c * F + q] / nrm : C[(size_t)c * F + q];
      W_bar[(size_t)2 * m2 * c + 2 * q + 1] = nrm > 0.0 ? C[(size_t)c * F + m2 + q] / nrm : C[(size_t)c * F + m2 + q];
    }
  }
  for (int n = 0; n < n_modes; ++n) {
    assign[n] = a[n];
    const double* Wn = W + (size_t)2 * m2 * n;
    const double* B = W_bar + (size_t)2 * m2 * a[n];
    double re = 0.0;
    for (int q = 0; q < m2; ++q) re += B[2 * q] * Wn[2 * q] + B[2 * q + 1] * Wn[2 * q + 1];  // Re(conj(B) W)
    lambda[n] = re;
  }
  if (iterations) *iterations = it;
  return TTNS_OK;
}
