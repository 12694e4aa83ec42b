// Host-side setup of the helical-wave basis: Bessel zeros, the Gauss-Jacobi(0,1) radial rule,
// the radial tables xi_{n,k}(r_p), the 1/r^2 tables of the nu != 0 terms, the kinetic-energy
// cutoff masks and the compact index maps.
//
// arXiv 2210.12252:
//   basis functions and normalisation c_{m,n,k}   eq. Phi_expanded_in_basis_set, Appendix B
//                                                   (eq. Basis_fun_derived)
//   lambda^0                                        eq. Laplacian_of_f_mnk
//   linear order of the coefficients                eq. wavefun_storage
//   grids and the 4x oversampling rule              Sec. "Wave function storage"
//   cutoff mask at each (eta, nu)                   eq. Energy_cutoff and the mask after it
//   Gauss-Jacobi radial nodes                       Sec. "Wave function storage"
//   1/r^2 tables I(n, k, k')                        eqs. ell_coeff, ell_mnk, I_nkk_prime
//
// The Gauss-Jacobi(0,1) nodes are found by Sturm-sequence bisection on the Jacobi matrix of the
// monic P_k^{(0,1)} and polished by Newton on the three-term recurrence; the weights are
// 4 / ((1 - x^2) P_n'(x)^2), the (alpha, beta) = (0, 1) case of the Gauss-Jacobi weight formula.
// Bessel J_p comes from the C++17 special-math library; zeros are bracketed by a scan for sign
// changes, bisected and polished by Newton with J_p' = (J_{p-1} - J_{p+1}) / 2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <string>

#include "hw_internal.h"

namespace hw {
namespace {

double besselj(int p, double x) {
  if (p < 0) {  // J_{-p} = (-1)^p J_p
    double v = std::cyl_bessel_j(double(-p), x);
    return ((-p) & 1) ? -v : v;
  }
  return std::cyl_bessel_j(double(p), x);
}

std::vector<double> bessel_zeros(int p, int K) {
  std::vector<double> z;
  z.reserve(K);
  const double h = 0.05;
  double x = std::max(double(p), 0.5);
  double fx = besselj(p, x);
  while ((int)z.size() < K) {
    double y = x + h, fy = besselj(p, y);
    if (fx == 0.0) {
      z.push_back(x);
    } else if (fx * fy < 0.0) {
      double a = x, b = y, fa = fx;
      for (int it = 0; it < 200 && b - a > 1e-13 * std::max(1.0, std::fabs(a)); ++it) {
        double c = 0.5 * (a + b), fc = besselj(p, c);
        if (fa * fc <= 0.0) {
          b = c;
        } else {
          a = c;
          fa = fc;
        }
      }
      double r = 0.5 * (a + b);
      for (int it = 0; it < 3; ++it) {
        double d = 0.5 * (besselj(p - 1, r) - besselj(p + 1, r));
        r -= besselj(p, r) / d;
      }
      z.push_back(r);
    }
    x = y;
    fx = fy;
  }
  return z;
}

// P_n^{(0,1)}(x) and P_{n-1}^{(0,1)}(x) by the standard three-term recurrence
void jacobi01(int n, double x, double& pn, double& pn1) {
  const double a = 0.0, b = 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) {
    pn = p0;
    pn1 = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a + b;
    double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
    double a2 = (c - 1.0) * (a * a - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
    double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pn1 = p0;
}

// derivative from (2n+a+b)(1-x^2) P_n' = n[(a-b) - (2n+a+b)x] P_n + 2(n+a)(n+b) P_{n-1}
double jacobi01_deriv(int n, double x, double pn, double pn1) {
  const double a = 0.0, b = 1.0, c = 2.0 * n + a + b;
  return (n * ((a - b) - c * x) * pn + 2.0 * (n + a) * (n + b) * pn1) / (c * (1.0 - x * x));
}

// number of eigenvalues of the Jacobi matrix below x (Sturm sequence)
int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = d[i] - x - (i ? e2[i - 1] / q : 0.0);
    if (q == 0.0) q = 1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

void gauss_jacobi01(int n, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> d(n), e2(std::max(n - 1, 0));
  for (int k = 0; k < n; ++k) d[k] = 1.0 / ((2.0 * k + 1.0) * (2.0 * k + 3.0));
  for (int k = 1; k < n; ++k) e2[k - 1] = double(k) * (k + 1) / ((2.0 * k + 1) * (2.0 * k + 1));
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double lo = -1.0, hi = 1.0;  // the i-th eigenvalue (ascending) lies in (-1, 1)
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
      double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e2, mid) > i) hi = mid;
      else lo = mid;
    }
    double xi = 0.5 * (lo + hi);
    for (int it = 0; it < 2; ++it) {  // Newton polish on P_n
      double pn, pn1;
      jacobi01(n, xi, pn, pn1);
      double dp = jacobi01_deriv(n, xi, pn, pn1);
      double step = pn / dp;
      if (std::fabs(step) < 1e-12) xi -= step;
    }
    double pn, pn1;
    jacobi01(n, xi, pn, pn1);
    double dp = jacobi01_deriv(n, xi, pn, pn1);
    x[i] = xi;
    w[i] = 4.0 / ((1.0 - xi * xi) * dp * dp);
  }
}

bool only_factors_23(int n) {
  if (n < 1) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

}  // namespace

bool make_fft_plan(int n, FftPlan& plan) {
  if (!only_factors_23(n)) return false;
  plan = FftPlan();
  plan.n = n;
  int m = n;
  while (m % 4 == 0) { plan.rad[plan.nst++] = 4; m /= 4; }
  while (m % 3 == 0) { plan.rad[plan.nst++] = 3; m /= 3; }
  while (m % 2 == 0) { plan.rad[plan.nst++] = 2; m /= 2; }
  return m == 1 && plan.nst <= 16;
}

std::string build_host_basis(const hw_basis_params& p, int nk, const double* eta,
                             const double* nu, const double* ecut_per_k, HostBasis& hb) {
  char buf[256];
  if (!(p.R > 0) || !(p.tau > 0) || !std::isfinite(p.alpha) || p.ncyc < 1)
    return "need R > 0, tau > 0, finite alpha, ncyc >= 1";
  if (p.oversample < 2) return "oversample must be >= 2";
  if (p.Nr < p.oversample) return "Nr must be >= oversample";
  if (!only_factors_23(p.Nth1) || !only_factors_23(p.Nth2))
    return "Nth1 and Nth2 may only have the prime factors 2 and 3";
  if (nk < 1 || !eta) return "need nk >= 1 k-points";
  hb = HostBasis();
  hb.prm = p;
  hb.M = (p.Nth1 - 1) / p.oversample;
  hb.N = (p.Nth2 - 1) / p.oversample;
  hb.K = p.Nr / p.oversample;
  if (hb.K < 1) return "K = floor(Nr/oversample) must be >= 1";
  if (p.Nth1 < 2 * hb.M + 1 || p.Nth2 < 2 * hb.N + 1) return "angular grid below 2*max+1";
  const int M = hb.M, N = hb.N, K = hb.K, Nr = p.Nr;
  // radial rule
  std::vector<double> x, w;
  gauss_jacobi01(Nr, x, w);
  hb.r.resize(Nr);
  hb.wr.resize(Nr);
  for (int i = 0; i < Nr; ++i) {
    hb.r[i] = p.R * (1.0 + x[i]) / 2.0;
    hb.wr[i] = p.R * p.R / 4.0 * w[i];
  }
  // zeros and radial tables; xi_{-n} = xi_n (J_{-q} = (-1)^q J_q and, at a zero of J_q,
  // J_{q-1} = -J_{q+1})
  hb.zeros.assign(N + 1, {});
  hb.xi.assign(size_t(N + 1) * Nr * K, 0.0);
  hb.xid.assign(size_t(N + 1) * Nr * K, 0.0);
  const double pi = 3.14159265358979323846;
  for (int n = 0; n <= N; ++n) {
    const int ord = n * p.ncyc;
    hb.zeros[n] = bessel_zeros(ord, K);
    for (int k = 0; k < K; ++k) {
      const double b = hb.zeros[n][k];
      const double c = std::sqrt(p.ncyc / (pi * p.tau)) / (p.R * besselj(ord + 1, b));
      for (int q = 0; q < Nr; ++q) {
        const double x = b * hb.r[q] / p.R;
        hb.xi[(size_t(n) * Nr + q) * K + k] = c * besselj(ord, x);
        // radial derivative (Appendix C, eq. B_r): c (b/R) J_p'(x), J_p' = (J_{p-1} - J_{p+1}) / 2
        hb.xid[(size_t(n) * Nr + q) * K + k] = c * (b / p.R) * 0.5 * (besselj(ord - 1, x) - besselj(ord + 1, x));
      }
    }
  }
  // 1/r^2 matrix of each |n| group (eqs. ell_coeff, ell_mnk, I_nkk_prime):
  //   qtab[g][k'][k] = <F_{m,n,k'}, F_{m,n,k} / r^2> = (2/R^2) I(n, k, k'),
  //   I = int_0^1 J_p(b_k q) J_p(b_k' q) / q dq / (J_{p+1}(b_k) J_{p+1}(b_k')),  p = g Ncyc.
  // For p >= 1 the integrand J J / q^2 (times the weight q) is smooth; a Gauss-Jacobi(0,1)
  // rule with enough nodes for the band limit b_k + b_k' gives it to rounding.  For p = 0 the
  // integral diverges at r = 0 (the paper's nu != 0 formulas meet J_0); the value of the
  // transform's own radial rule (nodes avoid r = 0) is used instead.
  hb.qtab.assign(size_t(N + 1) * K * K, 0.0);
  {
    double bmax = 0.0;
    for (int n = 0; n <= N; ++n) bmax = std::max(bmax, hb.zeros[n][K - 1]);
    const int nq = 64 + 2 * (int)std::ceil(bmax);
    std::vector<double> xq, wq;
    gauss_jacobi01(nq, xq, wq);
    std::vector<double> Jq((size_t)nq * K);
    for (int n = 0; n <= N; ++n) {
      const int ord = n * p.ncyc;
      double* Q = hb.qtab.data() + (size_t)n * K * K;
      if (ord == 0) {
        const double pref = 2.0 * pi * p.tau / p.ncyc;
        for (int k = 0; k < K; ++k)
          for (int kk = 0; kk < K; ++kk) {
            double s = 0.0;
            for (int q = 0; q < Nr; ++q)
              s += hb.wr[q] / (hb.r[q] * hb.r[q]) * hb.xi[(size_t(n) * Nr + q) * K + k] *
                   hb.xi[(size_t(n) * Nr + q) * K + kk];
            Q[(size_t)kk * K + k] = pref * s;
          }
        continue;
      }
      for (int i = 0; i < nq; ++i) {
        const double q = 0.5 * (1.0 + xq[i]);
        for (int k = 0; k < K; ++k) Jq[(size_t)i * K + k] = besselj(ord, hb.zeros[n][k] * q) / q;
      }
      for (int k = 0; k < K; ++k)
        for (int kk = 0; kk <= k; ++kk) {
          double s = 0.0;   // int_0^1 (J J / q^2) q dq = sum_i (w_i / 4) J J / q_i^2
          for (int i = 0; i < nq; ++i) s += 0.25 * wq[i] * Jq[(size_t)i * K + k] * Jq[(size_t)i * K + kk];
          const double v = 2.0 / (p.R * p.R) * s /
                           (besselj(ord + 1, hb.zeros[n][k]) * besselj(ord + 1, hb.zeros[n][kk]));
          Q[(size_t)kk * K + k] = v;
          Q[(size_t)k * K + kk] = v;
        }
    }
  }
  // k-points, masks
  hb.nk = nk;
  hb.eta.assign(eta, eta + nk);
  hb.nu.assign(nk, 0.0);
  hb.ecut.assign(nk, p.ecut);
  for (int b = 0; b < nk; ++b) {
    if (nu) hb.nu[b] = nu[b];
    if (ecut_per_k) hb.ecut[b] = ecut_per_k[b];
    if (!std::isfinite(hb.nu[b])) return "nu must be finite";
    if (!std::isfinite(hb.eta[b])) return "eta must be finite";
  }
  const double kz = 2.0 * pi / p.tau;
  // kept radial count per (b, m, n): KE increases with k at fixed (m, n), so the kept modes of
  // a pair are a prefix k < Kmn
  const int nm = 2 * M + 1, nn = 2 * N + 1;
  std::vector<int> kmn(size_t(nk) * nm * nn, 0);
  for (int b = 0; b < nk; ++b) {
    const double ec = hb.ecut[b];
    for (int im = 0; im < nm; ++im)
      for (int in = 0; in < nn; ++in) {
        const int m = im - M, n = in - N;
        const double ax = m - hb.eta[b] - p.alpha * (n * p.ncyc - hb.nu[b]);
        int cnt = 0;
        for (int k = 0; k < K; ++k) {
          const double br = hb.zeros[std::abs(n)][k] / p.R;
          const double ke = 0.5 * (br * br + kz * kz * ax * ax);
          if (ec <= 0.0 || ke <= ec * (1.0 + 1e-12)) cnt = k + 1;
          else break;
        }
        kmn[(size_t(b) * nm + im) * nn + in] = cnt;
      }
  }
  // union of active pairs, grouped by |n|, then n, then m
  std::vector<std::pair<int, int>> pairs;  // (n, m)
  for (int g = 0; g <= N; ++g) {
    const int signs[2] = {-g, g};
    for (int si = 0; si < (g == 0 ? 1 : 2); ++si) {
      const int n = signs[si];
      for (int m = -M; m <= M; ++m) {
        bool any = false;
        for (int b = 0; b < nk && !any; ++b)
          any = kmn[(size_t(b) * nm + (m + M)) * nn + (n + N)] > 0;
        if (any) pairs.push_back({n, m});
      }
    }
  }
  hb.nA = (int)pairs.size();
  if (hb.nA == 0) return "the cutoff keeps no mode";
  hb.pair_m.resize(hb.nA);
  hb.pair_n.resize(hb.nA);
  hb.group_start.assign(N + 2, 0);
  std::vector<int> gcount(N + 1, 0);
  std::map<int, int> mset;
  for (int a = 0; a < hb.nA; ++a) {
    hb.pair_n[a] = pairs[a].first;
    hb.pair_m[a] = pairs[a].second;
    gcount[std::abs(pairs[a].first)]++;
    mset[pairs[a].second] = 0;
  }
  for (int g = 0; g <= N; ++g) hb.group_start[g + 1] = hb.group_start[g] + gcount[g];
  hb.mrow_m.clear();
  for (auto& kv : mset) {
    kv.second = (int)hb.mrow_m.size();
    hb.mrow_m.push_back(kv.first);
  }
  hb.pair_mrow.resize(hb.nA);
  for (int a = 0; a < hb.nA; ++a) hb.pair_mrow[a] = mset[hb.pair_m[a]];
  hb.slot_pair.assign(hb.mrow_m.size() * (size_t)p.Nth2, -1);
  for (int a = 0; a < hb.nA; ++a)
    hb.slot_pair[(size_t)hb.pair_mrow[a] * p.Nth2 + ((hb.pair_n[a] % p.Nth2) + p.Nth2) % p.Nth2] = a;
  // compact offsets (box order restricted to the mask), kinetic energies, index maps
  hb.off.assign(size_t(nk) * hb.nA, 0);
  hb.Ka.assign(size_t(nk) * hb.nA, 0);
  hb.L.assign(nk, 0);
  hb.ke.assign(nk, {});
  hb.mnk.assign(nk, {});
  std::vector<int> boxoff(size_t(nm) * nn);
  for (int b = 0; b < nk; ++b) {
    int64_t o = 0;
    for (int im = 0; im < nm; ++im)
      for (int in = 0; in < nn; ++in) {
        boxoff[size_t(im) * nn + in] = (int)o;
        o += kmn[(size_t(b) * nm + im) * nn + in];
      }
    hb.L[b] = o;
    if (o == 0) {
      std::snprintf(buf, sizeof buf, "the cutoff keeps no mode at k-point %d", b);
      return buf;
    }
    if (o > (int64_t(1) << 31) - 1) return "basis too large";
    for (int a = 0; a < hb.nA; ++a) {
      const int im = hb.pair_m[a] + M, in = hb.pair_n[a] + N;
      hb.off[size_t(b) * hb.nA + a] = boxoff[size_t(im) * nn + in];
      hb.Ka[size_t(b) * hb.nA + a] = kmn[(size_t(b) * nm + im) * nn + in];
    }
    hb.ke[b].resize(o);
    hb.mnk[b].resize(3 * o);
    int64_t i = 0;
    for (int im = 0; im < nm; ++im)
      for (int in = 0; in < nn; ++in) {
        const int m = im - M, n = in - N;
        const int cnt = kmn[(size_t(b) * nm + im) * nn + in];
        const double ax = m - hb.eta[b] - p.alpha * (n * p.ncyc - hb.nu[b]);
        for (int k = 0; k < cnt; ++k, ++i) {
          const double br = hb.zeros[std::abs(n)][k] / p.R;
          hb.ke[b][i] = 0.5 * (br * br + kz * kz * ax * ax);
          hb.mnk[b][3 * i] = m;
          hb.mnk[b][3 * i + 1] = n;
          hb.mnk[b][3 * i + 2] = k;
        }
      }
  }
  return "";
}

}  // namespace hw
