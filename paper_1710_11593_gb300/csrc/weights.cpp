// Host-side weights of the L1 Caputo schemes, cancellation-free.
//
// Sub-diffusion (0<g<1), Lemma 2 / Eq. 19, b = 1-g, mu = tau^-g / Gamma(2-g):
//   a_0 = mu,  a_j = mu * l_j,  l_j = G_j - G_{j-1} = (j+1)^b - 2 j^b + (j-1)^b   (j >= 1)
// Hyperbolic (1<g<2), Eq. 17, b = 2-g, c = tau^-g / Gamma(3-g):
//   a_0 = c,  a_1 = c (M_1 - 2 M_0) = c (2^b - 3),
//   a_j = c W_j,  W_j = M_{j-2} - 2 M_{j-1} + M_j = (j+1)^b - 3 j^b + 3 (j-1)^b - (j-2)^b  (j >= 2)
//
// l_j and W_j are second and third differences of x^b; evaluated directly they lose up
// to ~j^2 (resp. j^3) relative digits.  For j >= kSeriesFrom they are summed as Taylor
// series of the difference operator about the stencil centre (every term has one sign
// pattern and the series converges like (const/j)^2); below that the plain differences
// are taken in long double, where the loss is at most ~1e4 ulp of that format.
//
// Derivatives with respect to g (for the gamma-gradient of the adjoint) differentiate
// the same series term by term, plus d ln(scale)/dg = -ln(tau) + digamma(2-g) (resp. 3-g).
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace ftoep {

namespace {

constexpr int64_t kSeriesFrom = 12;

// Falling factorial (b)_m = b (b-1) ... (b-m+1) and its b-derivative, accumulated.
struct Falling {
  double p = 1.0;   // (b)_m
  double dp = 0.0;  // d/db (b)_m
  int m = 0;
  void step(double b) {  // m -> m+1
    dp = dp * (b - m) + p;
    p = p * (b - m);
    ++m;
  }
};

// Second difference f(j+1) - 2 f(j) + f(j-1) of f(x) = x^b by the series
//   sum_{k>=1} 2 f^{(2k)}(j) / (2k)!,   f^{(m)}(x) = (b)_m x^{b-m},
// and (if d != nullptr) its derivative with respect to b:
//   sum_k 2/(2k)! [ (b)_{2k}' + (b)_{2k} ln j ] j^{b-2k}.
double second_diff_series(double b, int64_t j, double* d) {
  const double x = (double)j;
  const double lx = std::log(x);
  const double inv2 = 1.0 / (x * x);
  Falling F;
  F.step(b);
  F.step(b);  // (b)_2
  double pw = std::pow(x, b - 2.0);  // x^{b-2k}
  double fact = 2.0;                 // (2k)!
  double sum = 0.0, dsum = 0.0;
  for (int k = 1; k < 40; ++k) {
    double term = 2.0 * F.p * pw / fact;
    double dterm = 2.0 * (F.dp + F.p * lx) * pw / fact;
    sum += term;
    dsum += dterm;
    if (std::fabs(term) <= 1e-18 * std::fabs(sum) && std::fabs(dterm) <= 1e-18 * std::fabs(dsum)) break;
    F.step(b);
    F.step(b);
    pw *= inv2;
    fact *= (double)(2 * k + 1) * (double)(2 * k + 2);
  }
  if (d) *d = dsum;
  return sum;
}

// Third difference f(c+3/2) - 3 f(c+1/2) + 3 f(c-1/2) - f(c-3/2), c = j - 1/2, by
//   sum_{m odd >= 3} 2 f^{(m)}(c)/m! [ (3/2)^m - 3 (1/2)^m ]
// and its b-derivative.
double third_diff_series(double b, int64_t j, double* d) {
  const double c = (double)j - 0.5;
  const double lc = std::log(c);
  const double inv2 = 1.0 / (c * c);
  Falling F;
  F.step(b);
  F.step(b);
  F.step(b);  // (b)_3
  double pw = std::pow(c, b - 3.0);
  double fact = 6.0;        // m!
  double p32 = 27.0 / 8.0;  // (3/2)^m
  double p12 = 1.0 / 8.0;   // (1/2)^m
  double sum = 0.0, dsum = 0.0;
  for (int m = 3; m < 80; m += 2) {
    double w = 2.0 * (p32 - 3.0 * p12) / fact;
    double term = w * F.p * pw;
    double dterm = w * (F.dp + F.p * lc) * pw;
    sum += term;
    dsum += dterm;
    if (std::fabs(term) <= 1e-18 * std::fabs(sum) && std::fabs(dterm) <= 1e-18 * std::fabs(dsum)) break;
    F.step(b);
    F.step(b);
    pw *= inv2;
    fact *= (double)(m + 1) * (double)(m + 2);
    p32 *= 2.25;
    p12 *= 0.25;
  }
  if (d) *d = dsum;
  return sum;
}

long double lpow(long double x, long double b) { return x <= 0.0L ? 0.0L : std::pow(x, b); }
long double lxlog(long double x, long double b) { return x <= 0.0L ? 0.0L : std::pow(x, b) * std::log(x); }

// Direct differences in long double (small j only).
double second_diff_direct(double b, int64_t j, double* d) {
  long double B = b, x = (long double)j;
  long double v = lpow(x + 1, B) - 2.0L * lpow(x, B) + lpow(x - 1, B);
  if (d) *d = (double)(lxlog(x + 1, B) - 2.0L * lxlog(x, B) + lxlog(x - 1, B));
  return (double)v;
}

double third_diff_direct(double b, int64_t j, double* d) {
  long double B = b, x = (long double)j;
  long double v = lpow(x + 1, B) - 3.0L * lpow(x, B) + 3.0L * lpow(x - 1, B) - lpow(x - 2, B);
  if (d) *d = (double)(lxlog(x + 1, B) - 3.0L * lxlog(x, B) + 3.0L * lxlog(x - 1, B) - lxlog(x - 2, B));
  return (double)v;
}

// First difference (j+1)^b - j^b = j^b * expm1(b * log1p(1/j)) (j >= 1), and 1 for j = 0.
double first_diff(double b, int64_t j) {
  if (j == 0) return 1.0;
  double x = (double)j;
  return std::pow(x, b) * std::expm1(b * std::log1p(1.0 / x));
}

}  // namespace

// Digamma by upward recurrence to x >= 12 and the asymptotic series
// psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)  (Abramowitz & Stegun 6.3.18).
double digamma(double x) {
  double acc = 0.0;
  while (x < 12.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double inv = 1.0 / x, inv2 = inv * inv;
  // B2/2 = 1/12, B4/4 = -1/120, B6/6 = 1/252, B8/8 = -1/240, B10/10 = 1/132, B12/12 = -691/32760
  double s = inv2 * (1.0 / 12 - inv2 * (1.0 / 120 - inv2 * (1.0 / 252 - inv2 * (1.0 / 240 - inv2 * (1.0 / 132 - inv2 * (691.0 / 32760))))));
  return acc + std::log(x) - 0.5 * inv - s;
}

double scheme_scale(int kind, double gamma, double tau) {
  long double g = gamma;
  long double p = std::exp(-g * std::log((long double)tau));
  return (double)(p / std::tgamma((kind == 0 ? 2.0L : 3.0L) - g));
}

void scheme_weights(int kind, double gamma, double tau, int64_t n, double* a, double* dadg) {
  const double s = scheme_scale(kind, gamma, tau);
  // d ln(s)/dg
  const double dls = -std::log(tau) + digamma((kind == 0 ? 2.0 : 3.0) - gamma);
  const double b = kind == 0 ? 1.0 - gamma : 2.0 - gamma;
  // dg = -db
  for (int64_t j = 0; j < n; ++j) {
    double v, dv_db = 0.0;
    if (j == 0) {
      v = 1.0;
      dv_db = 0.0;
    } else if (kind == 0) {
      v = (j >= kSeriesFrom) ? second_diff_series(b, j, &dv_db) : second_diff_direct(b, j, &dv_db);
    } else if (j == 1) {
      v = std::exp2(b) - 3.0;
      dv_db = std::exp2(b) * std::log(2.0);
    } else {
      v = (j >= kSeriesFrom) ? third_diff_series(b, j, &dv_db) : third_diff_direct(b, j, &dv_db);
    }
    a[j] = s * v;
    if (dadg) dadg[j] = s * (dls * v - dv_db);
  }
}

void difference_weights(int kind, double gamma, double tau, int64_t n, double* e) {
  // e_j = c1 q_j: the scheme rewritten in the difference quotients v_k = (u^k - u^{k-1})/tau
  // (the form in which the L1 quotient and Eq. 15 are written).  c1 = scale * tau.
  //   kind 0: q_j = G_j = (j+1)^b - j^b,                b = 1 - g
  //   kind 1: q_0 = M_0 = 1, q_j = M_j - M_{j-1},        b = 2 - g
  const double c1 = scheme_scale(kind, gamma, tau) * tau;
  const double b = kind == 0 ? 1.0 - gamma : 2.0 - gamma;
  for (int64_t j = 0; j < n; ++j) {
    double q;
    if (j == 0) {
      q = 1.0;
    } else if (kind == 0) {
      q = first_diff(b, j);
    } else {
      q = (j >= kSeriesFrom) ? second_diff_series(b, j, nullptr) : second_diff_direct(b, j, nullptr);
    }
    e[j] = c1 * q;
  }
}

void initial_weights(int kind, double gamma, double tau, int64_t n, double* wu0, double* wphi) {
  const double s = scheme_scale(kind, gamma, tau);
  if (kind == 0) {
    // +mu*G_{n-1} u^0 on the right-hand side of level n (L1 quotient expanded)
    const double b = 1.0 - gamma;
    for (int64_t k = 1; k <= n; ++k) {
      wu0[k - 1] = s * first_diff(b, k - 1);
      wphi[k - 1] = 0.0;
    }
  } else {
    // +c (M_{n-1} - M_{n-2}) u^0 + c tau M_{n-1} phi, with M_{-1} = 0
    const double b = 2.0 - gamma;
    for (int64_t k = 1; k <= n; ++k) {
      double mprev = first_diff(b, k - 1);
      double d;
      if (k == 1) {
        d = 1.0;  // M_0 - M_{-1}
      } else if (k - 1 >= kSeriesFrom) {
        d = second_diff_series(b, k - 1, nullptr);  // M_{k-1} - M_{k-2}
      } else {
        d = second_diff_direct(b, k - 1, nullptr);
      }
      wu0[k - 1] = s * d;
      wphi[k - 1] = s * tau * mprev;
    }
  }
}

}  // namespace ftoep
