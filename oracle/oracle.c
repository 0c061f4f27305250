/*
 * oracle.c -- plain, slow CPU oracle for the L1 Caputo time-marching schemes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it (through oracle/oracle.py).  It shares no code, no
 * header and no table with the CUDA path.
 *
 * What it computes (Liu, Cheng, Li, Wang, "Fast procedures for Caputo fractional
 * ordinary and partial differential equations"):
 *
 *   - L1 weights G_k = (k+1)^(1-g) - k^(1-g)          (Lemma 1; Sec. 3 definitions)
 *     and M_k = (k+1)^(2-g) - k^(2-g)                  (Sec. 3 definitions)
 *     evaluated in binary128 and rounded once to double (the paper does not state
 *     a precision; the differences cancel catastrophically in double).
 *   - Scheme 4 (Eq. 19) advanced by the direct time-marching procedure of Eq. 20:
 *     for n = 1..N solve the tridiagonal system
 *         (mu*G_0 + 2/h^2) u_j^n - (u_{j-1}^n + u_{j+1}^n)/h^2
 *             = f_j^n + mu*[ sum_{k=1}^{n-1} (G_{n-k-1} - G_{n-k}) u_j^k + G_{n-1} u_j^0 ]
 *     (mu = tau^-g / Gamma(2-g); the u^0 coefficient follows from expanding the L1
 *     quotient, see or_initial_weights()).  The paper states no precision for these
 *     sums; in this form the history terms carry tau^-g and cancel to the size of f, so
 *     the coefficients and the marched values are kept as double-double pairs (hi + lo)
 *     and the history sums are accumulated with error-free products and sums (the
 *     double-double dot product of Ogita, Rump and Oishi, "Accurate sum and dot product",
 *     2005); each level's right-hand side and the tridiagonal level solve are done in
 *     binary128 (see dd_history() and thomas_const()).
 *   - The hyperbolic L1 scheme of Eq. 15 / Eq. 17 (1<g<2, c = tau^-g/Gamma(3-g)) with
 *     the advection term replaced by the central second difference, spatial term at
 *     level n and f at t_{n-1/2}:
 *         c*M_0 u^n + c(M_1-2M_0) u^{n-1} + c sum_{k=1}^{n-2} W_{n-k} u^k
 *             + c(M_{n-2}-M_{n-1}) u^0 - c*tau*M_{n-1} phi - (u_xx)_h^n = f^{n-1/2}
 *     with W_j = M_{j-2} - 2M_{j-1} + M_j and M_{-1} = 0.
 *   - kind 2: the same hyperbolic time discretization (Eq. 15) with the spatial term
 *     taken as the average of levels n and n-1, the Crank-Nicolson form of the scheme
 *     that Eq. 15 is taken from (Sun and Wu, cited in Sec. 3 for Eq. 15):
 *         [same time terms as kind 1] - (u_xx)_h^{n-1/2} = f^{n-1/2},
 *         (u_xx)_h^{n-1/2} = ((u_xx)_h^n + (u_xx)_h^{n-1})/2,  u^{n-1} = u^0 at n = 1,
 *     which moves half of the spatial operator to the previous level: O(tau^(3-g) + h^2).
 *   - the scalar problem D^g u = -lambda u + f on the same time grid (no space).
 *   - the transposed (adjoint) system, marched backwards in time.
 *   - the orthonormal sine projection of one spatial mode, and a dense Toeplitz
 *     matrix-vector product, as plain sums.
 *
 * Layout of every field: [M][N] row-major, time index contiguous; entry (j, n-1)
 * holds the value at x_j = j*h (j = 1..M) and time level n (n = 1..N).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__aarch64__)
/* AArch64 Linux: long double is IEEE binary128. */
typedef long double qreal;
#define QPOW(a, b) powl((a), (b))
#define QLOG(a) logl(a)
#define QEXP(a) expl(a)
#define QTGAMMA(a) tgammal(a)
#define QLIT(x) x##L
#else
#include <quadmath.h>
typedef __float128 qreal;
#define QPOW(a, b) powq((a), (b))
#define QLOG(a) logq(a)
#define QEXP(a) expq(a)
#define QTGAMMA(a) tgammaq(a)
#define QLIT(x) x##Q
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* kind: 0 = sub-diffusion L1 (0<g<1), 1 = hyperbolic L1 (1<g<2), 2 = hyperbolic L1 with
 * the spatial term averaged over levels n and n-1 (1<g<2).  Kinds 1 and 2 share every
 * time weight; kind_time() maps a kind to the family of its weights. */
/* space: 0 = scalar (D^g u = -lambda u + f), 1 = Dirichlet Laplacian on (0, L). */

/* k^beta in binary128, with 0^beta = 0 for beta > 0. */
static qreal qpow_int(int64_t k, qreal beta) {
  if (k <= 0) return QLIT(0.0);
  return QPOW((qreal)k, beta);
}

/* G_k = (k+1)^(1-g) - k^(1-g), k >= 0 (Lemma 1). */
static qreal q_G(int64_t k, qreal g) {
  qreal b = QLIT(1.0) - g;
  return qpow_int(k + 1, b) - qpow_int(k, b);
}

/* M_k = (k+1)^(2-g) - k^(2-g), k >= 0; M_{-1} = M_{-2} = 0 (Sec. 3 definitions). */
static qreal q_M(int64_t k, qreal g) {
  if (k < 0) return QLIT(0.0);
  qreal b = QLIT(2.0) - g;
  return qpow_int(k + 1, b) - qpow_int(k, b);
}

/* Scale of the time stencil: mu = tau^-g/Gamma(2-g) (Lemma 2) or
 * c = tau^-g/Gamma(3-g) (Eq. 17), in binary128. */
static int kind_time(int kind);

static qreal q_scale(int kind, qreal g, qreal tau) {
  kind = kind_time(kind);
  qreal p = QEXP(-g * QLOG(tau));
  return kind == 0 ? p / QTGAMMA(QLIT(2.0) - g) : p / QTGAMMA(QLIT(3.0) - g);
}

static int check_kind(int kind, double g) {
  if (kind == 0) return (g > 0.0 && g < 1.0) ? OR_OK : OR_EINVAL;
  if (kind == 1 || kind == 2) return (g > 1.0 && g < 2.0) ? OR_OK : OR_EINVAL;
  return OR_EINVAL;
}

static int kind_time(int kind) { return kind == 2 ? 1 : kind; }

/* Weight of the level-n spatial operator in the level-n row: 1, or 1/2 for kind 2 (the
 * other half acts on level n-1). */
static qreal space_weight(int kind) { return kind == 2 ? QLIT(0.5) : QLIT(1.0); }

/* (S w)_j for the spatial operator S of the left-hand side: -(w_{j-1} - 2w_j + w_{j+1})/h^2
 * (space 1, zero boundary values) or lambda w_j (space 0), of the double-pair field
 * wh + wl at stride `stride` (row j at j*stride), in binary128. */
static qreal apply_space(int space, int64_t M, int64_t j, const double* wh, const double* wl, int64_t stride,
                         qreal inv_h2, qreal lambda) {
  const qreal c = (qreal)wh[j * stride] + (qreal)(wl ? wl[j * stride] : 0.0);
  if (space == 0) return lambda * c;
  const qreal lft = j > 0 ? (qreal)wh[(j - 1) * stride] + (qreal)(wl ? wl[(j - 1) * stride] : 0.0) : QLIT(0.0);
  const qreal rgt = j + 1 < M ? (qreal)wh[(j + 1) * stride] + (qreal)(wl ? wl[(j + 1) * stride] : 0.0) : QLIT(0.0);
  return (QLIT(2.0) * c - lft - rgt) * inv_h2;
}

/* G_k for k = 0..K-1, rounded to double. */
int or_G(double g, int64_t K, double* out) {
  if (!(g > 0.0 && g < 1.0) || K < 0 || (K > 0 && !out)) return OR_EINVAL;
  for (int64_t k = 0; k < K; ++k) out[k] = (double)q_G(k, (qreal)g);
  return OR_OK;
}

/* M_k for k = 0..K-1, rounded to double. */
int or_M(double g, int64_t K, double* out) {
  if (!(g > 1.0 && g < 2.0) || K < 0 || (K > 0 && !out)) return OR_EINVAL;
  for (int64_t k = 0; k < K; ++k) out[k] = (double)q_M(k, (qreal)g);
  return OR_OK;
}

/* Unscaled coefficient of u^{n-j} on the left-hand side at level n, for j = 0..N-1,
 * each formed in binary128 from the paper's weights and rounded once:
 *   kind 0 (Eq. 4/19):  j = 0: G_0;          j >= 1: -(G_{j-1} - G_j)
 *   kind 1 (Eq. 17):    j = 0: M_0;  j = 1: M_1 - 2 M_0;  j >= 2: W_j = M_{j-2} - 2M_{j-1} + M_j
 * The full left-hand coefficient is scale * coef[j]. */
static qreal q_coef(int kind, int64_t j, qreal g) {
  kind = kind_time(kind);
  if (kind == 0) {
    if (j == 0) return q_G(0, g);
    return -(q_G(j - 1, g) - q_G(j, g));
  }
  if (j == 0) return q_M(0, g);
  if (j == 1) return q_M(1, g) - QLIT(2.0) * q_M(0, g);
  return q_M(j - 2, g) - QLIT(2.0) * q_M(j - 1, g) + q_M(j, g);
}

int or_time_coeffs(int kind, double g, int64_t N, double* coef) {
  if (check_kind(kind, g) != OR_OK || N < 1 || !coef) return OR_EINVAL;
  for (int64_t j = 0; j < N; ++j) coef[j] = (double)q_coef(kind, j, (qreal)g);
  return OR_OK;
}

/* Scale mu (kind 0) or c (kind 1) for step tau, rounded to double. */
double or_scale(int kind, double g, double tau) { return (double)q_scale(kind, (qreal)g, (qreal)tau); }

/* d/dg of the full coefficients scale(g) * coef_j(g), j = 0..N-1, by a central
 * difference of the binary128 definitions (step 1e-10: truncation ~1e-20 and
 * rounding ~1e-24 relative, both far below double precision). */
int or_time_coeffs_dgamma(int kind, double g, double tau, int64_t N, double* out) {
  if (check_kind(kind, g) != OR_OK || N < 1 || !out) return OR_EINVAL;
  const qreal d = QLIT(1e-10);
  qreal gp = (qreal)g + d, gm = (qreal)g - d;
  qreal sp = q_scale(kind, gp, (qreal)tau), sm = q_scale(kind, gm, (qreal)tau);
  for (int64_t j = 0; j < N; ++j) {
    qreal vp = sp * q_coef(kind, j, gp), vm = sm * q_coef(kind, j, gm);
    out[j] = (double)((vp - vm) / (QLIT(2.0) * d));
  }
  return OR_OK;
}

/* Right-hand-side weights of the initial data at level n = 1..N (index n-1), from
 * expanding the stencils:
 *   kind 0: L1 quotient mu*sum_{k=1}^{n} G_{n-k}(u^k - u^{k-1}) leaves -mu*G_{n-1} u^0
 *           on the left, i.e. +mu*G_{n-1} u^0 on the right.  (Eq. 4 prints "+G_n u_0";
 *           the expansion gives G_{n-1}, which is what is used here.)
 *   kind 1: Eq. 17 leaves c(M_{n-2} - M_{n-1}) u^0 - c*tau*M_{n-1} phi on the left, with
 *           M_{-1} = 0 (at n = 1 the u^0 weight is -c*M_0, which the expansion of Eq. 15
 *           gives directly), i.e. +c(M_{n-1} - M_{n-2}) u^0 + c*tau*M_{n-1} phi on the right.
 * w_u0[n-1] and w_phi[n-1] include the scale; w_phi is zero for kind 0. */
int or_initial_weights(int kind, double g, double tau, int64_t N, double* w_u0, double* w_phi) {
  if (check_kind(kind, g) != OR_OK || N < 1 || !w_u0 || !w_phi) return OR_EINVAL;
  qreal s = q_scale(kind, (qreal)g, (qreal)tau);
  kind = kind_time(kind);
  for (int64_t n = 1; n <= N; ++n) {
    if (kind == 0) {
      w_u0[n - 1] = (double)(s * q_G(n - 1, (qreal)g));
      w_phi[n - 1] = 0.0;
    } else {
      w_u0[n - 1] = (double)(s * (q_M(n - 1, (qreal)g) - q_M(n - 2, (qreal)g)));
      w_phi[n - 1] = (double)(s * (qreal)tau * q_M(n - 1, (qreal)g));
    }
  }
  return OR_OK;
}

/* Thomas algorithm for the constant tridiagonal system
 *   diag*x_j + off*(x_{j-1} + x_{j+1}) = r_j,  j = 0..M-1, x_{-1} = x_M = 0,
 * carried out in binary128.  With diag ~ 2/h^2 >> mu the matrix has condition
 * ~ (mu + 4/h^2)/(mu + pi^2), e.g. 1.6e3 at h = 1/1024, mu = 2.6e3: a double sweep loses
 * that factor times eps at every level.  cp: scratch of length M.  Overwrites r with x. */
static void thomas_const(int64_t M, qreal diag, qreal off, qreal* r, qreal* cp) {
  cp[0] = off / diag;
  r[0] = r[0] / diag;
  for (int64_t j = 1; j < M; ++j) {
    qreal den = diag - off * cp[j - 1];
    cp[j] = off / den;
    r[j] = (r[j] - off * r[j - 1]) / den;
  }
  for (int64_t j = M - 2; j >= 0; --j) r[j] -= cp[j] * r[j + 1];
}

/* Double-double arithmetic (error-free transformations, Knuth / Dekker with FMA). */
static inline void two_sum(double a, double b, double* s, double* e) {
  const double x = a + b;
  const double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

/* sum_{i<n} (ch_i + cl_i)(xh_i + xl_i) as an unevaluated sum hi + lo, accurate to about
 * 2^-104 of sum |c x| + 2^-53 of the result: the hi*hi products and their running sum
 * are error-free (FMA residual, two-sum), the small cross terms are added plainly. */
static void dd_dot(const double* ch, const double* cl, const double* xh, const double* xl, int64_t n, qreal* out) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double a = ch[i], al = cl[i];
    const double p = a * xh[i];
    const double pe = fma(a, xh[i], -p);
    double t, te;
    two_sum(s, p, &t, &te);
    s = t;
    c += te + pe + (a * xl[i] + al * xh[i]);
  }
  *out = (qreal)s + (qreal)c;
}

/* Split a binary128 value into a double pair. */
static inline void q_split(qreal v, double* hi, double* lo) {
  *hi = (double)v;
  *lo = (double)(v - (qreal)*hi);
}

/*
 * Direct time marching (Eq. 20 for kind 0, the direct procedure of Eq. 17 for kind 1,
 * and the scalar analogue for space 0).  Cost O(M N^2).
 *
 * f, u: [M][N] (time contiguous).  u0, phi: length M or NULL (= 0).  For space 0 every
 * row j is an independent scalar problem with the same lambda.
 * T: final time (tau = T/N).  Lx: length of the space interval (h = Lx/(M+1)).
 */
int or_march(int kind, int space, double g, double T, double Lx, double lambda, int64_t N, int64_t M,
             const double* f, const double* u0, const double* phi, double* u, int nthreads) {
  if (check_kind(kind, g) != OR_OK || (space != 0 && space != 1) || N < 1 || M < 1 || !f || !u)
    return OR_EINVAL;
  if (!(T > 0.0) || (space == 1 && !(Lx > 0.0))) return OR_EINVAL;
  const double tau = T / (double)N;
  /* full left-hand coefficients a_j = scale*coef_j (binary128, split into double pairs),
   * stored reversed so that the history sum of level n runs forward in memory:
   * rh[N-1-j] + rl[N-1-j] = a_j */
  double* rh = (double*)malloc(sizeof(double) * (size_t)N);
  double* rl = (double*)malloc(sizeof(double) * (size_t)N);
  double* wu0 = (double*)malloc(sizeof(double) * (size_t)N);
  double* wphi = (double*)malloc(sizeof(double) * (size_t)N);
  double* ulo = (double*)malloc(sizeof(double) * (size_t)N * (size_t)M);
  qreal* rq = (qreal*)malloc(sizeof(qreal) * (size_t)M);
  qreal* cp = (qreal*)malloc(sizeof(qreal) * (size_t)M);
  if (!rh || !rl || !wu0 || !wphi || !ulo || !rq || !cp) {
    free(rh); free(rl); free(wu0); free(wphi); free(ulo); free(rq); free(cp);
    return OR_ENOMEM;
  }
  const qreal qs = q_scale(kind, (qreal)g, (qreal)tau);
  for (int64_t j = 0; j < N; ++j) q_split(qs * q_coef(kind, j, (qreal)g), &rh[N - 1 - j], &rl[N - 1 - j]);
  or_initial_weights(kind, g, tau, N, wu0, wphi);
  /* level matrix: a_0 + sw*2/h^2 on the diagonal, -sw/h^2 off it (binary128), sw the
   * weight of the level-n spatial operator (1/2 for kind 2, whose other half acts on
   * level n-1 and moves to the right-hand side) */
  qreal diag, off, inv_h2 = QLIT(0.0);
  const qreal a0 = qs * q_coef(kind, 0, (qreal)g);
  const qreal sw = space_weight(kind);
  if (space == 1) {
    qreal h = (qreal)Lx / (qreal)(M + 1);
    inv_h2 = QLIT(1.0) / (h * h);
    diag = a0 + sw * QLIT(2.0) * inv_h2;
    off = -sw * inv_h2;
  } else {
    diag = a0 + sw * (qreal)lambda;
    off = QLIT(0.0);
  }
  if (nthreads < 1) nthreads = 1;
  for (int64_t n = 1; n <= N; ++n) {
    /* r_j = f_j^n - sum_{k=1}^{n-1} a_{n-k} u_j^k (+ initial-data terms)
     *       [kind 2: - (1/2) (S u^{n-1})_j, u^0 the initial value] */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t j = 0; j < M; ++j) {
      qreal s = QLIT(0.0);
      if (n > 1) dd_dot(rh + (N - n), rl + (N - n), u + j * N, ulo + j * N, n - 1, &s);
      qreal r = (qreal)f[j * N + (n - 1)] - s;
      if (u0) r += (qreal)wu0[n - 1] * (qreal)u0[j];
      if (phi) r += (qreal)wphi[n - 1] * (qreal)phi[j];
      if (kind == 2) {
        if (n > 1)
          r -= (QLIT(1.0) - sw) * apply_space(space, M, j, u + (n - 2), ulo + (n - 2), N, inv_h2, (qreal)lambda);
        else if (u0)
          r -= (QLIT(1.0) - sw) * apply_space(space, M, j, u0, NULL, 1, inv_h2, (qreal)lambda);
      }
      rq[j] = r;
    }
    if (space == 1) {
      thomas_const(M, diag, off, rq, cp);
    } else {
      for (int64_t j = 0; j < M; ++j) rq[j] = rq[j] / diag;
    }
    for (int64_t j = 0; j < M; ++j) q_split(rq[j], &u[j * N + (n - 1)], &ulo[j * N + (n - 1)]);
  }
  free(rh); free(rl); free(wu0); free(wphi); free(ulo); free(rq); free(cp);
  return OR_OK;
}

/*
 * Transposed system A^T lam = g, A the left-hand operator of or_march (zero initial
 * data).  The time part of A is lower-triangular Toeplitz with first column
 * scale*coef; its transpose is upper triangular, so the march runs n = N..1:
 *   diag*lam_j^n + off*(lam_{j-1}^n + lam_{j+1}^n) = g_j^n - scale*sum_{k=n+1}^{N} coef_{k-n} lam_j^k
 */
int or_adjoint_march(int kind, int space, double g, double T, double Lx, double lambda, int64_t N,
                     int64_t M, const double* gin, double* lam, int nthreads) {
  if (check_kind(kind, g) != OR_OK || (space != 0 && space != 1) || N < 1 || M < 1 || !gin || !lam)
    return OR_EINVAL;
  const double tau = T / (double)N;
  /* a_j = scale*coef_j as double pairs, in natural order (the sum of level n runs over
   * k = n+1..N with weight a_{k-n}) */
  double* ah = (double*)malloc(sizeof(double) * (size_t)N);
  double* al = (double*)malloc(sizeof(double) * (size_t)N);
  double* llo = (double*)malloc(sizeof(double) * (size_t)N * (size_t)M);
  qreal* rq = (qreal*)malloc(sizeof(qreal) * (size_t)M);
  qreal* cp = (qreal*)malloc(sizeof(qreal) * (size_t)M);
  if (!ah || !al || !llo || !rq || !cp) {
    free(ah); free(al); free(llo); free(rq); free(cp);
    return OR_ENOMEM;
  }
  const qreal qs = q_scale(kind, (qreal)g, (qreal)tau);
  for (int64_t j = 0; j < N; ++j) q_split(qs * q_coef(kind, j, (qreal)g), &ah[j], &al[j]);
  qreal diag, off, inv_h2 = QLIT(0.0);
  const qreal a0 = qs * q_coef(kind, 0, (qreal)g);
  const qreal sw = space_weight(kind);
  if (space == 1) {
    qreal h = (qreal)Lx / (qreal)(M + 1);
    inv_h2 = QLIT(1.0) / (h * h);
    diag = a0 + sw * QLIT(2.0) * inv_h2;
    off = -sw * inv_h2;
  } else {
    diag = a0 + sw * (qreal)lambda;
    off = QLIT(0.0);
  }
  if (nthreads < 1) nthreads = 1;
  for (int64_t n = N; n >= 1; --n) {
    /* kind 2: the level-(n+1) row holds (1/2) S u^n, so the transposed row n holds
     * (1/2) S lam^{n+1} (S symmetric) */
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int64_t j = 0; j < M; ++j) {
      qreal s = QLIT(0.0);
      if (n < N) dd_dot(ah + 1, al + 1, lam + j * N + n, llo + j * N + n, N - n, &s);
      if (kind == 2 && n < N)
        s += (QLIT(1.0) - sw) * apply_space(space, M, j, lam + n, llo + n, N, inv_h2, (qreal)lambda);
      rq[j] = (qreal)gin[j * N + (n - 1)] - s;
    }
    if (space == 1) {
      thomas_const(M, diag, off, rq, cp);
    } else {
      for (int64_t j = 0; j < M; ++j) rq[j] = rq[j] / diag;
    }
    for (int64_t j = 0; j < M; ++j) q_split(rq[j], &lam[j * N + (n - 1)], &llo[j * N + (n - 1)]);
  }
  free(ah); free(al); free(llo); free(rq); free(cp);
  return OR_OK;
}

/*
 * Advection schemes of Sec. 3, direct method (time order; at every level a forward sweep in
 * space from the inflow boundary u(0, t) = 0, a = 1).  Cost O(M N^2).
 *   scheme 2 (0 < g < 1, Eq. 12/13): the L1 quotient at x_{i-1/2} as the average of the L1
 *     formulas of nodes i and i-1 (scale c = tau^-g/(2 Gamma(2-g)), i.e. half the scale of
 *     Eq. 4), the derivative (U_i - U_{i-1})/h, f at (x_{i-1/2}, t_n):
 *        c L1[U_i]^n + c L1[U_{i-1}]^n + (U_i^n - U_{i-1}^n)/h = f_{i-1/2}^n,
 *     L1[U]^n = sum_{k=1}^{n} l_{n-k} U^k - G_{n-1} U^0 (l_0 = 1, l_j = G_j - G_{j-1}).
 *   scheme 3 (1 < g < 2, Eq. 16/17): the time terms of Eq. 17 at node i (scale
 *     c = tau^-g/Gamma(3-g), the hyperbolic first column and initial-data weights) with the
 *     derivative (U_i^n - U_{i-1}^n)/h at level n, f at (x_i, t_{n-1/2}).
 * Nodes x_i = i h, h = Lx/M, i = 1..M, U_0 = 0.  f, u: [M][N]; u0, phi: length M or NULL
 * (phi used by scheme 3 only).  Level values in binary128; history sums by the double-double
 * dot product (as or_march).
 */
int or_advection_march(int scheme, double g, double T, double Lx, int64_t N, int64_t M, const double* f,
                       const double* u0, const double* phi, double* u) {
  if (!((scheme == 2 && g > 0.0 && g < 1.0) || (scheme == 3 && g > 1.0 && g < 2.0))) return OR_EINVAL;
  if (N < 1 || M < 1 || !f || !u || !(T > 0.0) || !(Lx > 0.0)) return OR_EINVAL;
  const int kind = scheme == 2 ? 0 : 1;
  const double tau = T / (double)N;
  const qreal h = (qreal)Lx / (qreal)M;
  double* rh = (double*)malloc(sizeof(double) * (size_t)N);
  double* rl = (double*)malloc(sizeof(double) * (size_t)N);
  double* wu0 = (double*)malloc(sizeof(double) * (size_t)N);
  double* wphi = (double*)malloc(sizeof(double) * (size_t)N);
  double* ulo = (double*)malloc(sizeof(double) * (size_t)N * (size_t)M);
  qreal* hist = (qreal*)malloc(sizeof(qreal) * (size_t)M);
  if (!rh || !rl || !wu0 || !wphi || !ulo || !hist) {
    free(rh); free(rl); free(wu0); free(wphi); free(ulo); free(hist);
    return OR_ENOMEM;
  }
  /* a_j = scale * coef_j (reversed, double pairs), scale halved for scheme 2 */
  const qreal qs = q_scale(kind, (qreal)g, (qreal)tau) * (scheme == 2 ? QLIT(0.5) : QLIT(1.0));
  for (int64_t j = 0; j < N; ++j) q_split(qs * q_coef(kind, j, (qreal)g), &rh[N - 1 - j], &rl[N - 1 - j]);
  or_initial_weights(kind, g, tau, N, wu0, wphi);  /* full scale; halved below for scheme 2 */
  const qreal a0 = qs * q_coef(kind, 0, (qreal)g);
  const qreal ih = QLIT(1.0) / h;
  for (int64_t n = 1; n <= N; ++n) {
    for (int64_t i = 0; i < M; ++i) {
      qreal s = QLIT(0.0);
      if (n > 1) dd_dot(rh + (N - n), rl + (N - n), u + i * N, ulo + i * N, n - 1, &s);
      hist[i] = s;
    }
    qreal prev = QLIT(0.0), prev_hist = QLIT(0.0), prev_u0 = QLIT(0.0);  /* node 0: U = 0 */
    for (int64_t i = 0; i < M; ++i) {
      qreal r = (qreal)f[i * N + (n - 1)] - hist[i];
      const qreal ui0 = u0 ? (qreal)u0[i] : QLIT(0.0);
      qreal x;
      if (scheme == 2) {
        /* + c G_{n-1} (U_i^0 + U_{i-1}^0): the initial-data term of both L1 formulas */
        r += QLIT(0.5) * (qreal)wu0[n - 1] * (ui0 + prev_u0);
        r += (ih - a0) * prev - prev_hist;
        x = r / (a0 + ih);
      } else {
        r += (qreal)wu0[n - 1] * ui0;
        if (phi) r += (qreal)wphi[n - 1] * (qreal)phi[i];
        r += ih * prev;
        x = r / (a0 + ih);
      }
      q_split(x, &u[i * N + (n - 1)], &ulo[i * N + (n - 1)]);
      prev = x;
      prev_hist = hist[i];
      prev_u0 = ui0;
    }
  }
  free(rh); free(rl); free(wu0); free(wphi); free(ulo); free(hist);
  return OR_OK;
}

/* Orthonormal sine coefficient of mode m (1..M) of every time column:
 *   out[n] = sqrt(2/(M+1)) * sum_{j=1}^{M} f_j^n sin(m*pi*j/(M+1)).
 * The sine values are taken in binary128 and rounded; the sum is plain double. */
int or_sine_project(int64_t M, int64_t N, const double* f, int64_t m, double* out) {
  if (M < 1 || N < 1 || m < 1 || m > M || !f || !out) return OR_EINVAL;
  double* sv = (double*)malloc(sizeof(double) * (size_t)M);
  if (!sv) return OR_ENOMEM;
#if defined(__aarch64__)
  const qreal qpi = 3.141592653589793238462643383279502884L;
#define QSIN(a) sinl(a)
#else
  const qreal qpi = M_PIq;
#define QSIN(a) sinq(a)
#endif
  qreal nrm = QPOW((qreal)2.0 / (qreal)(M + 1), QLIT(0.5));
  for (int64_t j = 1; j <= M; ++j) {
    /* reduce m*j modulo 2(M+1) exactly before the sine */
    int64_t r = (m * j) % (2 * (M + 1));
    sv[j - 1] = (double)(nrm * QSIN(qpi * (qreal)r / (qreal)(M + 1)));
  }
  for (int64_t n = 0; n < N; ++n) out[n] = 0.0;
  for (int64_t j = 0; j < M; ++j) {
    const double* fj = f + j * N;
    double s = sv[j];
    for (int64_t n = 0; n < N; ++n) out[n] += s * fj[n];
  }
  free(sv);
  return OR_OK;
}

/* Dense lower-triangular Toeplitz product, first column a (length N):
 *   transpose = 0: y_n = sum_{k<=n} a_{n-k} x_k;  transpose = 1: y_n = sum_{k>=n} a_{k-n} x_k.
 * Applied to nlines independent lines of length N (stride N). */
int or_toeplitz_matvec(const double* a, int64_t N, const double* x, double* y, int64_t nlines, int transpose) {
  if (N < 1 || nlines < 1 || !a || !x || !y) return OR_EINVAL;
  for (int64_t l = 0; l < nlines; ++l) {
    const double* xl = x + l * N;
    double* yl = y + l * N;
    for (int64_t n = 0; n < N; ++n) {
      double s = 0.0;
      if (!transpose)
        for (int64_t k = 0; k <= n; ++k) s += a[n - k] * xl[k];
      else
        for (int64_t k = n; k < N; ++k) s += a[k - n] * xl[k];
      yl[n] = s;
    }
  }
  return OR_OK;
}
