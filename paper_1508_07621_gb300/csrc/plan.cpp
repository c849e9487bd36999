// Host planning (FP64): drive samples, Magnus-4 scalars, spectral bounds, Bessel weights.
//
// Everything here is computed once per plan, before any propagation (§3: the commutators are
// formed a single time for the whole chain; the set-up part of Algorithm 1).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

static thread_local char g_err[512] = "";

void fq_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* floquet_last_error(void) { return g_err; }

fq_status fq_cuda_fail(cudaError_t e, const char* what) {
  fq_set_error("%s: %s", what, cudaGetErrorString(e));
  return FQ_ECUDA;
}

// f(t) = f_dc + f_ac cos(omega t + phi0) and its first two derivatives (Eq. 13).
double fq_drive_f(int deriv, double f_dc, double f_ac, double omega, double phi0, double t) {
  const double x = omega * t + phi0;
  if (deriv == 0) return f_dc + f_ac * cos(x);
  if (deriv == 1) return -f_ac * omega * sin(x);
  return -f_ac * omega * omega * cos(x);
}

// J_0(R) .. J_L(R) by Miller's backward recurrence (J.C.P. Miller, British Association
// Mathematical Tables X, 1952): run J_{k-1} = (2k/R) J_k - J_{k+1} downward from an index
// well above max(L, R) with an arbitrary seed, then normalise with the identity
// J_0 + 2 sum_{k>=1} J_{2k} = 1.  Downward recurrence is the stable direction for k > R.
void fq_bessel_miller(double R, int L, double* out) {
  if (fabs(R) < 0.5) {
    // small argument: the power series J_l(R) = sum_k (-1)^k (R/2)^{2k+l} / (k! (k+l)!)
    // converges to full precision in a few terms (and avoids 2k/R overflow).
    const double x = 0.5 * R;
    double lead = 1.0;  // (R/2)^l / l!
    for (int l = 0; l <= L; ++l) {
      if (l > 0) lead *= x / l;
      double term = lead, sum = lead;
      for (int k = 1; k < 30 && term != 0.0; ++k) {
        term *= -x * x / ((double)k * (k + l));
        sum += term;
      }
      out[l] = sum;
    }
    return;
  }
  const double top = std::max((double)L, fabs(R));
  int K = (int)(top + 30.0 + 6.0 * sqrt(top));
  K += K & 1;  // even start index keeps the normalisation sum simple
  std::vector<double> j(K + 2, 0.0);
  j[K + 1] = 0.0;
  j[K] = 1e-300;
  for (int k = K; k >= 1; --k) {
    j[k - 1] = (2.0 * k / R) * j[k] - j[k + 1];
    if (fabs(j[k - 1]) > 1e250) {  // rescale everything computed so far
      for (int q = k - 1; q <= K + 1; ++q) j[q] *= 1e-250;
    }
  }
  double s = j[0];
  for (int k = 2; k <= K; k += 2) s += 2.0 * j[k];
  for (int l = 0; l <= L; ++l) out[l] = j[l] / s;
}

// Truncation order (reading R5): smallest integer l > R, l >= 1, with |J_{l+1}(R)| < tol.
// J_l(R) falls faster than geometrically once l - R exceeds a few R^{1/3}, so the search ends
// within a few hundred indices of R (it stops at R + 4096 whatever tol is).
int fq_cheb_order(double R, double tol) {
  const int l0 = std::max(1, (int)floor(R) + 1);
  for (int l = l0;; ++l) {
    std::vector<double> j(l + 2);
    fq_bessel_miller(R, l + 1, j.data());
    if (fabs(j[l + 1]) < tol || l >= l0 + 4096) return l;
  }
}

// Number of eigenvalues < x of the symmetric tridiagonal (diag, off) by the Sturm count of
// the LDL^T pivots.
static int sturm_count(const double* d, const double* e, int n, double x) {
  int c = 0;
  double q = d[0] - x;
  if (q < 0) ++c;
  for (int i = 1; i < n; ++i) {
    if (q == 0.0) q = 1e-300;
    q = (d[i] - x) - e[i - 1] * e[i - 1] / q;
    if (q < 0) ++c;
  }
  return c;
}

// Extreme eigenvalues of a real symmetric tridiagonal matrix by bisection on Sturm counts,
// bracketed by Gershgorin discs; converged to a few ulps of the spectral radius.
void fq_tridiag_extremes(const double* d, const double* e, int n, double* lo, double* hi) {
  double glo = 1e300, ghi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    glo = std::min(glo, d[i] - r);
    ghi = std::max(ghi, d[i] + r);
  }
  const double scale = std::max(fabs(glo), fabs(ghi)) + 1e-300;
  // lowest: smallest x with count(x) >= 1
  double a = glo - 1e-12 * scale, b = ghi + 1e-12 * scale;
  for (int it = 0; it < 200 && b - a > 4e-16 * scale; ++it) {
    double m = 0.5 * (a + b);
    if (sturm_count(d, e, n, m) >= 1) b = m; else a = m;
  }
  *lo = a;  // count(a) = 0: every eigenvalue >= a
  a = glo - 1e-12 * scale;
  b = ghi + 1e-12 * scale;
  for (int it = 0; it < 200 && b - a > 4e-16 * scale; ++it) {
    double m = 0.5 * (a + b);
    if (sturm_count(d, e, n, m) >= n) b = m; else a = m;
  }
  *hi = b;  // count(b) = n: every eigenvalue < b
}

// sum_i a[i] b[i] with four independent partial sums (the compiler may not reassociate one)
static double dot4(const double* a, const double* b, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = 0;
  for (; i + 4 <= n; i += 4) {
    s0 += a[i] * b[i];
    s1 += a[i + 1] * b[i + 1];
    s2 += a[i + 2] * b[i + 2];
    s3 += a[i + 3] * b[i + 3];
  }
  for (; i < n; ++i) s0 += a[i] * b[i];
  return (s0 + s1) + (s2 + s3);
}

// y = A x for a dense row-major symmetric A, rows split over host threads.
static void matvec(const double* a, const double* x, double* y, int n, int nthreads) {
  auto work = [&](int r0, int r1) {
    for (int i = r0; i < r1; ++i) y[i] = dot4(a + (size_t)i * n, x, n);
  };
  if (nthreads <= 1 || n < 256) { work(0, n); return; }
  std::vector<std::thread> th;
  int chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int r0 = t * chunk, r1 = std::min(n, r0 + chunk);
    if (r0 < r1) th.emplace_back(work, r0, r1);
  }
  for (auto& t : th) t.join();
}

// Extreme Ritz values of the Lanczos tridiagonal T_m (alpha, beta[1..m-1]) and the residual
// beta_m |s_{m-1}| of each extreme Ritz vector s (inverse iteration on T_m); a Ritz pair has an
// eigenvalue of A within its residual.
static void ritz_extremes(const std::vector<double>& alpha, const std::vector<double>& beta, int m, bool exact,
                          double* tlo, double* thi, double* rlo, double* rhi) {
  std::vector<double> off(std::max(1, m - 1));
  for (int i = 0; i + 1 < m; ++i) off[i] = beta[i + 1];
  fq_tridiag_extremes(alpha.data(), off.data(), m, tlo, thi);
  auto resid = [&](double theta, bool top) {
    if (exact) return 0.0;
    std::vector<double> x(m, 1.0), dd(m), cc(m), y(m);
    const double shift = theta + 1e-10 * (fabs(theta) + 1.0) * (top ? 1 : -1);
    for (int it = 0; it < 4; ++it) {
      // solve (T - shift) y = x by the tridiagonal Thomas algorithm
      for (int i = 0; i < m; ++i) dd[i] = alpha[i] - shift;
      for (int i = 0; i + 1 < m; ++i) cc[i] = off[i];
      std::vector<double> rhs = x;
      for (int i = 1; i < m; ++i) {
        double piv = dd[i - 1] != 0.0 ? dd[i - 1] : 1e-300;
        double f = off[i - 1] / piv;
        dd[i] -= f * cc[i - 1];
        rhs[i] -= f * rhs[i - 1];
      }
      y[m - 1] = rhs[m - 1] / (dd[m - 1] != 0.0 ? dd[m - 1] : 1e-300);
      for (int i = m - 2; i >= 0; --i) y[i] = (rhs[i] - cc[i] * y[i + 1]) / (dd[i] != 0 ? dd[i] : 1e-300);
      double nn = 0.0;
      for (double v : y) nn += v * v;
      nn = sqrt(nn);
      for (int i = 0; i < m; ++i) x[i] = y[i] / nn;
    }
    return fabs(beta[m] * x[m - 1]);
  };
  *rlo = resid(*tlo, false);
  *rhi = resid(*thi, true);
}

// Extreme eigenvalues of the dense symmetric A by the Lanczos method (Lanczos 1950) with
// full reorthogonalisation.  Returned [lo, hi] is the Ritz interval widened by the residual
// norms of the two extreme Ritz pairs (each such pair has an eigenvalue within its residual)
// plus 1e-6 of the span; with k >= n it is exact up to rounding.  The iteration stops early
// once both residuals are below 1e-5 of the span (checked every 8 steps from step 24); the
// returned interval is widened by them, so this only trades a slightly wider interval for time.
void fq_lanczos_extremes(const fq_matvec& mv, int n, int ksteps, uint64_t seed, double* lo, double* hi) {
  const int k = std::min(n, ksteps);
  std::vector<double> V((size_t)(k + 1) * n), w(n), alpha(k), beta(k + 1, 0.0);
  // start vector: splitmix64 uniforms in (-1, 1)
  uint64_t s = seed;
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    V[i] = ((double)(z >> 11) + 0.5) * (2.0 / 9007199254740992.0) - 1.0;
    nrm += V[i] * V[i];
  }
  nrm = sqrt(nrm);
  for (int i = 0; i < n; ++i) V[i] /= nrm;
  int m = k;
  for (int j = 0; j < k; ++j) {
    double* vj = &V[(size_t)j * n];
    mv(vj, w.data());
    const double al = dot4(w.data(), vj, n);
    alpha[j] = al;
    // full reorthogonalisation (twice is enough)
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q <= j; ++q) {
        const double* vq = &V[(size_t)q * n];
        const double c = dot4(w.data(), vq, n);
        for (int i = 0; i < n; ++i) w[i] -= c * vq[i];
      }
    const double b = sqrt(dot4(w.data(), w.data(), n));
    beta[j + 1] = b;
    if (j + 1 == k) break;
    if (b < 1e-13 * (fabs(al) + 1e-300)) { m = j + 1; break; }  // invariant subspace
    if (j + 1 >= 24 && (j + 1) % 8 == 0) {
      double tl, th, rl, rh;
      ritz_extremes(alpha, beta, j + 1, false, &tl, &th, &rl, &rh);
      if (std::max(rl, rh) < 1e-5 * (th - tl)) { m = j + 1; break; }
    }
    double* vn = &V[(size_t)(j + 1) * n];
    for (int i = 0; i < n; ++i) vn[i] = w[i] / b;
  }
  double tlo, thi, rlo, rhi;
  ritz_extremes(alpha, beta, m, m >= n, &tlo, &thi, &rlo, &rhi);
  const double span = thi - tlo;
  *lo = tlo - rlo - 1e-6 * span;
  *hi = thi + rhi + 1e-6 * span;
}

// ---------------------------------------------------------------- 6th-order Magnus (reading R12)
// Elements of span{H0, H1, K, K0, K1, K00, K01, K10, K11, KK0, KK1} as complex coefficient
// vectors; comm() is the commutator table of the pairs Eq. 14 needs for H = H0 + f H1.
namespace {
struct Cx { double re = 0, im = 0; };
using Lie = Cx[FQ_M6_TERMS];
void lie_zero(Lie& a) { for (auto& c : a) c = Cx{}; }
void lie_axpy(Lie& y, double ar, double ai, const Lie& x) {  // y += (ar + i ai) x
  for (int q = 0; q < FQ_M6_TERMS; ++q) {
    y[q].re += ar * x[q].re - ai * x[q].im;
    y[q].im += ar * x[q].im + ai * x[q].re;
  }
}
// [e_i, e_j] = sign * e_k, or 0 (k = -1)
void comm_basis(int i, int j, int* k, double* sign) {
  static const int tab[5][5] = {
      // H0   H1   K    K0   K1
      {-1, 2, 3, 5, 6},    // H0: [H0,H1]=K, [H0,K]=K0, [H0,K0]=K00, [H0,K1]=K01
      {-2, -1, 4, 7, 8},   // H1: [H1,H0]=-K, [H1,K]=K1, [H1,K0]=K10, [H1,K1]=K11
      {-3, -4, -1, 9, 10}  // K:  [K,H0]=-K0, [K,H1]=-K1, [K,K0]=KK0, [K,K1]=KK1
  };
  *k = -1;
  *sign = 0;
  if (i > 2 || j > 4) return;
  const int t = tab[i][j];
  if (t == -1) return;
  // entries 2..10 positive; -2 / -3 / -4 encode minus K, K0, K1
  if (i == 1 && j == 0) { *k = 2; *sign = -1; return; }
  if (i == 2 && j == 0) { *k = 3; *sign = -1; return; }
  if (i == 2 && j == 1) { *k = 4; *sign = -1; return; }
  *k = t;
  *sign = 1;
}
void lie_comm(Lie& out, const Lie& x, const Lie& y) {
  lie_zero(out);
  for (int i = 0; i < FQ_M6_TERMS; ++i) {
    if (x[i].re == 0 && x[i].im == 0) continue;
    for (int j = 0; j < FQ_M6_TERMS; ++j) {
      if (y[j].re == 0 && y[j].im == 0) continue;
      int k;
      double sg;
      if (i <= 2 && j <= 4) comm_basis(i, j, &k, &sg);
      else if (j <= 2 && i <= 4) { comm_basis(j, i, &k, &sg); sg = -sg; }
      else { k = -2; sg = 0; }
      if (k == -2) continue;  // outside the table: never produced by Eq. 14 for H0 + f H1
      if (k < 0) continue;    // commutator of an element with itself
      out[k].re += sg * (x[i].re * y[j].re - x[i].im * y[j].im);
      out[k].im += sg * (x[i].re * y[j].im + x[i].im * y[j].re);
    }
  }
}
}  // namespace

// Omega_H of step [t0, t0 + h] for Eq. 14 with alphas as 3-point Gauss-Legendre moments of
// A = -i(H0 + f H1): alpha1 = h A_2, alpha2 = (sqrt(15) h/3)(A_3 - A_1),
// alpha3 = (10 h/3)(A_3 - 2 A_2 + A_1); C1 = [alpha1, alpha2], C2 = -(1/60)[alpha1, 2 alpha3 + C1],
// Omega_A = alpha1 + alpha3/12 + (1/240)[-20 alpha1 - alpha3 + C1, alpha2 + C2], Omega_H = i Omega_A.
// out[q]: real coefficient of symmetric basis element q, imaginary factor of antisymmetric ones.
static void magnus6_coefficients(double h, double f1, double f2, double f3, double* out) {
  Lie a1, a2, a3, c1, c2, t, x, y, xy, om;
  lie_zero(a1); lie_zero(a2); lie_zero(a3);
  a1[0].im = -h; a1[1].im = -h * f2;
  a2[1].im = -sqrt(15.0) * h / 3.0 * (f3 - f1);
  a3[1].im = -10.0 * h / 3.0 * (f3 - 2.0 * f2 + f1);
  lie_comm(c1, a1, a2);
  lie_zero(t);
  lie_axpy(t, 2.0, 0.0, a3);
  lie_axpy(t, 1.0, 0.0, c1);
  lie_comm(c2, a1, t);
  for (auto& c : c2) { c.re /= -60.0; c.im /= -60.0; }
  lie_zero(x);
  lie_axpy(x, -20.0, 0.0, a1);
  lie_axpy(x, -1.0, 0.0, a3);
  lie_axpy(x, 1.0, 0.0, c1);
  lie_zero(y);
  lie_axpy(y, 1.0, 0.0, a2);
  lie_axpy(y, 1.0, 0.0, c2);
  lie_comm(xy, x, y);
  lie_zero(om);
  lie_axpy(om, 1.0, 0.0, a1);
  lie_axpy(om, 1.0 / 12.0, 0.0, a3);
  lie_axpy(om, 1.0 / 240.0, 0.0, xy);
  // Omega_H = i Omega_A: (re, im) -> (-im, re)
  static const bool sym[FQ_M6_TERMS] = {true, true, false, true, true, false, false, false, false, true, true};
  for (int q = 0; q < FQ_M6_TERMS; ++q) {
    const double re = -om[q].im, im = om[q].re;
    out[q] = sym[q] ? re : im;
  }
}

// The 11 basis elements of the 6th-order scheme for a tridiagonal H0 (diagonal d0, off-diagonal
// e0) and a diagonal H1 (d1), as bands of half-width 3: H0 and K = [H0,H1] have half-width 1, each
// commutator with H0 or K widens it by one and one with H1 keeps it, so the deepest (K00 =
// [H0,K0], KK0 = [K,K0]) reach 3.  Entry (i, i + d) of element q at band[(q * 7 + d + 3) * n + i].
namespace {
struct Band7 {
  int n;
  std::vector<double> a;  // [7][n]
  explicit Band7(int n_) : n(n_), a((size_t)7 * n_, 0.0) {}
  double get(int i, int j) const { return (j - i >= -3 && j - i <= 3 && i >= 0 && i < n && j >= 0 && j < n) ? a[(size_t)(j - i + 3) * n + i] : 0.0; }
  void set(int i, int j, double v) { a[(size_t)(j - i + 3) * n + i] = v; }
};
// [X, Y] = XY - YX, entries beyond half-width 3 dropped (none arise in the 6th-order basis)
Band7 band_comm(const Band7& x, const Band7& y) {
  const int n = x.n;
  Band7 c(n);
  for (int i = 0; i < n; ++i)
    for (int j = std::max(0, i - 3); j <= std::min(n - 1, i + 3); ++j) {
      double v = 0.0;
      for (int k = std::max(0, i - 3); k <= std::min(n - 1, i + 3); ++k)
        v += x.get(i, k) * y.get(k, j) - y.get(i, k) * x.get(k, j);
      c.set(i, j, v);
    }
  return c;
}
}  // namespace

void fq_tridiag_band6(const double* d0, const double* e0, const double* d1, int n, std::vector<double>& out) {
  Band7 h0(n), h1(n);
  for (int i = 0; i < n; ++i) {
    h0.set(i, i, d0[i]);
    h1.set(i, i, d1[i]);
    if (i + 1 < n) {
      h0.set(i + 1, i, e0[i]);
      h0.set(i, i + 1, e0[i]);
    }
  }
  const Band7 k = band_comm(h0, h1);
  const Band7 k0 = band_comm(h0, k), k1 = band_comm(h1, k);
  const Band7* el[FQ_M6_TERMS];
  const Band7 k00 = band_comm(h0, k0), k01 = band_comm(h0, k1), k10 = band_comm(h1, k0), k11 = band_comm(h1, k1);
  const Band7 kk0 = band_comm(k, k0), kk1 = band_comm(k, k1);
  el[0] = &h0; el[1] = &h1; el[2] = &k; el[3] = &k0; el[4] = &k1; el[5] = &k00;
  el[6] = &k01; el[7] = &k10; el[8] = &k11; el[9] = &kk0; el[10] = &kk1;
  out.assign((size_t)FQ_M6_TERMS * 7 * n, 0.0);
  for (int q = 0; q < FQ_M6_TERMS; ++q) std::copy(el[q]->a.begin(), el[q]->a.end(), out.begin() + (size_t)q * 7 * n);
}

fq_status fq_finish_bounds(fq_plan* plan, double emin, double emax) {
  const double h = plan->h;
  const int M = plan->steps;
  if (!(std::isfinite(emin) && std::isfinite(emax) && emin < emax)) {
    fq_set_error("spectral bounds [%g, %g] of Omega/h are not a finite interval", emin, emax);
    return FQ_EINVAL;
  }
  const double half = 0.5 * emax - 0.5 * emin;  // Delta E, without overflow for bounds near DBL_MAX
  const double r = h * half;
  if (!(r <= FQ_R_MAX)) {
    fq_set_error("R = h Delta E = %g is above %g: the step is too long for the spectral width (use more steps)", r,
                 FQ_R_MAX);
    return FQ_EUNSUPPORTED;
  }
  plan->e_min = emin;
  plan->e_max = emax;
  plan->delta_e = half;
  plan->beta = plan->delta_e + emin;
  plan->R = h * plan->delta_e;
  plan->L = plan->cheb_terms > 0 ? std::max(plan->cheb_terms, fq_cheb_order(plan->R, 1.0)) : fq_cheb_order(plan->R, plan->tol);
  plan->cheb.assign(plan->L + 1, 0.0);
  fq_bessel_miller(plan->R, plan->L, plan->cheb.data());
  for (int l = 1; l <= plan->L; ++l) plan->cheb[l] *= 2.0;
  plan->phase_re = cos(plan->beta * h);
  plan->phase_im = -sin(plan->beta * h);
  // Omega~_m = (Omega_m / h - beta) / Delta E  (reading R2)
  const double inv = 1.0 / (h * plan->delta_e);
  plan->sa.resize(M);
  plan->sb.resize(M);
  plan->sc.resize(M);
  for (int m = 0; m < M; ++m) {
    plan->sa[m] = plan->ma[m] * inv;
    plan->sb[m] = plan->mb[m] * inv;
    plan->sc[m] = plan->mc[m] * inv;
  }
  plan->sbeta = plan->beta / plan->delta_e;
  return FQ_OK;
}

// Host part of plan creation: validates the problem, forms the Magnus scalars (reading R1),
// bounds (reading R4), R, L and a_l (Eq. 12, reading R5).  No device work.
void fq_dense_bounds(int n, double glo, double ghi, double kmax, const fq_dense_apply& apply, double* emin,
                     double* emax) {
  double l1, h1v, l2, h2v;
  fq_lanczos_extremes([&](const double* x, double* y) { apply(0, glo, x, y); }, n, 320, 0x1234567ull, &l1, &h1v);
  fq_lanczos_extremes([&](const double* x, double* y) { apply(0, ghi, x, y); }, n, 320, 0x7654321ull, &l2, &h2v);
  double lo = std::min(l1, l2), hi = std::max(h1v, h2v);
  if (kmax > 0) {  // ||[H0,H1]||_2 <= 2 ||H0||_2 ||H1||_2
    double a0, b0, a1, b1;
    fq_lanczos_extremes([&](const double* x, double* y) { apply(1, 0.0, x, y); }, n, 160, 0x51ull, &a0, &b0);
    fq_lanczos_extremes([&](const double* x, double* y) { apply(2, 0.0, x, y); }, n, 160, 0x52ull, &a1, &b1);
    const double w = kmax * 2.0 * std::max(fabs(a0), fabs(b0)) * std::max(fabs(a1), fabs(b1));
    lo -= w;
    hi += w;
  }
  *emin = lo;
  *emax = hi;
}

// The margins fq_host_plan adds to computed bounds, then the Chebyshev data (fq_finish_bounds).
fq_status fq_finish_computed_bounds(fq_plan* plan, double emin, double emax) {
  const double margin = 1e-12 * std::max(std::max(fabs(emin), fabs(emax)), 1.0);
  emin -= margin;
  emax += margin;
  if (!(emax > emin)) {  // degenerate spectrum (N = 1, or H a multiple of 1)
    const double w = 1e-12 * std::max(fabs(emin), 1.0);
    emin -= w;
    emax += w;
  }
  return fq_finish_bounds(plan, emin, emax);
}

fq_status fq_host_plan(const fq_problem* p, fq_plan* plan, bool defer_dense_bounds) {
  if (!p) { fq_set_error("problem is NULL"); return FQ_EINVAL; }
  if (p->n < 1 || p->steps < 1 || !(p->period > 0) || !std::isfinite(p->period)) {
    fq_set_error("need n >= 1, steps >= 1, finite period > 0 (got %d, %d, %g)", p->n, p->steps, p->period);
    return FQ_EINVAL;
  }
  if (p->format != FQ_DENSE && p->format != FQ_TRIDIAG) { fq_set_error("bad format %d", p->format); return FQ_EINVAL; }
  if (!p->h0 || !p->h1 || (p->format == FQ_TRIDIAG && p->n > 1 && !p->h0_off)) {
    fq_set_error("operator arrays missing");
    return FQ_EINVAL;
  }
  if (p->drive_kind != FQ_DRIVE_COS && p->drive_kind != FQ_DRIVE_PIECEWISE) {
    fq_set_error("bad drive kind %d", p->drive_kind);
    return FQ_EINVAL;
  }
  if (p->drive_kind == FQ_DRIVE_PIECEWISE && !p->f_steps) { fq_set_error("piecewise drive needs f_steps"); return FQ_EINVAL; }
  if (p->drive_kind == FQ_DRIVE_COS &&
      !(std::isfinite(p->f_dc) && std::isfinite(p->f_ac) && std::isfinite(p->omega) && std::isfinite(p->phi0))) {
    fq_set_error("drive parameters must be finite (f_dc %g, f_ac %g, omega %g, phi0 %g)", p->f_dc, p->f_ac, p->omega,
                 p->phi0);
    return FQ_EINVAL;
  }
  if (p->e_max > p->e_min && !(std::isfinite(p->e_min) && std::isfinite(p->e_max))) {
    fq_set_error("caller's bounds [%g, %g] must be finite", p->e_min, p->e_max);
    return FQ_EINVAL;
  }
  {  // every operator entry and drive sample finite: a NaN or Inf would reach the bounds and L
    const size_t nop = p->format == FQ_DENSE ? (size_t)p->n * p->n : (size_t)p->n;
    const struct { const double* a; size_t k; const char* what; } arrays[] = {
        {p->h0, nop, "H0"},
        {p->h1, nop, "H1"},
        {p->format == FQ_TRIDIAG ? p->h0_off : nullptr, (size_t)p->n - 1, "the H0 off-diagonal"},
        {p->drive_kind == FQ_DRIVE_PIECEWISE ? p->f_steps : nullptr, (size_t)p->steps, "f_steps"}};
    for (const auto& x : arrays)
      for (size_t i = 0; x.a && i < x.k; ++i)
        if (!std::isfinite(x.a[i])) {
          fq_set_error("%s has a non-finite entry at %zu", x.what, i);
          return FQ_EINVAL;
        }
  }
  if (p->precision < FQ_FP64 || p->precision > FQ_OZAKI) { fq_set_error("bad precision %d", p->precision); return FQ_EINVAL; }
  if (p->format == FQ_TRIDIAG && (p->precision == FQ_BF16X3 || p->precision == FQ_BF16X6)) {
    fq_set_error("tridiagonal format supports FQ_FP64, FQ_FP32, FQ_DF32 and FQ_OZAKI");
    return FQ_EUNSUPPORTED;
  }
  if (p->format == FQ_DENSE && p->precision == FQ_FP32) {
    fq_set_error("dense format supports FQ_FP64, FQ_DF32 (N <= 128), FQ_BF16X3, FQ_BF16X6 and FQ_OZAKI");
    return FQ_EUNSUPPORTED;
  }
  const int n = p->n, M = p->steps;
  const int order = p->magnus_order == 0 ? 4 : p->magnus_order;
  if (order != 4 && order != 6) { fq_set_error("magnus_order must be 4 or 6 (got %d)", p->magnus_order); return FQ_EINVAL; }
  if (order == 6 && p->drive_kind != FQ_DRIVE_COS) {
    fq_set_error("6th-order Magnus needs FQ_DRIVE_COS");
    return FQ_EUNSUPPORTED;
  }
  if (order == 6 && p->format == FQ_TRIDIAG && p->precision != FQ_FP64) {
    fq_set_error("6th-order Magnus on a tridiagonal plan runs in FQ_FP64 (its nested commutators make Omega~ "
                 "heptadiagonal, which the streaming FP64 kernel applies)");
    return FQ_EUNSUPPORTED;
  }
  plan->order = order;
  plan->n = n;
  plan->steps = M;
  plan->format = p->format;
  plan->precision = p->precision;
  plan->drive_kind = p->drive_kind;
  plan->stride = p->checkpoint_stride > 0 ? p->checkpoint_stride : 16;
  if (p->tile_n != 0 && p->tile_n != 64 && p->tile_n != 128) {
    fq_set_error("tile_n must be 0, 64 or 128 (got %d)", p->tile_n);
    return FQ_EINVAL;
  }
  plan->tile_n = p->tile_n ? p->tile_n : 128;
  if (p->tile_k != 0 && p->tile_k != 32 && p->tile_k != 64) {
    fq_set_error("tile_k must be 0, 32 or 64 (got %d)", p->tile_k);
    return FQ_EINVAL;
  }
  plan->tile_k = p->tile_k == 64 ? 0 : p->tile_k;
  if (p->kernel < FQ_KERNEL_AUTO || p->kernel > FQ_KERNEL_BAND) {
    fq_set_error("kernel must be one of FQ_KERNEL_AUTO .. FQ_KERNEL_BAND (got %d)", p->kernel);
    return FQ_EINVAL;
  }
  plan->period = p->period;
  plan->tol = p->cheb_tol > 0 ? p->cheb_tol : 1e-14;
  if (p->cheb_terms < 0 || p->cheb_terms > 1024) {
    fq_set_error("cheb_terms must be in [0, 1024] (got %d)", p->cheb_terms);
    return FQ_EINVAL;
  }
  plan->cheb_terms = p->cheb_terms;
  plan->f_dc = p->f_dc;
  plan->f_ac = p->f_ac;
  plan->omega = p->omega;
  plan->phi0 = p->phi0;
  const double h = p->period / M;
  plan->h = h;
  plan->ma.assign(M, h);
  plan->mb.resize(M);
  plan->mc.resize(M);
  if (order == 6) plan->coef6.assign((size_t)M * FQ_M6_TERMS, 0.0);
  for (int m = 0; m < M; ++m) {
    const double tau = (m + 0.5) * h;
    if (order == 6) {
      const double c = sqrt(15.0) / 10.0;
      const double f1 = fq_drive_f(0, p->f_dc, p->f_ac, p->omega, p->phi0, tau - c * h);
      const double f2 = fq_drive_f(0, p->f_dc, p->f_ac, p->omega, p->phi0, tau);
      const double f3 = fq_drive_f(0, p->f_dc, p->f_ac, p->omega, p->phi0, tau + c * h);
      double* cm = &plan->coef6[(size_t)m * FQ_M6_TERMS];
      magnus6_coefficients(h, f1, f2, f3, cm);
      plan->mb[m] = cm[1];  // leading part h (H0 + g H1); the commutator terms widen the bounds later
      plan->mc[m] = 0.0;
    } else if (p->drive_kind == FQ_DRIVE_COS) {
      const double f = fq_drive_f(0, p->f_dc, p->f_ac, p->omega, p->phi0, tau);
      const double f1 = fq_drive_f(1, p->f_dc, p->f_ac, p->omega, p->phi0, tau);
      const double f2 = fq_drive_f(2, p->f_dc, p->f_ac, p->omega, p->phi0, tau);
      plan->mb[m] = h * f + h * h * h * f2 / 24.0;
      plan->mc[m] = h * h * h * f1 / 12.0;
    } else {
      plan->mb[m] = h * p->f_steps[m];
      plan->mc[m] = 0.0;
    }
  }
  // range of the H1 coefficient g_m = b_m / h
  double glo = 1e300, ghi = -1e300, kmax = 0.0;
  for (int m = 0; m < M; ++m) {
    glo = std::min(glo, plan->mb[m] / h);
    ghi = std::max(ghi, plan->mb[m] / h);
    kmax = std::max(kmax, fabs(plan->mc[m] / h));
  }
  if (p->drive_kind == FQ_DRIVE_PIECEWISE) {  // reading R11: widen by 10% and freeze
    const double pad = 0.1 * std::max(std::max(ghi - glo, fabs(glo)), std::max(fabs(ghi), 1e-3));
    glo -= pad;
    ghi += pad;
  }
  double emin, emax;
  if (p->e_max > p->e_min) {
    emin = p->e_min;
    emax = p->e_max;
  } else if (p->format == FQ_TRIDIAG) {
    std::vector<double> d(n), k(std::max(1, n - 1));
    double l1, h1v, l2, h2v;
    for (int i = 0; i < n; ++i) d[i] = p->h0[i] + glo * p->h1[i];
    fq_tridiag_extremes(d.data(), p->h0_off, n, &l1, &h1v);
    for (int i = 0; i < n; ++i) d[i] = p->h0[i] + ghi * p->h1[i];
    fq_tridiag_extremes(d.data(), p->h0_off, n, &l2, &h2v);
    emin = std::min(l1, l2);
    emax = std::max(h1v, h2v);
    if (order == 6) {  // Weyl widening by every commutator term, ||B_q||_2 <= its largest row sum
      fq_tridiag_band6(p->h0, p->h0_off, p->h1, n, plan->band6);
      double wsum = 0.0;
      for (int q = 2; q < FQ_M6_TERMS; ++q) {
        double cmax = 0.0;
        for (int m = 0; m < M; ++m) cmax = std::max(cmax, fabs(plan->coef6[(size_t)m * FQ_M6_TERMS + q]));
        double rmax = 0.0;
        for (int i = 0; i < n; ++i) {
          double r = 0.0;
          for (int d = 0; d < 7; ++d) r += fabs(plan->band6[((size_t)q * 7 + d) * n + i]);
          rmax = std::max(rmax, r);
        }
        wsum += cmax / h * rmax;
      }
      emin -= wsum;
      emax += wsum;
    }
    if (kmax > 0 && n > 1) {  // ||[H0,H1]||_2 from the tridiagonal with |K_{i+1,i}|
      std::vector<double> z(n, 0.0);
      for (int i = 0; i + 1 < n; ++i) k[i] = fabs(p->h0_off[i] * (p->h1[i] - p->h1[i + 1]));
      double kl, kh;
      fq_tridiag_extremes(z.data(), k.data(), n, &kl, &kh);
      const double w = kmax * std::max(fabs(kl), fabs(kh));
      emin -= w;
      emax += w;
    }
  } else if (defer_dense_bounds) {
    plan->dense_bounds_pending = true;
    plan->dense_glo = glo;
    plan->dense_ghi = ghi;
    plan->dense_kmax = kmax;
    return FQ_OK;
  } else {
    // about 2^20 multiply-adds per thread at least: thread start-up costs more below that
    const int nt = (int)std::max(1u, std::min<unsigned>(std::min(16u, std::thread::hardware_concurrency()),
                                                         (unsigned)(((size_t)n * n) >> 20)));
    std::vector<double> t(n);
    const fq_dense_apply apply = [&](int which, double g, const double* x, double* y) {
      if (which == 2) {
        matvec(p->h1, x, y, n, nt);
        return;
      }
      matvec(p->h0, x, y, n, nt);
      if (which == 0 && g != 0.0) {
        matvec(p->h1, x, t.data(), n, nt);
        for (int i = 0; i < n; ++i) y[i] += g * t[i];
      }
    };
    fq_dense_bounds(n, glo, ghi, kmax, apply, &emin, &emax);
  }
  if (p->e_max > p->e_min) return fq_finish_bounds(plan, emin, emax);
  return fq_finish_computed_bounds(plan, emin, emax);
}
