/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the Dual-Tree Fast Gauss
 * Transform (Lee, Gray & Moore, "Dual-Tree Fast Gauss Transforms").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two meet only
 * through the seeded point generators.
 *
 * Every routine follows one passage of the paper (cited beside it) in its
 * own order and notation, in double precision, with no blocking or
 * reordering beyond what that passage states.  Readings of garbled or
 * inconsistent passages are marked "Reading:" in place.
 *
 * Conventions
 *   - points are row-major double[n][D];
 *   - a coefficient table of order p in D dimensions is stored with radix
 *     pm >= p (the paper stores p_max^D terms per node and reads the first
 *     p^D multi-indices out of it, Appendix "linear array");
 *   - s = 1/sqrt(2 h^2) is the scale every expansion uses.
 *
 * Pins (tests/test_oracle_*.py): Hermite closed forms and Rodrigues'
 * formula, the generating-function identity, convergence of every
 * truncated expansion to the exact Gaussian sum, the truncation lemmas,
 * exactness of far-to-far and local-to-local translation, grid
 * factorisation of the exact sum, and the per-query epsilon guarantee
 * plus the partition property of the traversal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 32
#define ORC_INF_ORDER (-1)

/* ------------------------------------------------------------------ */
/* Small helpers                                                       */
/* ------------------------------------------------------------------ */

static double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

static int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

/* alpha! = prod_d alpha[d]!  (Section 3.1, multi-index notation) */
static double multi_fact(const int* a, int D) {
  double f = 1.0;
  for (int d = 0; d < D; ++d) f *= fact(a[d]);
  return f;
}

/* |alpha| = sum_d alpha[d] */
static int multi_abs(const int* a, int D) {
  int s = 0;
  for (int d = 0; d < D; ++d) s += a[d];
  return s;
}

/* x^alpha = prod_d x[d]^alpha[d]  (pow(0,0) = 1) */
static double multi_pow(const double* x, const int* a, int D) {
  double f = 1.0;
  for (int d = 0; d < D; ++d) f *= pow(x[d], (double)a[d]);
  return f;
}

/* alpha < p  <=>  every component < p  (Section 3.1) */
static int multi_lt(const int* a, int p, int D) {
  for (int d = 0; d < D; ++d)
    if (a[d] >= p) return 0;
  return 1;
}

/* alpha <= gamma componentwise */
static int multi_le(const int* a, const int* g, int D) {
  for (int d = 0; d < D; ++d)
    if (a[d] > g[d]) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Linear coefficient layout (Appendix, MultiIndexToPosition and its    */
/* inverse PositionToMultiindex)                                       */
/* ------------------------------------------------------------------ */

/* Radix-p number whose least significant digit is the last dimension.
 * MultiIndexToPosition walks d = D..1 multiplying the place value by p. */
int orc_multi_to_pos(const int* alpha, int p, int D) {
  int x = 0, f = 1;
  for (int d = D - 1; d >= 0; --d) {
    x += f * alpha[d];
    f *= p;
  }
  return x;
}

/* Reading: the printed PositionToMultiindex is garbled; this is the
 * inverse of MultiIndexToPosition (last dimension least significant). */
void orc_pos_to_multi(int i, int p, int D, int* alpha) {
  for (int d = D - 1; d >= 0; --d) {
    alpha[d] = i % p;
    i /= p;
  }
}

/* p_max by dimension (Section 3.6, query-tree initialisation): 6 for D=2,
 * 4 for D=3, 2 for D=4,5, 1 for D>=6.  Reading: D=1 is not listed; 8. */
int orc_pmax(int D) {
  if (D <= 1) return 8;
  if (D == 2) return 6;
  if (D == 3) return 4;
  if (D <= 5) return 2;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Hermite functions (Section 3.1)                                     */
/* ------------------------------------------------------------------ */

/* h_k(t) = e^{-t^2} H_k(t) for k < n by the recurrence
 * h_{k+1}(t) = 2t h_k(t) - 2k h_{k-1}(t), h_0 = e^{-t^2}, h_1 = 2t e^{-t^2}
 * (ComputePartialDerivatives, Appendix). */
void orc_hermite_functions(double t, int n, double* out) {
  if (n <= 0) return;
  out[0] = exp(-t * t);
  if (n > 1) out[1] = 2.0 * t * out[0];
  for (int k = 1; k + 1 < n; ++k) out[k + 1] = 2.0 * t * out[k] - 2.0 * (double)k * out[k - 1];
}

/* h_alpha(t) = prod_d h_{alpha[d]}(t[d])  (multivariate product form). */
static double hermite_multi(const double* t, const int* a, int D) {
  double f = 1.0;
  double tab[64];
  for (int d = 0; d < D; ++d) {
    orc_hermite_functions(t[d], a[d] + 1, tab);
    f *= tab[a[d]];
  }
  return f;
}

/* ------------------------------------------------------------------ */
/* Exact Gaussian sum, Eq. (5) / NaiveKDE (Algorithm 1) without the     */
/* normalisation                                                       */
/* ------------------------------------------------------------------ */

/* G(q_i) = sum_j exp(-||q_i - r_j||^2 / 2h^2) with direct differences and
 * a Neumaier-compensated sum.  Queries are independent, so they are
 * spread over host threads. */
void orc_naive_kde(const double* Q, int64_t nq, const double* R, int64_t nr, int D, double h,
                   double* G) {
  const double inv = 1.0 / (2.0 * h * h);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nq; ++i) {
    double s = 0.0, comp = 0.0;
    for (int64_t j = 0; j < nr; ++j) {
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) {
        double t = Q[i * D + d] - R[j * D + d];
        d2 += t * t;
      }
      double v = exp(-d2 * inv);
      double t = s + v;
      if (fabs(s) >= fabs(v))
        comp += (s - t) + v;
      else
        comp += (v - t) + s;
      s = t;
    }
    G[i] = s + comp;
  }
}

/* log G(q_i) for the same sum (Eq. 5), for sums that underflow double
 * precision: with x_j = ||q_i - r_j||^2 / 2h^2 and the per-query shift
 * m = min_j x_j,
 *     log G(q_i) = -m + log sum_j exp(-(x_j - m)),
 * the log-sum-exp form (every shifted term is <= 1 and the nearest one is
 * exactly 1, so the sum lies in [1, nr] and never underflows).  Direct
 * differences, Neumaier-compensated sum, log1p of the terms beyond the
 * first. */
void orc_log_naive_kde(const double* Q, int64_t nq, const double* R, int64_t nr, int D, double h,
                       double* logG) {
  const double inv = 1.0 / (2.0 * h * h);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < nq; ++i) {
    double m = INFINITY;
    for (int64_t j = 0; j < nr; ++j) {
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) {
        double t = Q[i * D + d] - R[j * D + d];
        d2 += t * t;
      }
      if (d2 * inv < m) m = d2 * inv;
    }
    /* sum of exp(-(x_j - m)) minus the one term equal to 1, so that
     * log(1 + rest) keeps full precision when the rest is small */
    double s = 0.0, comp = 0.0;
    int skipped = 0;
    for (int64_t j = 0; j < nr; ++j) {
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) {
        double t = Q[i * D + d] - R[j * D + d];
        d2 += t * t;
      }
      const double x = d2 * inv;
      if (!skipped && x == m) {
        skipped = 1;
        continue;
      }
      double v = exp(-(x - m));
      double t = s + v;
      if (fabs(s) >= fabs(v))
        comp += (s - t) + v;
      else
        comp += (v - t) + s;
      s = t;
    }
    logG[i] = -m + log1p(s + comp);
  }
}

/* Threads the OpenMP loops above use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Density estimate (Eq. 1) and the cross-validation scores of the      */
/* introduction (CV_LK, CV_LS), with the Gaussian kernel                */
/* ------------------------------------------------------------------ */

/* V_{D,h} = integral over R^D of exp(-||z||^2 / 2h^2) dz = (2 pi h^2)^{D/2},
 * the normalising constant of Eq. 1. */
double orc_gauss_volume(int D, double h) {
  const double pi = 3.14159265358979323846;
  return pow(2.0 * pi * h * h, 0.5 * D);
}

/* Leave-one-out sums over one point set (Q = R):
 * S_j = sum_{i != j} exp(-||x_j - x_i||^2 / 2h^2), Neumaier-compensated. */
void orc_loo_sums(const double* X, int64_t n, int D, double h, double* S) {
  const double inv = 1.0 / (2.0 * h * h);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0, comp = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (i == j) continue;
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) {
        const double t = X[j * D + d] - X[i * D + d];
        d2 += t * t;
      }
      const double v = exp(-d2 * inv);
      const double t = s + v;
      if (fabs(s) >= fabs(v))
        comp += (s - t) + v;
      else
        comp += (v - t) + s;
      s = t;
    }
    S[j] = s + comp;
  }
}

/* CV_LK(h) = (1/N) sum_j log p_{h,-j}(x_j) with the leave-one-out density
 * p_{h,-j}(x_j) = S_j / ((N - 1) V_{D,h}) (Eq. 1 over the N - 1 other
 * points); -inf when some S_j is 0. */
double orc_cv_lk(const double* X, int64_t n, int D, double h) {
  double* S = (double*)malloc(sizeof(double) * (size_t)n);
  orc_loo_sums(X, n, D, h, S);
  const double norm = (double)(n - 1) * orc_gauss_volume(D, h);
  double acc = 0.0;
  for (int64_t j = 0; j < n; ++j) acc += log(S[j] / norm);
  free(S);
  return acc / (double)n;
}

/* CV_LS(h) = (1/N) sum_j (p*_{-j}(x_j) - 2 p_{-j}(x_j)), p* the
 * leave-one-out estimate with the convolution kernel K_h * K_h.
 * Reading: the convolution of two Gaussians of standard deviation h is a
 * Gaussian of standard deviation sqrt(2) h (variance 2h^2, the "2h" of
 * the text), normalised by V_{D, sqrt(2) h}. */
double orc_cv_ls(const double* X, int64_t n, int D, double h) {
  double* S = (double*)malloc(sizeof(double) * (size_t)n);
  double* Ss = (double*)malloc(sizeof(double) * (size_t)n);
  const double hs = sqrt(2.0) * h;
  orc_loo_sums(X, n, D, h, S);
  orc_loo_sums(X, n, D, hs, Ss);
  const double norm = (double)(n - 1) * orc_gauss_volume(D, h);
  const double norm_s = (double)(n - 1) * orc_gauss_volume(D, hs);
  double acc = 0.0;
  for (int64_t j = 0; j < n; ++j) acc += Ss[j] / norm_s - 2.0 * S[j] / norm;
  free(S);
  free(Ss);
  return acc / (double)n;
}

/* Gradient of CV_LK(h) with respect to log h and to every point x_k.
 * With K_ij = exp(-|x_i - x_j|^2 / 2h^2) and S_i the leave-one-out sums,
 *   dCV/dlog h = (1/N) sum_i (1/S_i) sum_{j != i} K_ij |x_i - x_j|^2 / h^2 - D
 * (dK/dlog h = K |x_i - x_j|^2 / h^2, and log V_{D,h} grows by D per unit of
 * log h), and, since x_k enters S_k and every S_j with j != k,
 *   dCV/dx_k = -(1/(N h^2)) sum_{j != k} K_kj (x_k - x_j) (1/S_k + 1/S_j).
 * Plain double loops over all pairs; dx is [n][D]. */
void orc_cv_lk_grad(const double* X, int64_t n, int D, double h, double* dlogh, double* dx) {
  double* S = (double*)malloc(sizeof(double) * (size_t)n);
  orc_loo_sums(X, n, D, h, S);
  const double inv = 1.0 / (2.0 * h * h), h2 = h * h;
  double acc = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : acc)
  for (int64_t k = 0; k < n; ++k) {
    double a = 0.0;
    double g[64];
    for (int d = 0; d < D; ++d) g[d] = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == k) continue;
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) {
        const double t = X[k * D + d] - X[j * D + d];
        d2 += t * t;
      }
      const double K = exp(-d2 * inv);
      a += K * d2 / h2;
      const double w = K * (1.0 / S[k] + 1.0 / S[j]);
      for (int d = 0; d < D; ++d) g[d] += w * (X[k * D + d] - X[j * D + d]);
    }
    acc += a / S[k];
    for (int d = 0; d < D; ++d) dx[k * D + d] = -g[d] / ((double)n * h2);
  }
  *dlogh = acc / (double)n - (double)D;
  free(S);
}

/* ------------------------------------------------------------------ */
/* Expansions (Section 3.3) and translations (Section 3.5)             */
/* All tables have radix pm; only multi-indices below p are written.   */
/* ------------------------------------------------------------------ */

/* Far-field moments, Eq. (far_field_moments):
 * M_alpha(R,c) = sum_{r in R} (1/alpha!) ((r - c)/sqrt(2h^2))^alpha. */
void orc_farfield_moments(const double* R, int64_t nr, int D, const double* c, double h, int pm,
                          int p, double* M) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int a[ORC_MAXD];
  double x[ORC_MAXD];
  for (int i = 0; i < P; ++i) {
    M[i] = 0.0;
    orc_pos_to_multi(i, pm, D, a);
    if (!multi_lt(a, p, D)) continue;
    double acc = 0.0;
    for (int64_t j = 0; j < nr; ++j) {
      for (int d = 0; d < D; ++d) x[d] = (R[j * D + d] - c[d]) * s;
      acc += multi_pow(x, a, D);
    }
    M[i] = acc / multi_fact(a, D);
  }
}

/* Far-field evaluation (EvaluateFarFieldExpansion, Appendix):
 * sum_{alpha<p} M_alpha h_alpha((q - c)/sqrt(2h^2)). */
double orc_eval_farfield(const double* M, int D, int pm, int p, const double* c, double h,
                         const double* q) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int a[ORC_MAXD];
  double t[ORC_MAXD];
  for (int d = 0; d < D; ++d) t[d] = (q[d] - c[d]) * s;
  double w = 0.0;
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, a);
    if (!multi_lt(a, p, D)) continue;
    w += M[i] * hermite_multi(t, a, D);
  }
  return w;
}

/* Direct local moments, Eq. (local_moments):
 * L_beta += sum_{r in R} ((-1)^{|beta|}/beta!) h_beta((c - r)/sqrt(2h^2)),
 * beta < p.  Reading: the sign is (-1)^{|beta|} (Lemma 3.4 proof). */
void orc_direct_local(const double* R, int64_t nr, int D, const double* c, double h, int pm,
                      int p, double* L) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int b[ORC_MAXD];
  double t[ORC_MAXD];
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, b);
    if (!multi_lt(b, p, D)) continue;
    double acc = 0.0;
    for (int64_t j = 0; j < nr; ++j) {
      for (int d = 0; d < D; ++d) t[d] = (c[d] - R[j * D + d]) * s;
      acc += hermite_multi(t, b, D);
    }
    double sign = (multi_abs(b, D) & 1) ? -1.0 : 1.0;
    L[i] += sign / multi_fact(b, D) * acc;
  }
}

/* Far-to-local translation, Eq. (farfield_to_local_formula):
 * L_beta += ((-1)^{|beta|}/beta!) sum_{alpha<p} M_alpha h_{alpha+beta}((cQ - cR)/sqrt(2h^2)). */
void orc_far_to_local(const double* M, int D, int pm, int p, const double* cR, const double* cQ,
                      double h, double* L) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int a[ORC_MAXD], b[ORC_MAXD], ab[ORC_MAXD];
  double t[ORC_MAXD];
  for (int d = 0; d < D; ++d) t[d] = (cQ[d] - cR[d]) * s;
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, b);
    if (!multi_lt(b, p, D)) continue;
    double acc = 0.0;
    for (int j = 0; j < P; ++j) {
      orc_pos_to_multi(j, pm, D, a);
      if (!multi_lt(a, p, D)) continue;
      for (int d = 0; d < D; ++d) ab[d] = a[d] + b[d];
      acc += M[j] * hermite_multi(t, ab, D);
    }
    double sign = (multi_abs(b, D) & 1) ? -1.0 : 1.0;
    L[i] += sign / multi_fact(b, D) * acc;
  }
}

/* Far-to-far translation, Eq. (far_to_far_translation):
 * M_gamma(R, c') += sum_{0<=alpha<=gamma} M_alpha(R, R.c) ((R.c - c')/sqrt(2h^2))^{gamma-alpha} / (gamma-alpha)!,
 * gamma < p (the result is exact for gamma < p). */
void orc_far_to_far(const double* Mchild, int D, int pm, int p, const double* cchild,
                    const double* cnew, double h, double* Mnew) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int g[ORC_MAXD], a[ORC_MAXD], ga[ORC_MAXD];
  double x[ORC_MAXD];
  for (int d = 0; d < D; ++d) x[d] = (cchild[d] - cnew[d]) * s;
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, g);
    if (!multi_lt(g, p, D)) continue;
    double acc = 0.0;
    for (int j = 0; j < P; ++j) {
      orc_pos_to_multi(j, pm, D, a);
      if (!multi_le(a, g, D)) continue;
      for (int d = 0; d < D; ++d) ga[d] = g[d] - a[d];
      acc += Mchild[j] * multi_pow(x, ga, D) / multi_fact(ga, D);
    }
    Mnew[i] += acc;
  }
}

/* Local-to-local translation, Eq. (local_to_local_translation).
 * Reading: the left-hand side is indexed by alpha:
 * L_alpha(c') += sum_{alpha<=beta<p} beta!/(alpha!(beta-alpha)!) L_beta(Q.c) ((c' - Q.c)/sqrt(2h^2))^{beta-alpha}. */
void orc_local_to_local(const double* Lold, int D, int pm, int p, const double* cold,
                        const double* cnew, double h, double* Lnew) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int a[ORC_MAXD], b[ORC_MAXD], ba[ORC_MAXD];
  double x[ORC_MAXD];
  for (int d = 0; d < D; ++d) x[d] = (cnew[d] - cold[d]) * s;
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, a);
    if (!multi_lt(a, p, D)) continue;
    double acc = 0.0;
    for (int j = 0; j < P; ++j) {
      orc_pos_to_multi(j, pm, D, b);
      if (!multi_lt(b, p, D) || !multi_le(a, b, D)) continue;
      for (int d = 0; d < D; ++d) ba[d] = b[d] - a[d];
      double coef = multi_fact(b, D) / (multi_fact(a, D) * multi_fact(ba, D));
      acc += coef * Lold[j] * multi_pow(x, ba, D);
    }
    Lnew[i] += acc;
  }
}

/* Local expansion evaluation (EvaluateLocalExpansion, Appendix).
 * Reading: the loop runs over query points and accumulates
 * z += L_beta ((q - Q.c)/sqrt(2h^2))^beta. */
double orc_eval_local(const double* L, int D, int pm, int p, const double* c, double h,
                      const double* q) {
  const double s = 1.0 / sqrt(2.0 * h * h);
  const int P = ipow(pm, D);
  int b[ORC_MAXD];
  double x[ORC_MAXD];
  for (int d = 0; d < D; ++d) x[d] = (q[d] - c[d]) * s;
  double z = 0.0;
  for (int i = 0; i < P; ++i) {
    orc_pos_to_multi(i, pm, D, b);
    if (!multi_lt(b, p, D)) continue;
    z += L[i] * multi_pow(x, b, D);
  }
  return z;
}

/* ------------------------------------------------------------------ */
/* Truncation error bounds (Section 3.4)                               */
/* ------------------------------------------------------------------ */

/* Eq. (error_bound_far_field), also Eq. (error_bound_local):
 * |R|/(1-r)^D sum_{k=0}^{D-1} C(D,k) (1-r^p)^k (r^p/sqrt(p!))^{D-k}, r < 1. */
double orc_bound_farfield(double nR, int D, double r, int p) {
  double rp = pow(r, (double)p);
  double tail = rp / sqrt(fact(p));
  double sum = 0.0;
  for (int k = 0; k <= D - 1; ++k)
    sum += binom(D, k) * pow(1.0 - rp, (double)k) * pow(tail, (double)(D - k));
  return nR / pow(1.0 - r, (double)D) * sum;
}

double orc_bound_local(double nR, int D, double r, int p) { return orc_bound_farfield(nR, D, r, p); }

/* Eq. (error_bound_far_to_local):
 * |R|/(1-2r)^{2D} sum_{k=0}^{D-1} C(D,k) ((1-(2r)^p)^2)^k ((2r)^p (2-(2r)^p)/sqrt(p!))^{D-k}, r < 1/2. */
double orc_bound_f2l(double nR, int D, double r, int p) {
  double q = pow(2.0 * r, (double)p);
  double head = (1.0 - q) * (1.0 - q);
  double tail = q * (2.0 - q) / sqrt(fact(p));
  double sum = 0.0;
  for (int k = 0; k <= D - 1; ++k)
    sum += binom(D, k) * pow(head, (double)k) * pow(tail, (double)(D - k));
  return nR / pow(1.0 - 2.0 * r, (double)(2 * D)) * sum;
}

/* max_d (b[d].u - b[d].l) over a box */
static double max_side(const double* lo, const double* hi, int D) {
  double m = 0.0;
  for (int d = 0; d < D; ++d)
    if (hi[d] - lo[d] > m) m = hi[d] - lo[d];
  return m;
}

/* FarFieldOrder (Algorithm): r = max side of R / 2h; r >= 1 -> infinity;
 * least p <= p_max whose bound is <= tau, else infinity. */
int orc_order_farfield(const double* Rlo, const double* Rhi, double nR, int D, double h,
                       double tau, int pmax) {
  double r = max_side(Rlo, Rhi, D) / (2.0 * h);
  if (r >= 1.0) return ORC_INF_ORDER;
  for (int p = 1; p <= pmax; ++p)
    if (orc_bound_farfield(nR, D, r, p) <= tau) return p;
  return ORC_INF_ORDER;
}

/* LocalAccumulationOrder (Algorithm): same test with r from the query box. */
int orc_order_local(const double* Qlo, const double* Qhi, double nR, int D, double h, double tau,
                    int pmax) {
  double r = max_side(Qlo, Qhi, D) / (2.0 * h);
  if (r >= 1.0) return ORC_INF_ORDER;
  for (int p = 1; p <= pmax; ++p)
    if (orc_bound_local(nR, D, r, p) <= tau) return p;
  return ORC_INF_ORDER;
}

/* ConvertFarFieldToLocalOrder (Algorithm).  Reading: the lemma needs both
 * half-widths below r h with r < 1/2, so r = max over both boxes of
 * side / 2h (the printed side/4h would admit boxes the lemma excludes). */
int orc_order_f2l(const double* Qlo, const double* Qhi, const double* Rlo, const double* Rhi,
                  double nR, int D, double h, double tau, int pmax) {
  double sq = max_side(Qlo, Qhi, D), sr = max_side(Rlo, Rhi, D);
  double r = (sq > sr ? sq : sr) / (2.0 * h);
  if (r >= 0.5) return ORC_INF_ORDER;
  for (int p = 1; p <= pmax; ++p)
    if (orc_bound_f2l(nR, D, r, p) <= tau) return p;
  return ORC_INF_ORDER;
}

/* ------------------------------------------------------------------ */
/* Node-pair distance bounds, Eqs. (6)-(7)                             */
/* ------------------------------------------------------------------ */

void orc_dist_bounds(const double* Ql, const double* Qu, const double* Rl, const double* Ru, int D,
                     double* dl, double* du) {
  double sl = 0.0, su = 0.0;
  for (int k = 0; k < D; ++k) {
    double dlu_ji = Rl[k] - Qu[k]; /* d^{l,u}_{j,i} */
    double dlu_ij = Ql[k] - Ru[k]; /* d^{l,u}_{i,j} */
    double dul_ji = Ru[k] - Ql[k]; /* d^{u,l}_{j,i} */
    double dul_ij = Qu[k] - Rl[k]; /* d^{u,l}_{i,j} */
    double a = dlu_ji + fabs(dlu_ji) + dlu_ij + fabs(dlu_ij);
    sl += a * a;
    double m = dul_ji > dul_ij ? dul_ji : dul_ij;
    su += m * m;
  }
  *dl = 0.5 * sqrt(sl);
  *du = sqrt(su);
}

/* ------------------------------------------------------------------ */
/* ChooseBestMethod (Algorithm)                                        */
/* ------------------------------------------------------------------ */

enum { ORC_M_F = 0, ORC_M_D = 1, ORC_M_T = 2, ORC_M_E = 3 };

/* Reading: the printed costs N_Q D^{p+1} etc. disagree with the stated
 * complexities O(|Q| p^D), O(|R| p^D), O(D p^{2D}); the costs used are
 * c_F = D N_Q p_F^D, c_D = D N_R p_D^D, c_T = D p_T^{2D}, c_E = D N_Q N_R,
 * an infinite order gives an infinite cost, and ties go F, D, T, E in the
 * order of the if-chain.  Returns the method; *order receives its p. */
int orc_choose_best_method(const double* Qlo, const double* Qhi, double nQ, const double* Rlo,
                           const double* Rhi, double nR, int D, double h, double tau, int pmax,
                           int* order) {
  int pF = orc_order_farfield(Rlo, Rhi, nR, D, h, tau, pmax);
  int pD = orc_order_local(Qlo, Qhi, nR, D, h, tau, pmax);
  int pT = orc_order_f2l(Qlo, Qhi, Rlo, Rhi, nR, D, h, tau, pmax);
  double cF = pF == ORC_INF_ORDER ? INFINITY : D * nQ * pow((double)pF, (double)D);
  double cD = pD == ORC_INF_ORDER ? INFINITY : D * nR * pow((double)pD, (double)D);
  double cT = pT == ORC_INF_ORDER ? INFINITY : D * pow((double)pT, (double)(2 * D));
  double cE = D * nQ * nR;
  double m = cF;
  if (cD < m) m = cD;
  if (cT < m) m = cT;
  if (cE < m) m = cE;
  if (cF == m && pF != ORC_INF_ORDER) { *order = pF; return ORC_M_F; }
  if (cD == m && pD != ORC_INF_ORDER) { *order = pD; return ORC_M_D; }
  if (cT == m && pT != ORC_INF_ORDER) { *order = pT; return ORC_M_T; }
  *order = 0;
  return ORC_M_E;
}

/* ------------------------------------------------------------------ */
/* The dual-tree algorithm itself (Section 3.6): BuildKdTree, DFGTMain, */
/* DFGTInitQ, DFGTInitR, DFGT, DFGTBase, DFGTPost                       */
/* ------------------------------------------------------------------ */

typedef struct {
  double lo[ORC_MAXD], hi[ORC_MAXD], c[ORC_MAXD];
  int begin, count;
  int left, right;
  double* M;          /* far-field moments about c (reference tree) */
  double* L;          /* local moments about c (query tree) */
  int p_used;         /* highest order accumulated into L */
  double Gl, Gu, Dl, Du; /* G^l(Q), G^u(Q), Q.Delta^l, Q.Delta^u */
} onode;

typedef struct {
  onode* n;
  int nn, cap;
  int* idx;           /* point permutation: node points are idx[begin..begin+count) */
  const double* X;
  int D;
} otree;

static int tree_new_node(otree* t) {
  if (t->nn == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 64;
    t->n = (onode*)realloc(t->n, sizeof(onode) * (size_t)t->cap);
  }
  memset(&t->n[t->nn], 0, sizeof(onode));
  return t->nn++;
}

/* BuildKdTree (Algorithm 2): tight bounding box, split the widest
 * dimension at its midpoint while the node holds more points than the
 * leaf threshold.  Reading: a split that would leave one side empty (all
 * points coincide along the widest side, or the midpoint rounds onto the
 * upper bound) makes the node a leaf instead. */
static int build_kd(otree* t, int begin, int count, int leaf) {
  int id = tree_new_node(t);
  const int D = t->D;
  onode* N = &t->n[id];
  N->begin = begin;
  N->count = count;
  N->left = N->right = -1;
  for (int d = 0; d < D; ++d) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = begin; i < begin + count; ++i) {
      double x = t->X[(int64_t)t->idx[i] * D + d];
      if (x < lo) lo = x;
      if (x > hi) hi = x;
    }
    N->lo[d] = lo;
    N->hi[d] = hi;
    N->c[d] = 0.5 * (lo + hi);
  }
  if (count > leaf) {
    int sd = 0;
    for (int d = 1; d < D; ++d)
      if (N->hi[d] - N->lo[d] > N->hi[sd] - N->lo[sd]) sd = d;
    double sc = 0.5 * (N->lo[sd] + N->hi[sd]);
    /* stable partition: x[sd] <= sc to the left */
    int* tmp = (int*)malloc(sizeof(int) * (size_t)count);
    int nl = 0;
    for (int i = begin; i < begin + count; ++i)
      if (t->X[(int64_t)t->idx[i] * D + sd] <= sc) tmp[nl++] = t->idx[i];
    int nr = 0;
    for (int i = begin; i < begin + count; ++i)
      if (!(t->X[(int64_t)t->idx[i] * D + sd] <= sc)) tmp[nl + nr++] = t->idx[i];
    if (nl > 0 && nr > 0) {
      memcpy(t->idx + begin, tmp, sizeof(int) * (size_t)count);
      free(tmp);
      int l = build_kd(t, begin, nl, leaf);
      int r = build_kd(t, begin + nl, nr, leaf);
      t->n[id].left = l;
      t->n[id].right = r;
    } else {
      free(tmp);
    }
  }
  return id;
}

static void tree_init(otree* t, const double* X, int64_t n, int D, int leaf) {
  memset(t, 0, sizeof(*t));
  t->X = X;
  t->D = D;
  t->idx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) t->idx[i] = (int)i;
  build_kd(t, 0, (int)n, leaf);
}

static void tree_free(otree* t) {
  for (int i = 0; i < t->nn; ++i) {
    free(t->n[i].M);
    free(t->n[i].L);
  }
  free(t->n);
  free(t->idx);
}

/* State of one DFGTMain call. */
typedef struct {
  otree Qt, Rt;
  int D, pm, P;
  double h, eps, NR;
  double *Gl, *Gu;      /* per query point bounds */
  double *GE, *GF, *GL; /* exhaustive, far-field and local-expansion parts */
  double* acct;         /* optional: reference points accounted per query */
  long long stats[6];   /* prune, F, D, T, base-case pairs, DFGT calls */
} ostate;

static double Kh(double dist, double h) { return exp(-dist * dist / (2.0 * h * h)); }

/* DFGTInitR (Algorithm): leaf moments by AccumulateFarFieldMoment, internal
 * moments by translating both children's moments to the parent center. */
static void init_R(ostate* S, int id) {
  otree* t = &S->Rt;
  onode* N = &t->n[id];
  N->M = (double*)calloc((size_t)S->P, sizeof(double));
  if (N->left < 0) {
    double* pts = (double*)malloc(sizeof(double) * (size_t)N->count * (size_t)S->D);
    for (int i = 0; i < N->count; ++i)
      for (int d = 0; d < S->D; ++d)
        pts[i * S->D + d] = t->X[(int64_t)t->idx[N->begin + i] * S->D + d];
    orc_farfield_moments(pts, N->count, S->D, N->c, S->h, S->pm, S->pm, N->M);
    free(pts);
  } else {
    init_R(S, N->left);
    init_R(S, N->right);
    N = &t->n[id];
    orc_far_to_far(t->n[N->left].M, S->D, S->pm, S->pm, t->n[N->left].c, N->c, S->h, N->M);
    orc_far_to_far(t->n[N->right].M, S->D, S->pm, S->pm, t->n[N->right].c, N->c, S->h, N->M);
  }
}

/* DFGTInitQ (Algorithm): G^l = 0, G^u = |R|, Delta = 0, L = 0. */
static void init_Q(ostate* S) {
  for (int i = 0; i < S->Qt.nn; ++i) {
    onode* N = &S->Qt.n[i];
    N->Gl = 0.0;
    N->Gu = S->NR;
    N->Dl = N->Du = 0.0;
    N->L = (double*)calloc((size_t)S->P, sizeof(double));
    N->p_used = 0;
  }
}

static void account(ostate* S, const onode* Q, double nR) {
  if (!S->acct) return;
  for (int i = Q->begin; i < Q->begin + Q->count; ++i) S->acct[S->Qt.idx[i]] += nR;
}

/* DFGTBase (Algorithm): exhaustive leaf-leaf sum and bound refinement. */
static void dfgt_base(ostate* S, int qi, int ri) {
  onode* Q = &S->Qt.n[qi];
  const onode* R = &S->Rt.n[ri];
  const int D = S->D;
  Q->Gl = INFINITY;
  Q->Gu = -INFINITY;
  for (int a = Q->begin; a < Q->begin + Q->count; ++a) {
    int qidx = S->Qt.idx[a];
    const double* q = S->Qt.X + (int64_t)qidx * D;
    S->Gl[qidx] += Q->Dl;
    S->Gu[qidx] += Q->Du;
    for (int b = R->begin; b < R->begin + R->count; ++b) {
      const double* r = S->Rt.X + (int64_t)S->Rt.idx[b] * D;
      double d2 = 0.0;
      for (int d = 0; d < D; ++d) d2 += (q[d] - r[d]) * (q[d] - r[d]);
      double v = exp(-d2 / (2.0 * S->h * S->h));
      S->Gl[qidx] += v;
      S->GE[qidx] += v;
      S->Gu[qidx] += v - 1.0;
    }
    if (S->Gl[qidx] < Q->Gl) Q->Gl = S->Gl[qidx];
    if (S->Gu[qidx] > Q->Gu) Q->Gu = S->Gu[qidx];
  }
  Q->Dl = Q->Du = 0.0;
  account(S, Q, (double)R->count);
  S->stats[4]++;
}

/* Summarize (Algorithm) with the method chosen by ChooseBestMethod. */
static void summarize(ostate* S, int qi, int ri, int method, int p, double dl_, double du_) {
  onode* Q = &S->Qt.n[qi];
  const onode* R = &S->Rt.n[ri];
  const int D = S->D;
  if (method == ORC_M_F) {
    /* EvaluateFarFieldExpansion */
    for (int a = Q->begin; a < Q->begin + Q->count; ++a) {
      int qidx = S->Qt.idx[a];
      S->GF[qidx] += orc_eval_farfield(R->M, D, S->pm, p, R->c, S->h, S->Qt.X + (int64_t)qidx * D);
    }
    S->stats[1]++;
  } else if (method == ORC_M_D) {
    /* AccumulateDirectLocalMoment */
    double* pts = (double*)malloc(sizeof(double) * (size_t)R->count * (size_t)D);
    for (int i = 0; i < R->count; ++i)
      for (int d = 0; d < D; ++d) pts[i * D + d] = S->Rt.X[(int64_t)S->Rt.idx[R->begin + i] * D + d];
    orc_direct_local(pts, R->count, D, Q->c, S->h, S->pm, p, Q->L);
    free(pts);
    if (p > Q->p_used) Q->p_used = p;
    S->stats[2]++;
  } else if (method == ORC_M_T) {
    /* TransFarToLocal */
    orc_far_to_local(R->M, D, S->pm, p, R->c, Q->c, S->h, Q->L);
    if (p > Q->p_used) Q->p_used = p;
    S->stats[3]++;
  } else {
    /* Reading (finite-difference prune of the predecessor dual-tree
     * method): every query in Q receives |R|(K(d^l)+K(d^u))/2, error at
     * most |R|(K(d^l)-K(d^u))/2; it is stored as the constant term L_0. */
    Q->L[0] += 0.5 * (double)R->count * (Kh(dl_, S->h) + Kh(du_, S->h));
    if (Q->p_used < 1) Q->p_used = 1;
    S->stats[0]++;
  }
  account(S, Q, (double)R->count);
}

enum { ORC_PRUNE = 4 };

/* DFGT (Algorithm): the recursion over node pairs. */
static void dfgt(ostate* S, int qi, int ri) {
  onode* Q = &S->Qt.n[qi];
  const onode* R = &S->Rt.n[ri];
  const int D = S->D;
  S->stats[5]++;
  double dl_, du_;
  orc_dist_bounds(Q->lo, Q->hi, R->lo, R->hi, D, &dl_, &du_);
  double nR = (double)R->count, nQ = (double)Q->count;
  double delta_l = nR * Kh(du_, S->h);
  double delta_u = nR * (Kh(dl_, S->h) - 1.0);
  double Gl_new = Q->Gl + Q->Dl + delta_l;
  double tau = S->eps * nR * Gl_new / S->NR;
  /* CanSummarize: the finite-difference prune is tried first (reading),
   * then ChooseBestMethod with the same tau. */
  int method = ORC_M_E, p = 0;
  if (0.5 * nR * (Kh(dl_, S->h) - Kh(du_, S->h)) <= tau) {
    method = ORC_PRUNE;
  } else {
    method = orc_choose_best_method(Q->lo, Q->hi, nQ, R->lo, R->hi, nR, D, S->h, tau, S->pm, &p);
  }
  if (method != ORC_M_E) {
    Q->Dl += delta_l;
    Q->Du += delta_u;
    summarize(S, qi, ri, method, p, dl_, du_);
    return;
  }
  if (Q->left < 0) {
    if (R->left < 0) {
      dfgt_base(S, qi, ri);
    } else {
      int rl = R->left, rr = R->right;
      dfgt(S, qi, rl);
      dfgt(S, qi, rr);
    }
    return;
  }
  /* push postponed bound changes to the children */
  onode* QL = &S->Qt.n[Q->left];
  onode* QR = &S->Qt.n[Q->right];
  QL->Dl += Q->Dl;
  QR->Dl += Q->Dl;
  QL->Du += Q->Du;
  QR->Du += Q->Du;
  Q->Dl = Q->Du = 0.0;
  int ql = Q->left, qr = Q->right;
  if (R->left < 0) {
    dfgt(S, ql, ri);
    dfgt(S, qr, ri);
  } else {
    int rl = R->left, rr = R->right;
    dfgt(S, ql, rl);
    dfgt(S, ql, rr);
    dfgt(S, qr, rl);
    dfgt(S, qr, rr);
  }
  Q = &S->Qt.n[qi];
  QL = &S->Qt.n[ql];
  QR = &S->Qt.n[qr];
  double a = QL->Gl + QL->Dl, b = QR->Gl + QR->Dl;
  Q->Gl = a < b ? a : b;
  double c = QL->Gu + QL->Du, d = QR->Gu + QR->Du;
  Q->Gu = c > d ? c : d;
}

/* DFGTPost (Algorithm): local-to-local translation to the children,
 * push-down of the postponed bounds, leaf evaluation and the final sum
 * G~ = G~_{D u T} + G~_F + G~_E. */
static void dfgt_post(ostate* S, int qi) {
  onode* Q = &S->Qt.n[qi];
  const int D = S->D;
  if (Q->left < 0) {
    Q->Gl = INFINITY;
    Q->Gu = -INFINITY;
    for (int a = Q->begin; a < Q->begin + Q->count; ++a) {
      int qidx = S->Qt.idx[a];
      S->Gl[qidx] += Q->Dl;
      S->Gu[qidx] += Q->Du;
      if (S->Gl[qidx] < Q->Gl) Q->Gl = S->Gl[qidx];
      if (S->Gu[qidx] > Q->Gu) Q->Gu = S->Gu[qidx];
      if (Q->p_used > 0)
        S->GL[qidx] += orc_eval_local(Q->L, D, S->pm, Q->p_used, Q->c, S->h, S->Qt.X + (int64_t)qidx * D);
    }
    Q->Dl = Q->Du = 0.0;
    return;
  }
  int l = Q->left, r = Q->right;
  onode* QL = &S->Qt.n[l];
  onode* QR = &S->Qt.n[r];
  if (Q->p_used > 0) {
    orc_local_to_local(Q->L, D, S->pm, Q->p_used, Q->c, QL->c, S->h, QL->L);
    orc_local_to_local(Q->L, D, S->pm, Q->p_used, Q->c, QR->c, S->h, QR->L);
    if (QL->p_used < Q->p_used) QL->p_used = Q->p_used;
    if (QR->p_used < Q->p_used) QR->p_used = Q->p_used;
  }
  QL->Dl += Q->Dl;
  QR->Dl += Q->Dl;
  QL->Du += Q->Du;
  QR->Du += Q->Du;
  memset(Q->L, 0, sizeof(double) * (size_t)S->P);
  Q->Dl = Q->Du = 0.0;
  dfgt_post(S, l);
  dfgt_post(S, r);
  Q = &S->Qt.n[qi];
  Q->Gl = S->Qt.n[l].Gl < S->Qt.n[r].Gl ? S->Qt.n[l].Gl : S->Qt.n[r].Gl;
  Q->Gu = S->Qt.n[l].Gu > S->Qt.n[r].Gu ? S->Qt.n[l].Gu : S->Qt.n[r].Gu;
}

/* DFGTMain (Algorithm): build both trees, initialise, traverse, post-process.
 *   G      [nq] approximate sums G~(q_i)            (required)
 *   Gl, Gu [nq] final per-query bounds              (nullable)
 *   acct   [nq] reference points accounted per query (nullable; Theorem 3.2)
 *   stats  [6]  prune, F, D, T, base pairs, DFGT calls (nullable)
 * Returns 0, or -1 for invalid arguments. */
int orc_dfgt(const double* Qp, int64_t nq, const double* Rp, int64_t nr, int D, double h,
             double eps, int leaf, int pmax, double* G, double* Gl_out, double* Gu_out, double* acct,
             long long* stats) {
  if (nq <= 0 || nr <= 0 || D < 1 || D > ORC_MAXD || !(h > 0) || !(eps > 0) || leaf < 1) return -1;
  if (pmax <= 0) pmax = orc_pmax(D);
  ostate S;
  memset(&S, 0, sizeof(S));
  S.D = D;
  S.pm = pmax;
  S.P = ipow(pmax, D);
  S.h = h;
  S.eps = eps;
  S.NR = (double)nr;
  tree_init(&S.Qt, Qp, nq, D, leaf);
  tree_init(&S.Rt, Rp, nr, D, leaf);
  S.Gl = (double*)calloc((size_t)nq, sizeof(double));
  S.Gu = (double*)malloc(sizeof(double) * (size_t)nq);
  for (int64_t i = 0; i < nq; ++i) S.Gu[i] = S.NR;
  S.GE = (double*)calloc((size_t)nq, sizeof(double));
  S.GF = (double*)calloc((size_t)nq, sizeof(double));
  S.GL = (double*)calloc((size_t)nq, sizeof(double));
  S.acct = acct;
  if (acct) memset(acct, 0, sizeof(double) * (size_t)nq);
  init_Q(&S);
  init_R(&S, 0);
  dfgt(&S, 0, 0);
  dfgt_post(&S, 0);
  for (int64_t i = 0; i < nq; ++i) G[i] = S.GL[i] + S.GF[i] + S.GE[i];
  if (Gl_out) memcpy(Gl_out, S.Gl, sizeof(double) * (size_t)nq);
  if (Gu_out) memcpy(Gu_out, S.Gu, sizeof(double) * (size_t)nq);
  if (stats) memcpy(stats, S.stats, sizeof(S.stats));
  free(S.Gl);
  free(S.Gu);
  free(S.GE);
  free(S.GF);
  free(S.GL);
  tree_free(&S.Qt);
  tree_free(&S.Rt);
  return 0;
}
