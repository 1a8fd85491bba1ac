/*
 * CPU FP64 oracle for the metric-magnitude hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never does.
 * It shares no code, header, table or constant with the CUDA sources.
 *
 * Everything is IEEE double with libm sqrt/exp, straight loops, no blocking.
 * Paper: "Scalably computing metric magnitude" (arXiv 2607.23354).
 *   Sec. 2: Z = exp[-t d] with d_jk = ||x_j - x_k|| (Euclidean in R^m); a
 *           weighting is the solution of Zw = 1 (Eq. weighting); the magnitude
 *           is Mag(Z) = 1^T w; Z is positive definite for Euclidean d, so a
 *           Cholesky factor exists (Sec. 3.2) and w is unique.
 *   Sec. 1/2: t_+ is the least t with w >= 0, bounded above by
 *           log(n-1) / min_{j != k} d_jk, and found by root-finding on
 *           min_j w_j (bisection; Appendix A calls it binary search).
 *   Gradients are not in the paper; they follow from implicit
 *   differentiation of Zw = 1 (dw = -Z^{-1} dZ w), see orc_grad below.
 *
 * Parity status of each function (what pins it) is listed beside it; every
 * function here is pinned by a CPU test against closed forms, invariants,
 * values printed in the paper or library routines.
 *
 * OpenMP (if compiled with -fopenmp) only splits independent rows across
 * threads; it changes no arithmetic order inside a row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EDUPLICATE 2
#define ORC_ENOTPD 3
#define ORC_ENOBRACKET 5
#define ORC_ENOMEM 6

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- compensated summation (Neumaier's variant of Kahan summation) ---- */
typedef struct { double s, c; } orc_acc;

static void acc_add(orc_acc* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}
static double acc_value(const orc_acc* a) { return a->s + a->c; }

double orc_sum(const double* v, int64_t n) {
  orc_acc a = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) acc_add(&a, v[i]);
  return acc_value(&a);
}

/* ---- Sec. 2: Euclidean distance from coordinate differences ----
 * d_jk = sqrt(sum_l (x_jl - x_kl)^2), l ascending.  Pinned by Pythagorean
 * triples (exact integers) and by scipy's pdist. */
double orc_distance(const double* X, int64_t m, int64_t j, int64_t k) {
  double s = 0.0;
  for (int64_t l = 0; l < m; ++l) {
    double diff = X[j * m + l] - X[k * m + l];
    s += diff * diff;
  }
  return sqrt(s);
}

/* Full n x n distance matrix, row-major. */
void orc_distance_matrix(const double* X, int64_t n, int64_t m, double* D) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = 0; k < n; ++k) D[j * n + k] = orc_distance(X, m, j, k);
}

/* Sec. 2: Z_jk = exp(-t d_jk), so Z_jj = exp(0) = 1.  Full n x n, row-major. */
void orc_similarity_matrix(const double* X, int64_t n, int64_t m, double t, double* Z) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = 0; k < n; ++k) Z[j * n + k] = exp(-t * orc_distance(X, m, j, k));
}

/* min_{j != k} d_jk over all pairs (Sec. 1 bound).  Pinned by scipy pdist. */
double orc_min_distance(const double* X, int64_t n, int64_t m) {
  double best = INFINITY;
#pragma omp parallel for schedule(dynamic, 16) reduction(min : best)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = j + 1; k < n; ++k) {
      double d = orc_distance(X, m, j, k);
      if (d < best) best = d;
    }
  return best;
}

/* Sec. 1: the elementary bound t_+ <= log(n-1) / min_{j != k} d_jk. */
double orc_tplus_bound(const double* X, int64_t n, int64_t m) {
  return log((double)(n - 1)) / orc_min_distance(X, n, m);
}

/* ---- Sec. 3.2: Cholesky factorization A = L L^T (A positive definite) ----
 * Column-by-column (left-looking, "dot product" form):
 *   L_jj = sqrt(A_jj - sum_{k<j} L_jk^2)
 *   L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj      for i > j.
 * In place on the lower triangle of a row-major n x n array; the strict upper
 * triangle is set to zero on exit.  Returns 0, or j+1 if pivot j is not
 * positive (the PD check of Sec. 4.2).  Pinned against numpy's cholesky and
 * by reconstruction L L^T = A. */
int orc_cholesky(double* A, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    double* Aj = A + j * n;
    double s = Aj[j];
    for (int64_t k = 0; k < j; ++k) s -= Aj[k] * Aj[k];
    if (!(s > 0.0)) return (int)(j + 1);
    double ljj = sqrt(s);
    Aj[j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double* Ai = A + i * n;
      double v = Ai[j];
      for (int64_t k = 0; k < j; ++k) v -= Ai[k] * Aj[k];
      Ai[j] = v / ljj;
    }
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
  return 0;
}

/* Forward substitution L y = b (row form) and back substitution L^T x = y
 * (column-sweep form, reading rows of L).  x may alias y. */
void orc_forward(const double* L, int64_t n, const double* b, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
}

void orc_backward(const double* L, int64_t n, const double* y, double* x) {
  if (x != y) memcpy(x, y, (size_t)n * sizeof(double));
  for (int64_t i = n - 1; i >= 0; --i) {
    x[i] /= L[i * n + i];
    for (int64_t k = 0; k < i; ++k) x[k] -= L[i * n + k] * x[i];
  }
}

/* ---- residual of Zw = b with Z regenerated from the points ----
 * r_j = b_j - sum_k Z_jk w_k for the listed rows (all rows when rows == NULL),
 * each row sum compensated.  Also returns rowsum_j = sum_k Z_jk (so that
 * ||Z||_inf = max_j rowsum_j, all entries being positive).  b == NULL means
 * the all-ones right-hand side of Eq. weighting. */
void orc_residual_rows(const double* X, int64_t n, int64_t m, double t, const double* w,
                       const double* b, const int64_t* rows, int64_t nrows, double* r,
                       double* rowsum) {
  int64_t cnt = rows ? nrows : n;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < cnt; ++q) {
    int64_t j = rows ? rows[q] : q;
    orc_acc zw = {0.0, 0.0}, zs = {0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
      double z = exp(-t * orc_distance(X, m, j, k));
      acc_add(&zw, z * w[k]);
      acc_add(&zs, z);
    }
    double bj = b ? b[j] : 1.0;
    r[q] = (bj - zw.s) - zw.c;
    if (rowsum) rowsum[q] = acc_value(&zs);
  }
}

static double max_abs(const double* v, int64_t n) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i)
    if (fabs(v[i]) > m) m = fabs(v[i]);
  return m;
}

/* Relative residual ||b - Zw||_inf / (||Z||_inf ||w||_inf), the accuracy
 * measure for "numerically exact" solutions. */
double orc_relative_residual(const double* X, int64_t n, int64_t m, double t, const double* w,
                             const double* b) {
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* rs = (double*)malloc((size_t)n * sizeof(double));
  if (!r || !rs) { free(r); free(rs); return NAN; }
  orc_residual_rows(X, n, m, t, w, b, NULL, n, r, rs);
  double rel = max_abs(r, n) / (max_abs(rs, n) * max_abs(w, n));
  free(r);
  free(rs);
  return rel;
}

/* ---- Eq. weighting for a general right-hand side: solve Z x = b ----
 * Z built in full, Cholesky, forward/back substitution, then `ir_steps`
 * steps of FP64 iterative refinement (r = b - Zx with compensated sums,
 * x += solve(r)).  b == NULL means b = 1 (the weighting).
 * info (nullable, 3 doubles): relative residual, ||Z||_inf, ||x||_inf. */
int orc_solve(const double* X, int64_t n, int64_t m, double t, const double* b, int ir_steps,
              double* x, double* info) {
  if (n < 1 || m < 1 || !(t > 0.0) || !isfinite(t)) return ORC_EINVAL;
  double* L = (double*)malloc((size_t)n * (size_t)n * sizeof(double));
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* rs = (double*)malloc((size_t)n * sizeof(double));
  if (!L || !r || !rs) { free(L); free(r); free(rs); return ORC_ENOMEM; }
  orc_similarity_matrix(X, n, m, t, L);
  int st = orc_cholesky(L, n);
  if (st) { free(L); free(r); free(rs); return ORC_ENOTPD; }
  for (int64_t i = 0; i < n; ++i) r[i] = b ? b[i] : 1.0;
  orc_forward(L, n, r, x);
  orc_backward(L, n, x, x);
  for (int it = 0; it < ir_steps; ++it) {
    orc_residual_rows(X, n, m, t, x, b, NULL, n, r, rs);
    orc_forward(L, n, r, r);
    orc_backward(L, n, r, r);
    for (int64_t i = 0; i < n; ++i) x[i] += r[i];
  }
  if (info) {
    orc_residual_rows(X, n, m, t, x, b, NULL, n, r, rs);
    double zn = max_abs(rs, n), xn = max_abs(x, n);
    info[0] = max_abs(r, n) / (zn * xn);
    info[1] = zn;
    info[2] = xn;
  }
  free(L);
  free(r);
  free(rs);
  return ORC_OK;
}

/* Sec. 2: the weighting w (Zw = 1) and the magnitude Mag = 1^T w.
 * out (nullable, 4 doubles): Mag, relative residual, min_j w_j, max_j |w_j|. */
int orc_weighting(const double* X, int64_t n, int64_t m, double t, int ir_steps, double* w,
                  double* out) {
  double info[3];
  int st = orc_solve(X, n, m, t, NULL, ir_steps, w, info);
  if (st) return st;
  if (out) {
    double mn = INFINITY;
    for (int64_t i = 0; i < n; ++i)
      if (w[i] < mn) mn = w[i];
    out[0] = orc_sum(w, n);
    out[1] = info[0];
    out[2] = mn;
    out[3] = info[2];
  }
  return ORC_OK;
}

/* ---- App. C, Eq. scaleZero: the weighting at scale zero ----
 * lim_{t -> 0} Z(t)^{-1} 1 = d^{-1} 1 / (1^T d^{-1} 1).  d (zero diagonal,
 * conditionally negative definite for Euclidean points) is indefinite, so the
 * plain definition is a general solve: d built in full, Gaussian elimination
 * with partial pivoting, `ir_steps` FP64 refinement steps (r = 1 - d v with
 * compensated row sums), then s = 1^T v (compensated) and w0 = v / s.
 * out (nullable, 3 doubles): s = 1^T d^{-1} 1, relative residual
 * ||1 - d v||_inf / (||d||_inf ||v||_inf), ||d||_inf. */
static void orc_dist_residual(const double* X, int64_t n, int64_t m, const double* v, double* r,
                              double* rowsum) {
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t j = 0; j < n; ++j) {
    orc_acc dv = {0.0, 0.0}, ds = {0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
      const double d = orc_distance(X, m, j, k);
      acc_add(&dv, d * v[k]);
      acc_add(&ds, d);
    }
    r[j] = (1.0 - dv.s) - dv.c;
    if (rowsum) rowsum[j] = acc_value(&ds);
  }
}

/* LU with partial pivoting of the n x n row-major A in place; piv[k] = row
 * swapped with k.  Returns 1 + the first zero pivot, or 0. */
static int64_t orc_lu(double* A, int64_t n, int64_t* piv) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
    piv[k] = p;
    if (A[p * n + k] == 0.0) return k + 1;
    if (p != k)
      for (int64_t j = 0; j < n; ++j) {
        double tmp = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = tmp;
      }
#pragma omp parallel for schedule(static)
    for (int64_t i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return 0;
}

static void orc_lu_solve(const double* A, int64_t n, const int64_t* piv, double* x) {
  for (int64_t k = 0; k < n; ++k) {
    double tmp = x[k];
    x[k] = x[piv[k]];
    x[piv[k]] = tmp;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k < i; ++k) x[i] -= A[i * n + k] * x[k];
  for (int64_t i = n - 1; i >= 0; --i) {
    for (int64_t k = i + 1; k < n; ++k) x[i] -= A[i * n + k] * x[k];
    x[i] /= A[i * n + i];
  }
}

int orc_scale_zero(const double* X, int64_t n, int64_t m, int ir_steps, double* w0, double* out3) {
  if (n < 2 || m < 1) return ORC_EINVAL;
  double* A = (double*)malloc((size_t)n * n * sizeof(double));
  int64_t* piv = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  double* v = (double*)malloc((size_t)n * sizeof(double));
  double* r = (double*)malloc((size_t)n * sizeof(double));
  double* rs = (double*)malloc((size_t)n * sizeof(double));
  if (!A || !piv || !v || !r || !rs) {
    free(A); free(piv); free(v); free(r); free(rs);
    return ORC_ENOMEM;
  }
  orc_distance_matrix(X, n, m, A);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t k = 0; k < n; ++k)
      if (j != k && A[j * n + k] == 0.0) {
        free(A); free(piv); free(v); free(r); free(rs);
        return ORC_EDUPLICATE;
      }
  if (orc_lu(A, n, piv)) {
    free(A); free(piv); free(v); free(r); free(rs);
    return ORC_ENOTPD;
  }
  for (int64_t j = 0; j < n; ++j) v[j] = 1.0;
  orc_lu_solve(A, n, piv, v);
  for (int step = 0; step < ir_steps; ++step) {
    orc_dist_residual(X, n, m, v, r, NULL);
    orc_lu_solve(A, n, piv, r);
    for (int64_t j = 0; j < n; ++j) v[j] += r[j];
  }
  orc_dist_residual(X, n, m, v, r, rs);
  orc_acc sum = {0.0, 0.0};
  for (int64_t j = 0; j < n; ++j) acc_add(&sum, v[j]);
  const double sv = acc_value(&sum);
  for (int64_t j = 0; j < n; ++j) w0[j] = v[j] / sv;
  if (out3) {
    out3[0] = sv;
    out3[1] = max_abs(r, n) / (max_abs(rs, n) * max_abs(v, n));
    out3[2] = max_abs(rs, n);
  }
  free(A); free(piv); free(v); free(r); free(rs);
  return ORC_OK;
}

/* ---- Sec. 2 cutoff t_+ by bisection on the sign of min_j w_j ----
 * feasible(t) <=> min_j w_j(t) >= 0.  t_hi <= 0 means the Sec. 1 bound.
 * Invariant: feasible(hi) and not feasible(lo); midpoint lo + (hi - lo)/2;
 * stop when hi - lo <= rel_tol * hi; t_+ is the feasible end hi.
 * If feasible(t_lo) already holds, t_+ = t_lo with *below = 1.
 * If the upper end is not feasible, ORC_ENOBRACKET.
 * out (nullable): t_plus, lo, hi;  probes: number of solves;  w, mag at t_+. */
int orc_tplus(const double* X, int64_t n, int64_t m, double t_lo, double t_hi, double rel_tol,
              int ir_steps, double* out3, int* below, int* probes, double* w, double* mag) {
  if (n < 2) return ORC_EINVAL;
  double dmin = orc_min_distance(X, n, m);
  if (!(dmin > 0.0)) return ORC_EDUPLICATE;
  if (t_hi <= 0.0) t_hi = log((double)(n - 1)) / dmin;
  if (!(t_lo > 0.0) || !(t_hi > t_lo)) return ORC_EINVAL;
  double* wt = (double*)malloc((size_t)n * sizeof(double));
  if (!wt) return ORC_ENOMEM;
  double o[4];
  int np = 0, st;
  *below = 0;
  st = orc_weighting(X, n, m, t_hi, ir_steps, w, o);
  ++np;
  if (st) { free(wt); return st; }
  if (!(o[2] >= 0.0)) { free(wt); *probes = np; return ORC_ENOBRACKET; }
  *mag = o[0];
  st = orc_weighting(X, n, m, t_lo, ir_steps, wt, o);
  ++np;
  if (st) { free(wt); return st; }
  double lo = t_lo, hi = t_hi;
  if (o[2] >= 0.0) {
    *below = 1;
    hi = t_lo;
    memcpy(w, wt, (size_t)n * sizeof(double));
    *mag = o[0];
  } else {
    while (hi - lo > rel_tol * hi) {
      double mid = lo + (hi - lo) / 2.0;
      st = orc_weighting(X, n, m, mid, ir_steps, wt, o);
      ++np;
      if (st) { free(wt); return st; }
      if (o[2] >= 0.0) {
        hi = mid;
        memcpy(w, wt, (size_t)n * sizeof(double));
        *mag = o[0];
      } else {
        lo = mid;
      }
    }
  }
  if (out3) { out3[0] = hi; out3[1] = lo; out3[2] = hi; }
  *probes = np;
  free(wt);
  return ORC_OK;
}

/* ---- Sec. 2 cutoff t_+ by Ridders' method (the root-finder the paper
 * prefers for its fewer evaluations; Ridders, IEEE Trans. Circuits Syst. 26
 * (1979)) on f(t) = min_j w_j(t), with the bracket kept on feasibility as in
 * orc_tplus: feasible(hi) (f >= 0), not feasible(lo) (f < 0), stop when
 * hi - lo <= rel_tol * hi, t_+ = hi.  One iteration, with f1 = f(lo),
 * f2 = f(hi) at its start:
 *   1. x3 = lo + (hi - lo)/2, f3 = f(x3); the bracket end of x3's class
 *      moves to x3;
 *   2. Ridders' point x4 = x3 + (x3 - x1) sign(f1 - f2) f3 / sqrt(f3^2 - f1 f2)
 *      (x1 = the old lo); if it lies strictly inside the current bracket,
 *      f4 = f(x4) and the end of x4's class moves to x4;
 *   3. once two successive x4 agree to within delta = rel_tol * hi / 2, one
 *      more evaluation at x4 -/+ delta (toward the other end) closes the
 *      bracket around the converged estimate.
 * Same outputs and errors as orc_tplus. */
int orc_tplus_ridders(const double* X, int64_t n, int64_t m, double t_lo, double t_hi, double rel_tol,
                      int ir_steps, double* out3, int* below, int* probes, double* w, double* mag) {
  if (n < 2) return ORC_EINVAL;
  double dmin = orc_min_distance(X, n, m);
  if (!(dmin > 0.0)) return ORC_EDUPLICATE;
  if (t_hi <= 0.0) t_hi = log((double)(n - 1)) / dmin;
  if (!(t_lo > 0.0) || !(t_hi > t_lo)) return ORC_EINVAL;
  double* wt = (double*)malloc((size_t)n * sizeof(double));
  if (!wt) return ORC_ENOMEM;
  double o[4];
  int np = 0, st;
  *below = 0;
  st = orc_weighting(X, n, m, t_hi, ir_steps, w, o);
  ++np;
  if (st) { free(wt); return st; }
  if (!(o[2] >= 0.0)) { free(wt); *probes = np; return ORC_ENOBRACKET; }
  *mag = o[0];
  double fhi = o[2];
  st = orc_weighting(X, n, m, t_lo, ir_steps, wt, o);
  ++np;
  if (st) { free(wt); return st; }
  double lo = t_lo, hi = t_hi, flo = o[2];
  /* evaluate f at t and move the bracket end of t's class there */
#define ORC_PROBE(tt, fout)                                     \
  do {                                                          \
    st = orc_weighting(X, n, m, (tt), ir_steps, wt, o);         \
    ++np;                                                       \
    if (st) { free(wt); return st; }                            \
    (fout) = o[2];                                              \
    if (o[2] >= 0.0) {                                          \
      hi = (tt); fhi = o[2];                                    \
      memcpy(w, wt, (size_t)n * sizeof(double));                \
      *mag = o[0];                                              \
    } else {                                                    \
      lo = (tt); flo = o[2];                                    \
    }                                                           \
  } while (0)
  if (flo >= 0.0) {
    *below = 1;
    hi = t_lo;
    memcpy(w, wt, (size_t)n * sizeof(double));
    *mag = o[0];
  } else {
    double prev_x4 = NAN;
    while (hi - lo > rel_tol * hi) {
      const double x1 = lo, f1 = flo, f2 = fhi;
      const double x3 = lo + (hi - lo) / 2.0;
      double f3, f4;
      ORC_PROBE(x3, f3);
      if (hi - lo <= rel_tol * hi) break;
      const double sq = sqrt(f3 * f3 - f1 * f2);
      if (!(sq > 0.0)) continue;
      const double x4 = x3 + (x3 - x1) * (f1 >= f2 ? 1.0 : -1.0) * f3 / sq;
      if (!(x4 > lo && x4 < hi)) { prev_x4 = NAN; continue; }
      ORC_PROBE(x4, f4);
      (void)f4;
      if (hi - lo <= rel_tol * hi) break;
      const double delta = 0.5 * rel_tol * hi;
      if (fabs(x4 - prev_x4) <= delta) {
        const double xc = (hi == x4) ? x4 - delta : x4 + delta;
        if (xc > lo && xc < hi) {
          double fc;
          ORC_PROBE(xc, fc);
          (void)fc;
        }
      }
      prev_x4 = x4;
    }
  }
#undef ORC_PROBE
  if (out3) { out3[0] = hi; out3[1] = lo; out3[2] = hi; }
  *probes = np;
  free(wt);
  return ORC_OK;
}

/* ---- gradients by implicit differentiation of Zw = 1 ----
 * For a loss L(w) with g = dL/dw and lambda = Z^{-1} g:
 *   dL = -lambda^T (dZ) w,
 *   dZ_jk/dt = -d_jk Z_jk                      =>  dL/dt = lambda^T (d o Z) w
 *   dZ_jk/dx_i = -t Z_jk u_jk (delta_ij - delta_ik),  u_jk = (x_j - x_k)/d_jk
 *                                              =>  dL/dx_i = t sum_{k != i} Z_ik u_ik (lambda_i w_k + lambda_k w_i).
 * For L = Mag (g = 1) lambda = w, giving dM/dt = w^T (d o Z) w and
 * dM/dx_i = 2 t w_i sum_k w_k Z_ik u_ik.  Pinned by closed forms (two points,
 * points on a line), translation/rotation/Euler identities and central
 * finite differences.  dL_dx is n x m row-major. */
void orc_grad(const double* X, int64_t n, int64_t m, double t, const double* w,
              const double* lambda, double* dL_dt, double* dL_dx) {
  double* rowt = (double*)malloc((size_t)n * sizeof(double));
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < n; ++i) {
    orc_acc at = {0.0, 0.0};
    double* gi = dL_dx + i * m;
    for (int64_t l = 0; l < m; ++l) gi[l] = 0.0;
    /* per-coordinate compensated accumulators would need m of them; a plain
       sum per coordinate is enough for the tolerances this is checked at, the
       t-derivative uses a compensated sum. */
    for (int64_t k = 0; k < n; ++k) {
      if (k == i) continue;
      double d = orc_distance(X, m, i, k);
      double z = exp(-t * d);
      acc_add(&at, lambda[i] * d * z * w[k]);
      double c = t * z * (lambda[i] * w[k] + lambda[k] * w[i]) / d;
      for (int64_t l = 0; l < m; ++l) gi[l] += c * (X[i * m + l] - X[k * m + l]);
    }
    rowt[i] = acc_value(&at);
  }
  *dL_dt = orc_sum(rowt, n);
  free(rowt);
}
