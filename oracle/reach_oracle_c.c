/*
 * reach_oracle_c.c -- the oracle's Jacobi (§3.1) and BiCGStab (§3.2) loops in plain C,
 * FP64, optionally spread over host cores with OpenMP.
 *
 * TEST INFRASTRUCTURE, not part of the product: it serves as the timed CPU baseline
 * (the paper compares its CUDA code with sequential C, §1 and §6) and is checked against
 * the numpy oracle and the closed forms by the CPU tests.  It shares no code with the CUDA
 * library and is never called by it.
 *
 * The system is M x = b with M in compressed row storage (§4), diagonal entries stored
 * (M = I - A of §2.3, as the numpy oracle's system_matrix builds it).  The steps follow the
 * numpy oracle (oracle/reach_oracle.py) one for one:
 *   Jacobi:   x_i <- (b_i - sum_{j != i} M_ij x'_j) / M_ii, x' the previous iterate (a
 *             second buffer), columns in stored (ascending) order, stop when
 *             max_i |x_i - x'_i| < eps, at most max_iter sweeps.
 *   BiCGStab: unpreconditioned, x = x0, r = b - M x, shadow q = r, y = a = w = 1,
 *             v = p = 0; per iteration y = q.r, p = r + (y a)/(y' w)(p - w v), v = M p,
 *             a = y / q.v, s = r - a v; stop with x += a p when max|s| < eps; else
 *             t = M s, w = t.s / t.t, x += a p + w s, r = s - w t; stop when max|r| < eps.
 *             A breakdown (q.r = 0, q.v = 0 or w = 0) restarts once as the numpy oracle.
 * Rows are independent in a Jacobi sweep, so the iterates do not depend on the number of
 * threads.  BiCGStab's dot products are reduced per thread, so their rounding does.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_c_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

/* Threads the loops will use when asked for `want` (0 = all available). */
int oracle_c_threads(int want) {
#ifdef _OPENMP
  if (want > 0) omp_set_num_threads(want);
  else omp_set_num_threads(omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)want;
  return 1;
#endif
}

static void diagonal(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* diag) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double dv = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) dv += v[k];
    diag[i] = dv;
  }
}

/* Jacobi for M x = b.  x: start vector in, final iterate out; work: n doubles.
 * Returns the number of sweeps; *delta = last max|x - x'|; *converged = 1 when it held. */
int64_t oracle_c_jacobi(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b,
                        double eps, int64_t max_iter, double* x, double* work, double* delta, int* converged) {
  double* diag = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!diag) return -1;
  diagonal(n, rp, ci, v, diag);
  double* cur = x;
  double* nxt = work;
  double d = INFINITY;
  int64_t it = 0;
  *converged = 0;
  for (it = 1; it <= max_iter; ++it) {
    double mx = 0.0;
#pragma omp parallel for schedule(static) reduction(max : mx)
    for (int64_t i = 0; i < n; ++i) {
      double t = 0.0;
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] != i) t += v[k] * cur[ci[k]];
      const double xi = (b[i] - t) / diag[i];
      const double dx = fabs(xi - cur[i]);
      if (dx > mx || dx != dx) mx = dx != dx ? INFINITY : dx;
      nxt[i] = xi;
    }
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
    d = n > 0 ? mx : 0.0;
    if (d < eps) {
      *converged = 1;
      break;
    }
  }
  if (it > max_iter) it = max_iter;
  if (cur != x) memcpy(x, cur, sizeof(double) * (size_t)n);
  *delta = d;
  free(diag);
  return it;
}

static void spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* u, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double t = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) t += v[k] * u[ci[k]];
    y[i] = t;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double maxabs(int64_t n, const double* a) {
  double m = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m)
  for (int64_t i = 0; i < n; ++i) {
    const double t = fabs(a[i]);
    if (t > m || t != t) m = t != t ? INFINITY : t;
  }
  return m;
}

/* BiCGStab for M x = b.  x: start vector in, solution out; work: 6 n doubles.
 * Returns 0 = converged, 1 = max_iter reached, 2 = breakdown after a restart.
 * *iters = iterations, *resid = last max|s| or max|r|. */
int oracle_c_bicgstab(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b,
                      double eps, int64_t max_iter, double* x, double* work, int64_t* iters, double* resid) {
  double *r = work, *q = work + n, *p = work + 2 * n, *vv = work + 3 * n, *s = work + 4 * n, *t = work + 5 * n;
  spmv(n, rp, ci, v, x, t);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  double rn = maxabs(n, r);
  *iters = 0;
  *resid = rn;
  if (n == 0 || rn < eps) return 0;
  memcpy(q, r, sizeof(double) * (size_t)n);
  memset(p, 0, sizeof(double) * (size_t)n);
  memset(vv, 0, sizeof(double) * (size_t)n);
  double y = 1.0, a = 1.0, w = 1.0;
  int restarted = 0;
  for (int64_t it = 1; it <= max_iter; ++it) {
    *iters = it;
    double yp = y;
    y = dot(n, q, r);
    if (y == 0.0) {
      if (restarted) return 2;
      restarted = 1;
      memcpy(q, r, sizeof(double) * (size_t)n);
      memset(p, 0, sizeof(double) * (size_t)n);
      memset(vv, 0, sizeof(double) * (size_t)n);
      yp = 1.0;
      a = 1.0;
      w = 1.0;
      y = dot(n, q, r);
    }
    const double beta = (y * a) / (yp * w);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - w * vv[i]);
    spmv(n, rp, ci, v, p, vv);
    double qv = dot(n, q, vv);
    if (qv == 0.0) {
      if (restarted) return 2;
      restarted = 1;
      memcpy(q, r, sizeof(double) * (size_t)n);
      memcpy(p, r, sizeof(double) * (size_t)n);
      spmv(n, rp, ci, v, r, vv);
      y = dot(n, q, r);
      qv = dot(n, q, vv);
      if (qv == 0.0) return 2;
    }
    a = y / qv;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) s[i] = r[i] - a * vv[i];
    const double sn = maxabs(n, s);
    if (sn < eps) {
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] + a * p[i];
      *resid = sn;
      return 0;
    }
    spmv(n, rp, ci, v, s, t);
    const double tt = dot(n, t, t);
    w = dot(n, t, s) / tt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + a * p[i] + w * s[i];
      r[i] = s[i] - w * t[i];
    }
    rn = maxabs(n, r);
    *resid = rn;
    if (rn < eps) return 0;
    if (w == 0.0) {
      if (restarted) return 2;
      restarted = 1;
      memcpy(q, r, sizeof(double) * (size_t)n);
      memset(p, 0, sizeof(double) * (size_t)n);
      memset(vv, 0, sizeof(double) * (size_t)n);
      y = 1.0;
      a = 1.0;
      w = 1.0;
    }
  }
  return 1;
}
