/*
 * Oracle residual in double-double arithmetic (test infrastructure only).
 *
 * r = f - A u for the Kronecker operator of eq. A2D (2D) / eq. A3D (3D) with
 * the 1D matrices of eqs. matrixK / matrixM (absorbing corners 1 - i w h),
 * every product and sum carried in double-double (Dekker/Knuth error-free
 * transformations), rounded to double at the end.  Arrays are interleaved
 * complex, C order, last axis fastest.  Same operator as the numpy
 * oracle.fem.residual_dd, written for large grids (streaming, OpenMP).
 */
#include <math.h>
#include <stdint.h>

typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  dd r = {s, (a - (s - bb)) + (b - bb)};
  return r;
}
static inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  double c = 134217729.0 * a, ah = c - (c - a), al = a - ah;
  double d = 134217729.0 * b, bh = d - (d - b), bl = b - bh;
  dd r = {p, ((ah * bh - p) + ah * bl + al * bh) + al * bl};
  return r;
}
static inline dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  double e = s.lo + t.hi;
  dd v = fast_two_sum(s.hi, e);
  e = v.lo + t.lo;
  return fast_two_sum(v.hi, e);
}
static inline dd dd_mul_d(dd x, double b) {
  dd p = two_prod(x.hi, b);
  double e = p.lo + x.lo * b;
  return fast_two_sum(p.hi, e);
}
static inline dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  double e = p.lo + (x.hi * y.lo + x.lo * y.hi);
  return fast_two_sum(p.hi, e);
}
static inline dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static inline dd dd_d(double a) { dd r = {a, 0.0}; return r; }

typedef struct { dd re, im; } cdd;

static inline cdd cdd_add(cdd a, cdd b) { cdd r = {dd_add(a.re, b.re), dd_add(a.im, b.im)}; return r; }
/* complex dd * complex dd */
static inline cdd cdd_mul(cdd a, cdd b) {
  cdd r;
  r.re = dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im)));
  r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
  return r;
}
/* complex dd * complex double */
static inline cdd cdd_mul_cd(cdd a, double br, double bi) {
  cdd r;
  r.re = dd_add(dd_mul_d(a.re, br), dd_neg(dd_mul_d(a.im, bi)));
  r.im = dd_add(dd_mul_d(a.re, bi), dd_mul_d(a.im, br));
  return r;
}

/* 1D entries: X(i, i+d) for X = M (kind 0) or K (kind 1); K complex at
 * absorbing ends (corner 1/h - i wc; wc = 0 for a Neumann axis).  M is
 * h [(den-2)/den on the diagonal, 1/den off it, half the diagonal at the
 * ends]: den = 6 for the paper's elements, 12 for the modified ones. */
static void entry(int64_t n, double h, double omega, double den, int64_t i, int d, int kind, double* re,
                  double* im) {
  int end = (i == 0 || i == n - 1);
  if (kind == 0) {
    *re = (d == 0) ? (end ? (den - 2.0) / 2.0 : den - 2.0) * h / den : h / den;
    *im = 0.0;
  } else {
    if (d == 0) {
      *re = (end ? 1.0 : 2.0) / h;
      *im = end ? -omega : 0.0;
    } else {
      *re = -1.0 / h;
      *im = 0.0;
    }
  }
}

/* Coefficient of neighbour offset d[] at index idx[]: sum over terms of
 * products of 1D entries, each product formed in complex double-double. */
static cdd coefficient(int dim, const int64_t* n, const double* h, double omega, const double* wc, double den,
                       const int64_t* idx, const int* d) {
  cdd total = {dd_d(0.0), dd_d(0.0)};
  for (int j = 0; j <= dim; ++j) {
    cdd prod = {dd_d(1.0), dd_d(0.0)};
    for (int k = 0; k < dim; ++k) {
      double er, ei;
      entry(n[k], h[k], wc[k], den, idx[k], d[k], (k == j) ? 1 : 0, &er, &ei);
      prod = cdd_mul_cd(prod, er, ei);
    }
    if (j == dim) {
      /* -w^2 enters as one double, the same operator entry as eq. A2D's
       * (K - w^2 M) with w^2 rounded once */
      cdd s = {dd_d(-(omega * omega)), dd_d(0.0)};
      prod = cdd_mul(prod, s);
    }
    total = cdd_add(total, prod);
  }
  return total;
}

/* r = f - A u in double-double.  wc[k]: the w of the absorbing corner of
 * axis k (w itself on an absorbing axis, 0 on a Neumann axis, Section 2's
 * Gamma_A / Gamma_N); den: the mass matrix's denominator (element). */
void helm_oracle_dd_residual_el(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                                double den, const double* f, const double* u, double* r) {
  int64_t N = 1;
  for (int k = 0; k < dim; ++k) N *= n[k];
  int64_t stride[3];
  stride[dim - 1] = 1;
  for (int k = dim - 2; k >= 0; --k) stride[k] = stride[k + 1] * n[k + 1];
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < N; ++g) {
    int64_t idx[3] = {0, 0, 0}, rem = g;
    for (int k = dim - 1; k >= 0; --k) {
      idx[k] = rem % n[k];
      rem /= n[k];
    }
    cdd acc = {dd_d(f[2 * g]), dd_d(f[2 * g + 1])};
    int d[3] = {0, 0, 0};
    int cnt = 1;
    for (int k = 0; k < dim; ++k) cnt *= 3;
    for (int c = 0; c < cnt; ++c) {
      int t = c, ok = 1;
      int64_t off = 0;
      for (int k = dim - 1; k >= 0; --k) {
        d[k] = t % 3 - 1;
        t /= 3;
        int64_t j = idx[k] + d[k];
        if (j < 0 || j >= n[k]) ok = 0;
        off += d[k] * stride[k];
      }
      if (!ok) continue;
      cdd co = coefficient(dim, n, h, omega, wc, den, idx, d);
      cdd term = cdd_mul_cd(co, u[2 * (g + off)], u[2 * (g + off) + 1]);
      acc.re = dd_add(acc.re, dd_neg(term.re));
      acc.im = dd_add(acc.im, dd_neg(term.im));
    }
    r[2 * g] = acc.re.hi + acc.re.lo;
    r[2 * g + 1] = acc.im.hi + acc.im.lo;
  }
}

/* The paper's elements, per-axis conditions. */
void helm_oracle_dd_residual_bc(int dim, const int64_t* n, const double* h, double omega, const double* wc,
                                const double* f, const double* u, double* r) {
  helm_oracle_dd_residual_el(dim, n, h, omega, wc, 6.0, f, u, r);
}

/* Absorbing conditions on every face. */
void helm_oracle_dd_residual(int dim, const int64_t* n, const double* h, double omega, const double* f,
                             const double* u, double* r) {
  const double wc[3] = {omega, omega, omega};
  helm_oracle_dd_residual_bc(dim, n, h, omega, wc, f, u, r);
}
