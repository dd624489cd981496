/*
 * eo_oracle_fp64.c — the CPU arithmetic of the paper's own kernels for block
 * orthogonalization (arXiv:1806.01036, Sec. 4.2), in plain FP64 and in the
 * double-double ("DD") form the paper uses to raise the precision.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests and the CPU-baseline / reference legs of
 * the benchmark do.  It shares no code, header or constant with the CUDA path
 * or with the binary128 reference in eo_oracle.c.
 *
 * Where eo_oracle.c gives the exact value (up to binary128 rounding) against
 * which everything is checked, this file computes what a CPU computes with
 * FP64 hardware, so that (a) the loss of orthogonality of the two
 * arithmetics (kappa^2 u for FP64, kappa^2 u^2 for DD, Sec. 4.2) can be
 * pinned on the CPU, and (b) the GPU can be timed against the paper's own
 * arithmetic on the host's cores.  Two modes:
 *
 *   mode 0, plain FP64: every product and sum rounded to FP64 in the order of
 *     the definition (a dot product is summed in row order; no FMA
 *     contraction: the file is compiled with -ffp-contract=off);
 *   mode 1, DD: every dot product over the rows is Dot2 of Ogita, Rump and
 *     Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005):
 *     each product split exactly by TwoProduct (one FMA), the running sum by
 *     Knuth's TwoSum, the errors summed in FP64, and the pair (sum, error
 *     sum) kept as a double-double instead of being added at the end; the
 *     k-by-k steps (Cholesky, inverse) run in double-double arithmetic
 *     (addition and multiplication as in Joldes, Muller and Popescu, "Tight
 *     and rigorous error bounds for basic building blocks of double-word
 *     arithmetic", ACM TOMS 2017; division and square root by one Newton
 *     correction of the FP64 quotient or root).  The update Y~ Z and the
 *     projection X - W C sum their terms by Dot2 and round once.
 *
 * Functions and the passage each follows:
 *   eo64_gram     M = X^T Y                               (Sec. 4.2, M = Y~^T Y~)
 *   eo64_project  C = W^T X, Y~ = X - W C, M = Y~^T Y~    (Sec. 4.2, phase I)
 *   eo64_cholqr   passes of Gram -> Cholesky -> Y = Y~ R^{-1}  (Sec. 4.2, CholQR)
 *
 * Matrices are column-major FP64 with a leading dimension >= rows.  The
 * dot products over rows are parallel over output entries (OpenMP), each
 * summed in row order, so results do not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* ------------------------------------------ error-free transformations */

typedef struct {
  double hi, lo;
} ddv;

/* s + e = a + b exactly (Knuth's TwoSum, no condition on a, b). */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *e = (a - av) + (b - bv);
  *s = x;
}

/* s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum). */
static void fast_two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  *e = b - (x - a);
  *s = x;
}

/* p + e = a * b exactly (TwoProduct with one fused multiply-add). */
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* a + b for double-words (accurate addition of Joldes-Muller-Popescu). */
static ddv dd_add(ddv a, ddv b) {
  double sh, sl, th, tl, vh, vl;
  two_sum(a.hi, b.hi, &sh, &sl);
  two_sum(a.lo, b.lo, &th, &tl);
  double c = sl + th;
  fast_two_sum(sh, c, &vh, &vl);
  double w = tl + vl;
  ddv z;
  fast_two_sum(vh, w, &z.hi, &z.lo);
  return z;
}

static ddv dd_neg(ddv a) {
  ddv z = {-a.hi, -a.lo};
  return z;
}

/* a * b for double-words (product of Joldes-Muller-Popescu with FMA). */
static ddv dd_mul(ddv a, ddv b) {
  double ch, cl1;
  two_prod(a.hi, b.hi, &ch, &cl1);
  double tl = a.hi * b.lo;
  double cl2 = fma(a.lo, b.hi, tl);
  double cl3 = cl1 + cl2;
  ddv z;
  fast_two_sum(ch, cl3, &z.hi, &z.lo);
  return z;
}

/* a / b: the FP64 quotient q, the exact-to-DD residual a - b q, one Newton
 * correction d = residual / b_hi, then q + d normalized. */
static ddv dd_div(ddv a, ddv b) {
  double q = a.hi / b.hi;
  ddv bq = dd_mul(b, (ddv){q, 0.0});
  ddv r = dd_add(a, dd_neg(bq));
  double d = r.hi / b.hi;
  ddv z;
  fast_two_sum(q, d, &z.hi, &z.lo);
  return z;
}

/* sqrt(a) for a > 0: the FP64 root s, the residual a - s^2 (s^2 split
 * exactly by TwoProduct), one Newton correction residual / (2 s). */
static ddv dd_sqrt(ddv a) {
  double s = sqrt(a.hi);
  double p, e;
  two_prod(s, s, &p, &e);
  double res = ((a.hi - p) - e) + a.lo;
  ddv z;
  fast_two_sum(s, res / (2.0 * s), &z.hi, &z.lo);
  return z;
}

/* ----------------------------------------------------------- dot products */

/* sum_r x_r y_r over n rows with strides: plain FP64 in row order (mode 0),
 * or Dot2 kept as the double-word (p, s) normalized by TwoSum (mode 1). */
static ddv dot_rows(int mode, int64_t n, const double* x, const double* y) {
  ddv out = {0.0, 0.0};
  if (mode == 0) {
    double s = 0.0;
    for (int64_t r = 0; r < n; ++r) s = s + x[r] * y[r];
    out.hi = s;
    return out;
  }
  double p = 0.0, s = 0.0;
  for (int64_t r = 0; r < n; ++r) {
    double h, e, q;
    two_prod(x[r], y[r], &h, &e);
    two_sum(p, h, &p, &q);
    s = s + (q + e);
  }
  two_sum(p, s, &out.hi, &out.lo);
  return out;
}

/* Round-once evaluation of a0 + sum_i a_i (b_i.hi + b_i.lo) for the row
 * products (projection, update).  mode 0: FP64 in order with b_i.hi only
 * (plain arithmetic keeps no low parts); mode 1: Dot2 over the hi products
 * with the lo products (below 2^-53 of them) added to the error sum. */
static double row_sum(int mode, double a0, int m, const double* a, const ddv* b) {
  if (mode == 0) {
    double s = a0;
    for (int i = 0; i < m; ++i) s = s + a[i] * b[i].hi;
    return s;
  }
  double p = a0, s = 0.0;
  for (int i = 0; i < m; ++i) {
    double h, e, q;
    two_prod(a[i], b[i].hi, &h, &e);
    two_sum(p, h, &p, &q);
    s = s + (q + (e + a[i] * b[i].lo));
  }
  return p + s;
}

/* ------------------------------------------------------------------ Gram */

/* G = X^T Y (Y == NULL: Y = X); G_lo (nullable) gets the DD low parts
 * (zero in mode 0). */
void eo64_gram(int mode, int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
               double* G_hi, double* G_lo, int ldg) {
  if (!Y) {
    Y = X;
    ldy = ldx;
  }
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kx; ++i)
    for (int j = 0; j < ky; ++j) {
      ddv g = dot_rows(mode, n, &AT(X, ldx, 0, i), &AT(Y, ldy, 0, j));
      AT(G_hi, ldg, i, j) = g.hi;
      if (G_lo) AT(G_lo, ldg, i, j) = g.lo;
    }
}

/* ------------------------------------------------------------- Projection */

/* Phase I: C = W^T X (as eo64_gram), Y~ = X - W C with every entry summed as
 * in row_sum and rounded once into Yt (which may alias X), then M = Y~^T Y~
 * of the stored Y~ (skipped when M_hi is NULL).  C_hi/C_lo, M_lo nullable. */
void eo64_project(int mode, int64_t n, int kv, const double* W, int64_t ldw, int k, const double* X, int64_t ldx,
                  double* Yt, int64_t ldyt, double* C_hi, double* C_lo, int ldc, double* M_hi, double* M_lo,
                  int ldm) {
  double* ch = (double*)calloc((size_t)kv * k, sizeof(double));
  double* cl = (double*)calloc((size_t)kv * k, sizeof(double));
  eo64_gram(mode, n, kv, W, ldw, k, X, ldx, ch, cl, kv);
  if (C_hi)
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < kv; ++i) {
        AT(C_hi, ldc, i, j) = ch[(size_t)j * kv + i];
        if (C_lo) AT(C_lo, ldc, i, j) = cl[(size_t)j * kv + i];
      }
#pragma omp parallel
  {
    double* w = (double*)malloc(sizeof(double) * (size_t)kv);
    ddv* c = (ddv*)malloc(sizeof(ddv) * (size_t)kv);
    double* row = (double*)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      for (int i = 0; i < kv; ++i) w[i] = -AT(W, ldw, r, i);
      for (int j = 0; j < k; ++j) {
        for (int i = 0; i < kv; ++i) c[i] = (ddv){ch[(size_t)j * kv + i], cl[(size_t)j * kv + i]};
        row[j] = row_sum(mode, AT(X, ldx, r, j), kv, w, c);
      }
      for (int j = 0; j < k; ++j) AT(Yt, ldyt, r, j) = row[j];
    }
    free(w);
    free(c);
    free(row);
  }
  free(ch);
  free(cl);
  if (M_hi) eo64_gram(mode, n, k, Yt, ldyt, k, NULL, 0, M_hi, M_lo, ldm);
}

/* -------------------------------------------------- k-by-k factorizations */

static ddv dv_add(int mode, ddv a, ddv b) {
  if (mode == 0) return (ddv){a.hi + b.hi, 0.0};
  return dd_add(a, b);
}
static ddv dv_mul(int mode, ddv a, ddv b) {
  if (mode == 0) return (ddv){a.hi * b.hi, 0.0};
  return dd_mul(a, b);
}
static ddv dv_div(int mode, ddv a, ddv b) {
  if (mode == 0) return (ddv){a.hi / b.hi, 0.0};
  return dd_div(a, b);
}
static ddv dv_sqrt(int mode, ddv a) {
  if (mode == 0) return (ddv){sqrt(a.hi), 0.0};
  return dd_sqrt(a);
}

/* Cholesky M = R^T R (upper triangle of M read; R upper, positive diagonal)
 * in the mode's arithmetic.  Returns 0, or j >= 1 when the j-th pivot is
 * not positive. */
static int chol(int mode, int k, const ddv* M, ddv* R) {
  for (size_t t = 0; t < (size_t)k * k; ++t) R[t] = (ddv){0.0, 0.0};
  for (int j = 0; j < k; ++j) {
    ddv d = M[(size_t)j * k + j];
    for (int i = 0; i < j; ++i) d = dv_add(mode, d, dd_neg(dv_mul(mode, R[(size_t)j * k + i], R[(size_t)j * k + i])));
    if (!(d.hi > 0.0)) return j + 1;
    ddv rjj = dv_sqrt(mode, d);
    R[(size_t)j * k + j] = rjj;
    for (int l = j + 1; l < k; ++l) {
      ddv s = M[(size_t)l * k + j];
      for (int i = 0; i < j; ++i)
        s = dv_add(mode, s, dd_neg(dv_mul(mode, R[(size_t)j * k + i], R[(size_t)l * k + i])));
      R[(size_t)l * k + j] = dv_div(mode, s, rjj);
    }
  }
  return 0;
}

/* Z = R^{-1} for upper-triangular R, by back substitution. */
static void triinv(int mode, int k, const ddv* R, ddv* Z) {
  for (size_t t = 0; t < (size_t)k * k; ++t) Z[t] = (ddv){0.0, 0.0};
  for (int j = 0; j < k; ++j) {
    Z[(size_t)j * k + j] = dv_div(mode, (ddv){1.0, 0.0}, R[(size_t)j * k + j]);
    for (int i = j - 1; i >= 0; --i) {
      ddv s = {0.0, 0.0};
      for (int l = i + 1; l <= j; ++l) s = dv_add(mode, s, dv_mul(mode, R[(size_t)l * k + i], Z[(size_t)j * k + l]));
      Z[(size_t)j * k + i] = dd_neg(dv_div(mode, s, R[(size_t)i * k + i]));
    }
  }
}

/* X <- X Z, every entry summed as in row_sum (zero start) and rounded once. */
static void update(int mode, int64_t n, int k, double* X, int64_t ldx, const ddv* Z) {
#pragma omp parallel
  {
    double* x = (double*)malloc(sizeof(double) * (size_t)k);
    ddv* z = (ddv*)malloc(sizeof(ddv) * (size_t)k);
    double* row = (double*)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      for (int i = 0; i < k; ++i) x[i] = AT(X, ldx, r, i);
      for (int j = 0; j < k; ++j) {
        for (int i = 0; i < k; ++i) z[i] = Z[(size_t)j * k + i];
        row[j] = row_sum(mode, 0.0, j + 1, x, z);  /* Z upper triangular: rows 0..j */
      }
      for (int j = 0; j < k; ++j) AT(X, ldx, r, j) = row[j];
    }
    free(x);
    free(z);
    free(row);
  }
}

/* CholQR in the mode's arithmetic: per pass, M = X^T X (or the given M for
 * the first pass), M = R^T R, Z = R^{-1}, X <- X Z (rounded once per entry).
 * R_hi/R_lo (nullable) get the product R_p ... R_1 of the passes' factors.
 * Returns 0, or the Cholesky breakdown column (X then holds the last
 * complete pass). */
int eo64_cholqr(int mode, int64_t n, int k, double* X, int64_t ldx, const double* M_hi, const double* M_lo, int ldm,
                int passes, double* R_hi, double* R_lo, int ldr) {
  const size_t kk = (size_t)k * k;
  ddv *M = (ddv*)calloc(kk, sizeof(ddv)), *R = (ddv*)calloc(kk, sizeof(ddv)), *Z = (ddv*)calloc(kk, sizeof(ddv));
  ddv *Rt = (ddv*)calloc(kk, sizeof(ddv)), *T = (ddv*)calloc(kk, sizeof(ddv));
  double *gh = (double*)calloc(kk, sizeof(double)), *gl = (double*)calloc(kk, sizeof(double));
  for (int i = 0; i < k; ++i) Rt[(size_t)i * k + i] = (ddv){1.0, 0.0};
  int info = 0;
  for (int p = 0; p < passes; ++p) {
    if (p == 0 && M_hi) {
      for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) {
          const int a = i <= j ? i : j, b = i <= j ? j : i;
          M[(size_t)j * k + i] = (ddv){AT(M_hi, ldm, a, b), (M_lo && mode) ? AT(M_lo, ldm, a, b) : 0.0};
        }
    } else {
      eo64_gram(mode, n, k, X, ldx, k, NULL, 0, gh, gl, k);
      for (size_t t = 0; t < kk; ++t) M[t] = (ddv){gh[t], mode ? gl[t] : 0.0};
    }
    info = chol(mode, k, M, R);
    if (info) break;
    triinv(mode, k, R, Z);
    update(mode, n, k, X, ldx, Z);
    for (int j = 0; j < k; ++j) /* Rt <- R Rt */
      for (int i = 0; i < k; ++i) {
        ddv s = {0.0, 0.0};
        for (int l = i; l <= j; ++l) s = dv_add(mode, s, dv_mul(mode, R[(size_t)l * k + i], Rt[(size_t)j * k + l]));
        T[(size_t)j * k + i] = s;
      }
    memcpy(Rt, T, sizeof(ddv) * kk);
  }
  if (R_hi)
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        AT(R_hi, ldr, i, j) = Rt[(size_t)j * k + i].hi;
        if (R_lo) AT(R_lo, ldr, i, j) = Rt[(size_t)j * k + i].lo;
      }
  free(M); free(R); free(Z); free(Rt); free(T); free(gh); free(gl);
  return info;
}
