/*
 * eo_oracle.c — CPU oracle for block orthogonalization (arXiv:1806.01036, Sec. 4.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or constant with the CUDA path.
 *
 * Every quantity is computed from its plain definition in IEEE binary128
 * ("quad": 113-bit significand, unit roundoff 2^-113), so for the sizes used
 * here its own rounding error is far below the double-double (2^-106) level
 * that the GPU's compensated mode is checked against.  Results leave the
 * oracle as FP64 (rounded once) or as an unevaluated pair hi + lo of FP64
 * (hi = fl64(q), lo = fl64(q - hi)).
 *
 * Functions and the passage each follows:
 *   eoq_gram       M = X^T Y, the Gram product of phase II            (Sec. 4.2, M = Y~^T Y~)
 *   eoq_project    C = W^T X, Y~ = X - W C, then M = Y~^T Y~          (Sec. 4.2, phase I)
 *   eoq_project_apply  Y~ = X - W C for a given double-double C          (Sec. 4.2, phase I)
 *   eoq_cholesky   M = R^T R, R upper with positive diagonal          (Sec. 4.2, CholQR)
 *   eoq_triinv     Z = R^{-1}                                         (Sec. 4.2, CholQR: Z = R^{-1})
 *   eoq_jacobi     M = U Lambda U^T by cyclic Jacobi rotations         (Sec. 4.2, SVQB eigendecomposition)
 *   eoq_cholqr     one or two passes of Gram -> Cholesky -> Y = Y~ Z   (Sec. 4.2, CholQR)
 *   eoq_svqb       one or two passes of Gram -> eig -> Y = Y~ Z,
 *                  Z = U Lambda^{-1/2} U^T = M^{-1/2}                 (Sec. 4.2, SVQB with the
 *                                                                      Frobenius-optimal Z of the
 *                                                                      Procrustes argument)
 *   eoq_svqb_rot   one pass of SVQB with the transform as the section first
 *                  writes it, Z = D U Lambda^{-1/2} (D = diag(M)^{-1/2},
 *                  D M D = U Lambda U^T; eigenvalues ascending, each
 *                  eigenvector's largest entry positive)              (Sec. 4.2, SVQB, Z = U Lambda^{-1/2}
 *                                                                      with the diagonal scaling of
 *                                                                      Stathopoulos and Wu)
 *   eoq_cholqr_piv CholQR with a diagonally pivoted Cholesky stopped at the
 *                  numerical rank, then an unpivoted second pass          (Sec. 4.2, the pivoted, partial
 *                                                                      Cholesky of phase II)
 *   eoq_orthogonalize  phase I, the measures max(||W^T Y||_F, ||Y^T Y - I||_F),
 *                  then SVQB, repeated until the measures are <= eps      (Sec. 4.2, iterated two-phase
 *                                                                      algorithm; runtime figure)
 *   eoq_cholqr_b, eoq_svqb_b, eoq_project_b
 *                  the same with the inner product <x, y>_B = x^T B y of
 *                  a symmetric positive definite B, given through P = B X:
 *                  M = the symmetric part of X^T P, and every transform Z
 *                  applied to X is applied to P as well               (Sec. 4.2, closing remark:
 *                                                                      the method extends to
 *                                                                      B-inner products)
 *   eoq_orth_err_diag  ||Q^T D Q - I|| for a diagonal B = D            (B-orthonormality)
 *   eoq_orth_err   ||Q^T Q - I|| in 2-norm, Frobenius and max-abs     (Sec. 4.2, one-iteration accuracy figure)
 *   eoq_cross_err  ||W^T Q||_2                                        (same figure, left panel)
 *   eoq_fact_err   ||X - Q R||_F / ||X||_F                            (definition of a QR factorization)
 *
 * Matrices are column-major FP64 with a leading dimension >= rows.  The
 * precision of this file's arithmetic is fixed by the qreal typedef below;
 * -ffp-contract=off keeps the compiler from fusing or reordering anything.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 qreal;
#elif defined(__aarch64__)
typedef long double qreal;
_Static_assert(__LDBL_MANT_DIG__ == 113, "AArch64 long double must be IEEE binary128");
#else
#error "oracle needs an IEEE binary128 type"
#endif

#define AT(A, ld, i, j) ((A)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

/* ---------------------------------------------------------------- helpers */

static qreal qabs(qreal x) { return x < 0 ? -x : x; }

/* Square root in binary128: Newton's iteration y <- (y + x/y)/2 from the FP64
 * root; each step doubles the number of correct bits (53 -> 106 -> >113). */
static qreal qsqrt(qreal x) {
  if (x <= 0) return x == 0 ? (qreal)0 : (qreal)NAN;
  qreal y = (qreal)sqrt((double)x);
  for (int it = 0; it < 3; ++it) y = (y + x / y) / 2;
  return y;
}

static void q_to_dd(qreal q, double* hi, double* lo) {
  double h = (double)q;
  *hi = h;
  if (lo) *lo = (double)(q - (qreal)h);
}

static qreal dd_to_q(const double* hi, const double* lo, size_t idx) {
  qreal v = (qreal)hi[idx];
  if (lo) v += (qreal)lo[idx];
  return v;
}

static qreal* qalloc(size_t count) {
  qreal* p = (qreal*)calloc(count ? count : 1, sizeof(qreal));
  return p;
}

int eoq_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the later parallel loops (timing on one core or on all). */
void eoq_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* ----------------------------------------------------------- Gram product */

/* G = X^T Y: G_ij = sum_{r=0}^{n-1} X_ri Y_rj, summed in row order in binary128.
 * Y == NULL means Y = X.  G is kx-by-ky with leading dimension ldg. */
void eoq_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
              double* G_hi, double* G_lo, int ldg) {
  if (!Y) { Y = X; ldy = ldx; }
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kx; ++i)
    for (int j = 0; j < ky; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(X, ldx, r, i) * (qreal)AT(Y, ldy, r, j);
      q_to_dd(s, &AT(G_hi, ldg, i, j), G_lo ? &AT(G_lo, ldg, i, j) : NULL);
    }
}

/* FP32-input variant: the FP32 entries are widened to binary128 (exactly). */
void eoq_gram_f32(int64_t n, int kx, const float* X, int64_t ldx, int ky, const float* Y, int64_t ldy,
                  double* G_hi, double* G_lo, int ldg) {
  if (!Y) { Y = X; ldy = ldx; }
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kx; ++i)
    for (int j = 0; j < ky; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(X, ldx, r, i) * (qreal)AT(Y, ldy, r, j);
      q_to_dd(s, &AT(G_hi, ldg, i, j), G_lo ? &AT(G_lo, ldg, i, j) : NULL);
    }
}

/* ------------------------------------------------------------- Projection */

/* Phase I: C = W^T X (kv-by-k), Y~ = X - W C computed in binary128 with the
 * unrounded C and rounded once to FP64 into Yt (which may alias X), then
 * M = Y~^T Y~ of the rounded Y~ (k-by-k; skipped when M_hi is NULL). */
void eoq_project(int64_t n, int kv, const double* W, int64_t ldw, int k, const double* X, int64_t ldx,
                 double* Yt, int64_t ldyt, double* C_hi, double* C_lo, int ldc, double* M_hi, double* M_lo,
                 int ldm) {
  qreal* C = qalloc((size_t)kv * k);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kv; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(W, ldw, r, i) * (qreal)AT(X, ldx, r, j);
      C[(size_t)j * kv + i] = s;
    }
  if (C_hi)
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < kv; ++i) q_to_dd(C[(size_t)j * kv + i], &AT(C_hi, ldc, i, j), C_lo ? &AT(C_lo, ldc, i, j) : NULL);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r)
    for (int j = 0; j < k; ++j) {
      qreal s = (qreal)AT(X, ldx, r, j);
      for (int i = 0; i < kv; ++i) s -= (qreal)AT(W, ldw, r, i) * C[(size_t)j * kv + i];
      AT(Yt, ldyt, r, j) = (double)s;
    }
  free(C);
  if (M_hi) eoq_gram(n, k, Yt, ldyt, k, NULL, 0, M_hi, M_lo, ldm);
}

/* The application step of phase I with C supplied (C = C_hi + C_lo, kv-by-k,
 * C_lo may be NULL): Y~ = X - W C, every entry summed in binary128 and
 * rounded once to FP64. */
void eoq_project_apply(int64_t n, int kv, const double* W, int64_t ldw, int k, const double* X, int64_t ldx,
                       const double* C_hi, const double* C_lo, int ldc, double* Yt, int64_t ldyt) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r)
    for (int j = 0; j < k; ++j) {
      qreal s = (qreal)AT(X, ldx, r, j);
      for (int i = 0; i < kv; ++i) {
        const qreal c = (qreal)AT(C_hi, ldc, i, j) + (C_lo ? (qreal)AT(C_lo, ldc, i, j) : (qreal)0);
        s -= (qreal)AT(W, ldw, r, i) * c;
      }
      AT(Yt, ldyt, r, j) = (double)s;
    }
}

/* -------------------------------------------------- k-by-k factorizations */

/* Cholesky M = R^T R with R upper triangular and positive diagonal (the
 * factorization CholQR uses).  M = M_hi + M_lo (M_lo may be NULL), only the
 * upper triangle is read.  Returns 0, or j >= 1 when the j-th pivot is not
 * positive (R is then left with its first j-1 rows).  The strict lower
 * triangle of R is set to zero. */
static int q_cholesky(int k, const qreal* M, qreal* R) {
  for (size_t t = 0; t < (size_t)k * k; ++t) R[t] = 0;
  for (int j = 0; j < k; ++j) {
    qreal d = M[(size_t)j * k + j];
    for (int i = 0; i < j; ++i) d -= R[(size_t)j * k + i] * R[(size_t)j * k + i];
    if (!(d > 0)) return j + 1;
    qreal rjj = qsqrt(d);
    R[(size_t)j * k + j] = rjj;
    for (int l = j + 1; l < k; ++l) {
      qreal s = M[(size_t)l * k + j];
      for (int i = 0; i < j; ++i) s -= R[(size_t)j * k + i] * R[(size_t)l * k + i];
      R[(size_t)l * k + j] = s / rjj;
    }
  }
  return 0;
}

/* Z = R^{-1} for upper-triangular R by back substitution column by column. */
static void q_triinv(int k, const qreal* R, qreal* Z) {
  for (size_t t = 0; t < (size_t)k * k; ++t) Z[t] = 0;
  for (int j = 0; j < k; ++j) {
    Z[(size_t)j * k + j] = 1 / R[(size_t)j * k + j];
    for (int i = j - 1; i >= 0; --i) {
      qreal s = 0;
      for (int l = i + 1; l <= j; ++l) s += R[(size_t)l * k + i] * Z[(size_t)j * k + l];
      Z[(size_t)j * k + i] = -s / R[(size_t)i * k + i];
    }
  }
}

/* Cyclic Jacobi eigendecomposition of the symmetric k-by-k A (destroyed):
 * A = U diag(lam) U^T.  Each rotation annihilates A_pq with the classical
 * choice tan(phi) = t, t the smaller root of t^2 + 2 theta t - 1 = 0,
 * theta = (A_qq - A_pp) / (2 A_pq).  Sweeps continue until the off-diagonal
 * mass is negligible against the diagonal in binary128. */
static void q_jacobi(int k, qreal* A, qreal* U, qreal* lam) {
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) U[(size_t)j * k + i] = (i == j);
  for (int sweep = 0; sweep < 100; ++sweep) {
    qreal off = 0, diag = 0;
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        qreal v = A[(size_t)j * k + i] * A[(size_t)j * k + i];
        if (i == j) diag += v; else off += v;
      }
    if (off == 0 || off <= diag * (qreal)1e-70) break;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        qreal apq = A[(size_t)q * k + p];
        if (apq == 0) continue;
        qreal app = A[(size_t)p * k + p], aqq = A[(size_t)q * k + q];
        qreal theta = (aqq - app) / (2 * apq);
        qreal t = 1 / (qabs(theta) + qsqrt(theta * theta + 1));
        if (theta < 0) t = -t;
        qreal c = 1 / qsqrt(t * t + 1), s = t * c;
        for (int r = 0; r < k; ++r) {  /* A <- A J (columns p, q) */
          qreal arp = A[(size_t)p * k + r], arq = A[(size_t)q * k + r];
          A[(size_t)p * k + r] = c * arp - s * arq;
          A[(size_t)q * k + r] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {  /* A <- J^T A (rows p, q) */
          qreal apr = A[(size_t)r * k + p], aqr = A[(size_t)r * k + q];
          A[(size_t)r * k + p] = c * apr - s * aqr;
          A[(size_t)r * k + q] = s * apr + c * aqr;
        }
        A[(size_t)q * k + p] = 0;
        A[(size_t)p * k + q] = 0;
        for (int r = 0; r < k; ++r) {  /* U <- U J */
          qreal urp = U[(size_t)p * k + r], urq = U[(size_t)q * k + r];
          U[(size_t)p * k + r] = c * urp - s * urq;
          U[(size_t)q * k + r] = s * urp + c * urq;
        }
      }
  }
  for (int i = 0; i < k; ++i) lam[i] = A[(size_t)i * k + i];
}

static void load_sym(int k, const double* M_hi, const double* M_lo, int ldm, qreal* M) {
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      int a = i <= j ? i : j, b = i <= j ? j : i; /* read the upper triangle */
      M[(size_t)j * k + i] = dd_to_q(M_hi, M_lo, (size_t)b * ldm + a);
    }
}

static void store_dd(int k, const qreal* A, double* hi, double* lo, int ld) {
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) q_to_dd(A[(size_t)j * k + i], &AT(hi, ld, i, j), lo ? &AT(lo, ld, i, j) : NULL);
}

int eoq_cholesky(int k, const double* M_hi, const double* M_lo, int ldm, double* R_hi, double* R_lo, int ldr) {
  qreal *M = qalloc((size_t)k * k), *R = qalloc((size_t)k * k);
  load_sym(k, M_hi, M_lo, ldm, M);
  int info = q_cholesky(k, M, R);
  store_dd(k, R, R_hi, R_lo, ldr);
  free(M); free(R);
  return info;
}

void eoq_triinv(int k, const double* R_hi, const double* R_lo, int ldr, double* Z_hi, double* Z_lo, int ldz) {
  qreal *R = qalloc((size_t)k * k), *Z = qalloc((size_t)k * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) R[(size_t)j * k + i] = i <= j ? dd_to_q(R_hi, R_lo, (size_t)j * ldr + i) : 0;
  q_triinv(k, R, Z);
  store_dd(k, Z, Z_hi, Z_lo, ldz);
  free(R); free(Z);
}

/* Eigenvalues (unsorted, as the rotations leave them) and eigenvectors. */
void eoq_jacobi(int k, const double* M_hi, const double* M_lo, int ldm, double* U_out, int ldu, double* lam_hi,
                double* lam_lo) {
  qreal *A = qalloc((size_t)k * k), *U = qalloc((size_t)k * k), *lam = qalloc(k);
  load_sym(k, M_hi, M_lo, ldm, A);
  q_jacobi(k, A, U, lam);
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < k; ++i) AT(U_out, ldu, i, j) = (double)U[(size_t)j * k + i];
    q_to_dd(lam[j], &lam_hi[j], lam_lo ? &lam_lo[j] : NULL);
  }
  free(A); free(U); free(lam);
}

/* SVQB transform Z = U Lambda^{+1/2} U^T of M = U Lambda U^T, where
 * Lambda^{+1/2} inverts the square root of every eigenvalue above
 * tol * lambda_max and zeroes the others.  Returns the number kept. */
static int q_svqb_z(int k, const qreal* M, qreal tol, qreal* Z) {
  qreal *A = qalloc((size_t)k * k), *U = qalloc((size_t)k * k), *lam = qalloc(k), *w = qalloc(k);
  memcpy(A, M, sizeof(qreal) * (size_t)k * k);
  q_jacobi(k, A, U, lam);
  qreal lmax = 0;
  for (int i = 0; i < k; ++i) if (lam[i] > lmax) lmax = lam[i];
  int rank = 0;
  for (int i = 0; i < k; ++i) {
    if (lmax > 0 && lam[i] > tol * lmax) { w[i] = 1 / qsqrt(lam[i]); ++rank; }
    else w[i] = 0;
  }
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      qreal s = 0;
      for (int l = 0; l < k; ++l) s += U[(size_t)l * k + i] * w[l] * U[(size_t)l * k + j];
      Z[(size_t)j * k + i] = s;
    }
  free(A); free(U); free(lam); free(w);
  return rank;
}

int eoq_svqb_z(int k, const double* M_hi, const double* M_lo, int ldm, double tol, double* Z_hi, double* Z_lo, int ldz) {
  qreal *M = qalloc((size_t)k * k), *Z = qalloc((size_t)k * k);
  load_sym(k, M_hi, M_lo, ldm, M);
  int rank = q_svqb_z(k, M, (qreal)tol, Z);
  store_dd(k, Z, Z_hi, Z_lo, ldz);
  free(M); free(Z);
  return rank;
}

/* The rotated SVQB transform: with d_i = M_ii^{-1/2} (0 for a column with
 * no positive diagonal entry) and D M D = U Lambda U^T, Z = D U Lambda^{+1/2}
 * with the eigenpairs in ascending order of eigenvalue (equal ones by index)
 * and each eigenvector's largest-magnitude entry made positive (the first
 * one on a tie).  Eigenvalues not above tol * lambda_max give zero columns.
 * Returns the number kept. */
static int q_svqb_rot_z(int k, const qreal* M, qreal tol, qreal* Z) {
  qreal *A = qalloc((size_t)k * k), *U = qalloc((size_t)k * k), *lam = qalloc(k), *d = qalloc(k);
  int* order = (int*)malloc(sizeof(int) * (size_t)k);
  for (int i = 0; i < k; ++i) d[i] = M[(size_t)i * k + i] > 0 ? 1 / qsqrt(M[(size_t)i * k + i]) : 0;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) A[(size_t)j * k + i] = d[i] * M[(size_t)j * k + i] * d[j];
  q_jacobi(k, A, U, lam);
  for (int a = 0; a < k; ++a) order[a] = a;
  for (int a = 1; a < k; ++a) {  /* insertion sort, ascending, stable */
    int v = order[a], b = a - 1;
    while (b >= 0 && lam[order[b]] > lam[v]) { order[b + 1] = order[b]; --b; }
    order[b + 1] = v;
  }
  for (int a = 0; a < k; ++a) {  /* sign: the largest |U(m, a)| positive */
    int mbest = 0;
    for (int m = 1; m < k; ++m)
      if (qabs(U[(size_t)a * k + m]) > qabs(U[(size_t)a * k + mbest])) mbest = m;
    if (U[(size_t)a * k + mbest] < 0)
      for (int m = 0; m < k; ++m) U[(size_t)a * k + m] = -U[(size_t)a * k + m];
  }
  qreal lmax = 0;
  for (int i = 0; i < k; ++i) if (lam[i] > lmax) lmax = lam[i];
  int rank = 0;
  for (int j = 0; j < k; ++j) {
    const int a = order[j];
    const int keep = lmax > 0 && lam[a] > tol * lmax;
    const qreal w = keep ? 1 / qsqrt(lam[a]) : 0;
    rank += keep;
    for (int i = 0; i < k; ++i) Z[(size_t)j * k + i] = d[i] * U[(size_t)a * k + i] * w;
  }
  free(A); free(U); free(lam); free(d); free(order);
  return rank;
}

/* Q = X Z with every entry summed in binary128 and rounded once; Q may alias X. */
static void q_update(int64_t n, int k, double* X, int64_t ldx, const qreal* Z) {
#pragma omp parallel
  {
    double* row = (double*)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      for (int j = 0; j < k; ++j) {
        qreal s = 0;
        for (int i = 0; i < k; ++i) s += (qreal)AT(X, ldx, r, i) * Z[(size_t)j * k + i];
        row[j] = (double)s;
      }
      for (int j = 0; j < k; ++j) AT(X, ldx, r, j) = row[j];
    }
    free(row);
  }
}

static void q_gram_sym(int64_t n, int k, const double* X, int64_t ldx, qreal* M) {
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(X, ldx, r, i) * (qreal)AT(X, ldx, r, j);
      M[(size_t)j * k + i] = s;
    }
}

/* C = A B for k-by-k upper-triangular A, B (binary128). */
static void q_trmul(int k, const qreal* A, const qreal* B, qreal* C) {
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      qreal s = 0;
      for (int l = 0; l < k; ++l) s += A[(size_t)l * k + i] * B[(size_t)j * k + l];
      C[(size_t)j * k + i] = s;
    }
}

/* CholQR: per pass, M = X^T X, M = R^T R, Z = R^{-1}, X <- X Z (rounded to
 * FP64 once per pass).  After `passes` passes X holds Q and R = R_p ... R_1.
 * If M_hi is given, the first pass uses that Gram matrix instead of X^T X.
 * Returns 0 or the Cholesky breakdown column (X then holds the last complete
 * pass, R the product so far). */
int eoq_cholqr(int64_t n, int k, double* X, int64_t ldx, const double* M_hi, const double* M_lo, int ldm,
               int passes, double* R_hi, double* R_lo, int ldr) {
  size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *R = qalloc(kk), *Z = qalloc(kk), *Rt = qalloc(kk), *T = qalloc(kk);
  for (int i = 0; i < k; ++i) Rt[(size_t)i * k + i] = 1;
  int info = 0;
  for (int p = 0; p < passes; ++p) {
    if (p == 0 && M_hi) load_sym(k, M_hi, M_lo, ldm, M);
    else q_gram_sym(n, k, X, ldx, M);
    info = q_cholesky(k, M, R);
    if (info) break;
    q_triinv(k, R, Z);
    q_update(n, k, X, ldx, Z);
    q_trmul(k, R, Rt, T);
    memcpy(Rt, T, sizeof(qreal) * kk);
  }
  if (R_hi) store_dd(k, Rt, R_hi, R_lo, ldr);
  free(M); free(R); free(Z); free(Rt); free(T);
  return info;
}

/* SVQB: per pass, M = X^T X, Z = M^{-1/2} (pseudo-inverse square root with
 * relative eigenvalue cut tol), X <- X Z.  Z_out gets the product of the
 * passes' transforms (Z_1 Z_2 ...).  Returns the rank of the last pass. */
/* Rotated SVQB, one pass: M = X^T X (or the given one), Z from
 * q_svqb_rot_z, X <- X Z.  Returns the number of kept directions. */
int eoq_svqb_rot(int64_t n, int k, double* X, int64_t ldx, const double* M_hi, const double* M_lo, int ldm,
                 double tol, double* Z_hi, double* Z_lo, int ldz);

int eoq_svqb(int64_t n, int k, double* X, int64_t ldx, const double* M_hi, const double* M_lo, int ldm,
             double tol, int passes, double* Z_hi, double* Z_lo, int ldz) {
  size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *Z = qalloc(kk), *Zt = qalloc(kk), *T = qalloc(kk);
  for (int i = 0; i < k; ++i) Zt[(size_t)i * k + i] = 1;
  int rank = k;
  for (int p = 0; p < passes; ++p) {
    if (p == 0 && M_hi) load_sym(k, M_hi, M_lo, ldm, M);
    else q_gram_sym(n, k, X, ldx, M);
    rank = q_svqb_z(k, M, (qreal)tol, Z);
    q_update(n, k, X, ldx, Z);
    for (int j = 0; j < k; ++j)  /* Zt <- Zt Z (full matrices) */
      for (int i = 0; i < k; ++i) {
        qreal s = 0;
        for (int l = 0; l < k; ++l) s += Zt[(size_t)l * k + i] * Z[(size_t)j * k + l];
        T[(size_t)j * k + i] = s;
      }
    memcpy(Zt, T, sizeof(qreal) * kk);
  }
  if (Z_hi) store_dd(k, Zt, Z_hi, Z_lo, ldz);
  free(M); free(Z); free(Zt); free(T);
  return rank;
}

int eoq_svqb_rot(int64_t n, int k, double* X, int64_t ldx, const double* M_hi, const double* M_lo, int ldm,
                 double tol, double* Z_hi, double* Z_lo, int ldz) {
  size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *Z = qalloc(kk);
  if (M_hi) load_sym(k, M_hi, M_lo, ldm, M);
  else q_gram_sym(n, k, X, ldx, M);
  int rank = q_svqb_rot_z(k, M, (qreal)tol, Z);
  q_update(n, k, X, ldx, Z);
  if (Z_hi) store_dd(k, Z, Z_hi, Z_lo, ldz);
  free(M); free(Z);
  return rank;
}

/* --------------------------------------- pivoted, partial Cholesky QR */

/* Cholesky with diagonal pivoting, stopped early (Sec. 4.2 allows the
 * phase-II Cholesky factorization to be pivoted and partial, which makes it
 * rank-revealing).  On the symmetric M (k-by-k, binary128), step j takes
 * the largest remaining diagonal entry (lowest index on ties) as pivot p,
 * swaps rows and columns j and p, and stops with rank j when that entry is
 * not above tol * (largest diagonal entry of M); otherwise R(j,j) =
 * sqrt(pivot), R(j,l) = A(j,l) / R(j,j) and the trailing matrix loses the
 * outer product of row j of R.  perm[j] is the original index of the j-th
 * pivot; R (k-by-k, rows >= rank zero) satisfies P^T M P ~ R^T R on the
 * leading rank columns.  Returns the rank. */
static int q_pivchol(int k, const qreal* M, qreal tol, int* perm, qreal* R) {
  qreal* A = qalloc((size_t)k * k);
  memcpy(A, M, sizeof(qreal) * (size_t)k * k);
  for (size_t t = 0; t < (size_t)k * k; ++t) R[t] = 0;
  for (int i = 0; i < k; ++i) perm[i] = i;
  qreal dmax = 0;
  for (int i = 0; i < k; ++i) if (A[(size_t)i * k + i] > dmax) dmax = A[(size_t)i * k + i];
  int rank = 0;
  for (int j = 0; j < k; ++j) {
    int p = j;
    for (int i = j + 1; i < k; ++i) if (A[(size_t)i * k + i] > A[(size_t)p * k + p]) p = i;
    const qreal d = A[(size_t)p * k + p];
    if (!(d > 0) || !(d > tol * dmax)) break;
    if (p != j) {  /* symmetric swap of rows and columns j and p; also the rows of R built so far */
      for (int i = 0; i < k; ++i) {
        qreal t = A[(size_t)j * k + i]; A[(size_t)j * k + i] = A[(size_t)p * k + i]; A[(size_t)p * k + i] = t;
      }
      for (int i = 0; i < k; ++i) {
        qreal t = A[(size_t)i * k + j]; A[(size_t)i * k + j] = A[(size_t)i * k + p]; A[(size_t)i * k + p] = t;
      }
      for (int i = 0; i < j; ++i) {
        qreal t = R[(size_t)j * k + i]; R[(size_t)j * k + i] = R[(size_t)p * k + i]; R[(size_t)p * k + i] = t;
      }
      int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
    }
    const qreal rjj = qsqrt(A[(size_t)j * k + j]);
    R[(size_t)j * k + j] = rjj;
    for (int l = j + 1; l < k; ++l) R[(size_t)l * k + j] = A[(size_t)l * k + j] / rjj;
    for (int a = j + 1; a < k; ++a)
      for (int b = j + 1; b < k; ++b) A[(size_t)b * k + a] -= R[(size_t)a * k + j] * R[(size_t)b * k + j];
    rank = j + 1;
  }
  free(A);
  return rank;
}

/* Pivoted, partial CholQR: pass 1 factors M = X^T X with q_pivchol and sets
 * X <- X P [R11^{-1}, 0; 0, 0] (R11 the leading rank-by-rank block), so the
 * first rank columns of X are orthonormal and span X's numerical range and
 * the others are zero; pass 2 (passes = 2) factors the leading rank-by-rank
 * block of the new Gram matrix without pivoting, X <- X [R2^{-1}, 0; 0, 0],
 * and R <- R2 R.  Every entry of X is summed in binary128 and rounded once
 * per pass.  perm (k ints) and R (k-by-k, X P ~ Q R, rows >= rank zero) are
 * those of the whole; *rank_out the rank.  Returns 0, or j >= 1 if the
 * second pass breaks down at column j (X then holds the first pass). */
int eoq_cholqr_piv(int64_t n, int k, double* X, int64_t ldx, double tol, int passes, int* perm, int* rank_out,
                   double* R_hi, double* R_lo, int ldr) {
  const size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *R = qalloc(kk), *Z = qalloc(kk), *Zs = qalloc(kk), *R2 = qalloc(kk), *T = qalloc(kk);
  q_gram_sym(n, k, X, ldx, M);
  const int r = q_pivchol(k, M, (qreal)tol, perm, R);
  /* R11^{-1} (rank-by-rank upper triangular), placed at the pivots' rows */
  for (int j = 0; j < r; ++j) {
    Zs[(size_t)j * k + j] = 1 / R[(size_t)j * k + j];
    for (int i = j - 1; i >= 0; --i) {
      qreal s = 0;
      for (int l = i + 1; l <= j; ++l) s += R[(size_t)l * k + i] * Zs[(size_t)j * k + l];
      Zs[(size_t)j * k + i] = -s / R[(size_t)i * k + i];
    }
  }
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < r; ++i) Z[(size_t)j * k + perm[i]] = Zs[(size_t)j * k + i];
  q_update(n, k, X, ldx, Z);
  int info = 0;
  if (passes == 2 && r > 0) {
    q_gram_sym(n, k, X, ldx, M);
    qreal* Ml = qalloc((size_t)r * r);
    for (int j = 0; j < r; ++j)
      for (int i = 0; i < r; ++i) Ml[(size_t)j * r + i] = M[(size_t)j * k + i];
    qreal *Rr = qalloc((size_t)r * r), *Zr = qalloc((size_t)r * r);
    info = q_cholesky(r, Ml, Rr);
    if (!info) {
      q_triinv(r, Rr, Zr);
      for (size_t t = 0; t < kk; ++t) Z[t] = 0;
      for (int j = 0; j < r; ++j)
        for (int i = 0; i < r; ++i) {
          Z[(size_t)j * k + i] = Zr[(size_t)j * r + i];
          R2[(size_t)j * k + i] = Rr[(size_t)j * r + i];
        }
      q_update(n, k, X, ldx, Z);
      for (int j = 0; j < k; ++j) /* R <- R2 R (R2 upper rank-by-rank, R upper trapezoidal) */
        for (int i = 0; i < k; ++i) {
          qreal s = 0;
          for (int l = 0; l < r; ++l) s += R2[(size_t)l * k + i] * R[(size_t)j * k + l];
          T[(size_t)j * k + i] = i < r ? s : 0;
        }
      memcpy(R, T, sizeof(qreal) * kk);
    }
    free(Ml); free(Rr); free(Zr);
  }
  if (R_hi) store_dd(k, R, R_hi, R_lo, ldr);
  if (rank_out) *rank_out = r;
  free(M); free(R); free(Z); free(Zs); free(R2); free(T);
  return info;
}

/* ------------------------------------------ iterated two-phase algorithm */

/* The iterated orthogonalization of Sec. 4.2: the two phases are repeated in
 * turn until both orthogonality measures are at or below eps (the runtime
 * figure repeats them to eps = 1e-10).  Iteration it (0-based):
 *   phase I   C = W^T Y (binary128), Y <- Y - W C (binary128, rounded once);
 *   measure   M = Y^T Y of the rounded Y (binary128),
 *             e = max(||C||_F, ||M - I||_F)  (the Frobenius norm bounds the
 *             2-norm from above, so e <= eps certifies both 2-norm measures);
 *   stop      if e <= eps: return it, the number of phase-II updates applied;
 *   phase II  Z = M^{-1/2} with eigenvalue cut tol (the SVQB transform of
 *             q_svqb_z), Y <- Y Z (binary128, rounded once).
 * Returns -max_iter when e > eps after max_iter iterations.  *rank_out gets
 * the rank of the last SVQB applied (k when none was). */
int eoq_orthogonalize(int64_t n, int kv, const double* W, int64_t ldw, int k, double* Y, int64_t ldy, double eps,
                      int max_iter, double tol, int* rank_out) {
  size_t kk = (size_t)k * k;
  qreal *C = qalloc((size_t)kv * k), *M = qalloc(kk), *Z = qalloc(kk);
  int rank = k, iters = -max_iter;
  for (int it = 0; it < max_iter; ++it) {
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int i = 0; i < kv; ++i)
      for (int j = 0; j < k; ++j) {
        qreal s = 0;
        for (int64_t r = 0; r < n; ++r) s += (qreal)AT(W, ldw, r, i) * (qreal)AT(Y, ldy, r, j);
        C[(size_t)j * kv + i] = s;
      }
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r)
      for (int j = 0; j < k; ++j) {
        qreal s = (qreal)AT(Y, ldy, r, j);
        for (int i = 0; i < kv; ++i) s -= (qreal)AT(W, ldw, r, i) * C[(size_t)j * kv + i];
        AT(Y, ldy, r, j) = (double)s;
      }
    q_gram_sym(n, k, Y, ldy, M);
    qreal ec = 0, em = 0;
    for (size_t t = 0; t < (size_t)kv * k; ++t) ec += C[t] * C[t];
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        qreal e = M[(size_t)j * k + i] - (i == j ? 1 : 0);
        em += e * e;
      }
    ec = qsqrt(ec);
    em = qsqrt(em);
    if ((ec > em ? ec : em) <= (qreal)eps) {
      iters = it;
      break;
    }
    rank = q_svqb_z(k, M, (qreal)tol, Z);
    q_update(n, k, Y, ldy, Z);
  }
  if (rank_out) *rank_out = rank;
  free(C); free(M); free(Z);
  return iters;
}

/* ------------------------------------------------------- B-inner products */

/* M = (X^T P + P^T X) / 2: the Gram matrix of <x, y>_B = x^T B y from the
 * given P = B X (the two triangles of X^T P differ only by the rounding of P). */
static void q_gram_b(int64_t n, int k, const double* X, int64_t ldx, const double* P, int64_t ldp, qreal* M) {
  qreal* G = qalloc((size_t)k * k);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(X, ldx, r, i) * (qreal)AT(P, ldp, r, j);
      G[(size_t)j * k + i] = s;
    }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) M[(size_t)j * k + i] = (G[(size_t)j * k + i] + G[(size_t)i * k + j]) / 2;
  free(G);
}

/* B-CholQR: per pass, M = sym(X^T P), M = R^T R, Z = R^{-1}, X <- X Z and
 * P <- P Z (each rounded once).  Returns 0 or the breakdown column. */
int eoq_cholqr_b(int64_t n, int k, double* X, int64_t ldx, double* P, int64_t ldp, int passes, double* R_hi,
                 double* R_lo, int ldr) {
  size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *R = qalloc(kk), *Z = qalloc(kk), *Rt = qalloc(kk), *T = qalloc(kk);
  for (int i = 0; i < k; ++i) Rt[(size_t)i * k + i] = 1;
  int info = 0;
  for (int p = 0; p < passes; ++p) {
    q_gram_b(n, k, X, ldx, P, ldp, M);
    info = q_cholesky(k, M, R);
    if (info) break;
    q_triinv(k, R, Z);
    q_update(n, k, X, ldx, Z);
    q_update(n, k, P, ldp, Z);
    q_trmul(k, R, Rt, T);
    memcpy(Rt, T, sizeof(qreal) * kk);
  }
  if (R_hi) store_dd(k, Rt, R_hi, R_lo, ldr);
  free(M); free(R); free(Z); free(Rt); free(T);
  return info;
}

/* B-SVQB: per pass, M = sym(X^T P), Z = M^{-1/2}, X <- X Z, P <- P Z.
 * Z_out gets the product of the passes' transforms; returns the last rank. */
int eoq_svqb_b(int64_t n, int k, double* X, int64_t ldx, double* P, int64_t ldp, double tol, int passes,
               double* Z_hi, double* Z_lo, int ldz) {
  size_t kk = (size_t)k * k;
  qreal *M = qalloc(kk), *Z = qalloc(kk), *Zt = qalloc(kk), *T = qalloc(kk);
  for (int i = 0; i < k; ++i) Zt[(size_t)i * k + i] = 1;
  int rank = k;
  for (int p = 0; p < passes; ++p) {
    q_gram_b(n, k, X, ldx, P, ldp, M);
    rank = q_svqb_z(k, M, (qreal)tol, Z);
    q_update(n, k, X, ldx, Z);
    q_update(n, k, P, ldp, Z);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        qreal s = 0;
        for (int l = 0; l < k; ++l) s += Zt[(size_t)l * k + i] * Z[(size_t)j * k + l];
        T[(size_t)j * k + i] = s;
      }
    memcpy(Zt, T, sizeof(qreal) * kk);
  }
  if (Z_hi) store_dd(k, Zt, Z_hi, Z_lo, ldz);
  free(M); free(Z); free(Zt); free(T);
  return rank;
}

/* B-projection against a B-orthonormal W with BW = B W: C = (BW)^T X,
 * X <- X - W C and P <- P - BW C (each entry summed in binary128 and rounded
 * once, in place), then M = sym(X^T P) of the rounded results.  C and M leave
 * as double-double pairs (M_hi may be NULL). */
void eoq_project_b(int64_t n, int kv, const double* W, int64_t ldw, const double* BW, int64_t ldbw, int k,
                   double* X, int64_t ldx, double* P, int64_t ldp, double* C_hi, double* C_lo, int ldc,
                   double* M_hi, double* M_lo, int ldm) {
  qreal* C = qalloc((size_t)kv * k);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kv; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(BW, ldbw, r, i) * (qreal)AT(X, ldx, r, j);
      C[(size_t)j * kv + i] = s;
    }
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r)
    for (int j = 0; j < k; ++j) {
      qreal sx = (qreal)AT(X, ldx, r, j), sp = (qreal)AT(P, ldp, r, j);
      for (int i = 0; i < kv; ++i) {
        sx -= (qreal)AT(W, ldw, r, i) * C[(size_t)j * kv + i];
        sp -= (qreal)AT(BW, ldbw, r, i) * C[(size_t)j * kv + i];
      }
      AT(X, ldx, r, j) = (double)sx;
      AT(P, ldp, r, j) = (double)sp;
    }
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < kv; ++i) q_to_dd(C[(size_t)j * kv + i], &AT(C_hi, ldc, i, j), &AT(C_lo, ldc, i, j));
  if (M_hi) {
    qreal* M = qalloc((size_t)k * k);
    q_gram_b(n, k, X, ldx, P, ldp, M);
    store_dd(k, M, M_hi, M_lo, ldm);
    free(M);
  }
  free(C);
}

/* --------------------------------------------------------------- measures */

/* ||Q^T D Q - I|| (2-norm, Frobenius, max-abs) for a diagonal B = diag(d), in binary128. */
void eoq_orth_err_diag(int64_t n, int k, const double* Q, int64_t ldq, const double* d, double* out);

/* E = Q^T Q - I in binary128; out[0] = ||E||_2 (largest |eigenvalue| of the
 * symmetric E, by Jacobi), out[1] = ||E||_F, out[2] = max |E_ij|. */
static void q_err_norms(int k, qreal* E, double* out);

void eoq_orth_err(int64_t n, int k, const double* Q, int64_t ldq, double* out) {
  qreal* E = qalloc((size_t)k * k);
  q_gram_sym(n, k, Q, ldq, E);
  q_err_norms(k, E, out);
  free(E);
}

void eoq_orth_err_diag(int64_t n, int k, const double* Q, int64_t ldq, const double* d, double* out) {
  qreal* E = qalloc((size_t)k * k);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(Q, ldq, r, i) * (qreal)d[r] * (qreal)AT(Q, ldq, r, j);
      E[(size_t)j * k + i] = s;
    }
  q_err_norms(k, E, out);
  free(E);
}

/* out = (||E - I||_2, ||E - I||_F, max |E - I|) for a symmetric k-by-k E (overwritten). */
static void q_err_norms(int k, qreal* E, double* out) {
  size_t kk = (size_t)k * k;
  qreal *U = qalloc(kk), *lam = qalloc(k);
  for (int i = 0; i < k; ++i) E[(size_t)i * k + i] -= 1;
  qreal fro = 0, mx = 0;
  for (size_t t = 0; t < kk; ++t) {
    fro += E[t] * E[t];
    if (qabs(E[t]) > mx) mx = qabs(E[t]);
  }
  q_jacobi(k, E, U, lam);
  qreal two = 0;
  for (int i = 0; i < k; ++i) if (qabs(lam[i]) > two) two = qabs(lam[i]);
  out[0] = (double)two;
  out[1] = (double)qsqrt(fro);
  out[2] = (double)mx;
  free(U); free(lam);
}

/* ||W^T Q||_2 = sqrt(largest eigenvalue of (W^T Q)^T (W^T Q)), binary128. */
double eoq_cross_err(int64_t n, int kv, const double* W, int64_t ldw, int k, const double* Q, int64_t ldq) {
  qreal *C = qalloc((size_t)kv * k), *G = qalloc((size_t)k * k), *U = qalloc((size_t)k * k), *lam = qalloc(k);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int i = 0; i < kv; ++i)
    for (int j = 0; j < k; ++j) {
      qreal s = 0;
      for (int64_t r = 0; r < n; ++r) s += (qreal)AT(W, ldw, r, i) * (qreal)AT(Q, ldq, r, j);
      C[(size_t)j * kv + i] = s;
    }
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      qreal s = 0;
      for (int l = 0; l < kv; ++l) s += C[(size_t)i * kv + l] * C[(size_t)j * kv + l];
      G[(size_t)j * k + i] = s;
    }
  q_jacobi(k, G, U, lam);
  qreal mx = 0;
  for (int i = 0; i < k; ++i) if (lam[i] > mx) mx = lam[i];
  double r = (double)qsqrt(mx);
  free(C); free(G); free(U); free(lam);
  return r;
}

/* ||X - Q R||_F / ||X||_F with R = R_hi + R_lo upper triangular, binary128. */
double eoq_fact_err(int64_t n, int k, const double* X, int64_t ldx, const double* Q, int64_t ldq,
                    const double* R_hi, const double* R_lo, int ldr) {
  qreal num = 0, den = 0;
  for (int64_t r = 0; r < n; ++r)
    for (int j = 0; j < k; ++j) {
      qreal s = (qreal)AT(X, ldx, r, j);
      den += s * s;
      for (int i = 0; i <= j; ++i) s -= (qreal)AT(Q, ldq, r, i) * dd_to_q(R_hi, R_lo, (size_t)j * ldr + i);
      num += s * s;
    }
  return (double)qsqrt(num / den);
}
