/*
 * eo.h — block orthogonalization on one GPU (NVIDIA GB300, sm_103a).
 *
 * The operations are those of the two-phase orthogonalization of
 * arXiv:1806.01036, Sec. 4.2 ("Using higher precision for robust and fast
 * orthogonalization"): given a block X (n-by-k) and an orthonormal basis W
 * (n-by-kv; called V here), phase I forms Y~ = (I - V V^T) X, phase II builds
 * the Gram matrix M = Y~^T Y~, finds Z with Z^T M Z = I (Cholesky: Z = R^{-1};
 * SVQB: Z from M = U Lambda U^T) and returns Y = Y~ Z.  Each call runs in one
 * of three precisions (eo_prec): plain FP64, FP64 data with double-double
 * ("DD") accumulation as in the paper's DD kernels, or FP32 data with FP64
 * accumulation.
 *
 * Conventions shared by every call
 *  - Matrices are column-major with a leading dimension (ld*) >= rows.  Large
 *    matrices (n rows) are DEVICE pointers; they are borrowed, never freed.
 *  - Small matrices (k-by-k, kv-by-k) passed in or out are DEVICE pointers.
 *    A double-double value is the unevaluated sum hi + lo of two FP64 arrays
 *    with the same layout; every *_lo pointer may be NULL when the low part is
 *    not wanted (in FP64 and F32 modes the low parts are written as zero).
 *  - Calls are asynchronous on the context's stream (eo_set_stream) and may
 *    be captured in a CUDA graph once a first call of the same shape has run
 *    outside capture (the first call may grow the context's scratch memory).
 *  - The return value reports argument and CUDA errors only.  Numerical
 *    outcomes (Cholesky breakdown, SVQB rank) are written to device memory so
 *    that no call synchronizes with the host.
 *  - Sizes: 1 <= k, kv <= 64; n >= 0.  A context is not thread-safe; use one
 *    per host thread.
 *  - Ownership: the context owns its scratch memory (grown on demand, freed by
 *    eo_destroy); the caller owns every pointer it passes.
 */
#ifndef EO_H
#define EO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EO_KMAX 64

#if defined(__GNUC__)
#define EO_API __attribute__((visibility("default")))
#else
#define EO_API
#endif

/* Arithmetic of a call (Sec. 4.2: FP64 vs DD kernels; the FP32-input mode
 * is the building block of the single-precision iterations of Sec. 4.1). */
typedef enum {
  EO_FP64 = 0,   /* FP64 data, FP64 accumulation                                  */
  EO_DD = 1,     /* FP64 data, compensated accumulation (>= double-double accuracy),
                    results rounded once; the sums are formed exactly in fixed
                    point, on the tensor cores or the integer pipe (see below)     */
  EO_F32 = 2,    /* FP32 data (float*), FP64 accumulation of the exact products    */
  EO_DD_EFT = 3  /* as EO_DD, but the sums use the paper's FP64 error-free
                    transformations (TwoProd + TwoSum) on the FP64 pipe           */
} eo_prec;

/* EO_DD accuracy: each group of values summed against another (a column of a
 * block of rows, a row of V or X, a column of C or Z) is aligned to an
 * exponent at or above its largest and held as a 104-bit integer (four
 * 26-bit limbs; the ten most significant limb products are kept) or, in Gram
 * products with 16 or more columns on one side, as a 105-bit integer of
 * fifteen balanced 7-bit digits whose products are summed on the tensor cores
 * (FP16 integer digits, exact FP32 sums; the 120 most significant digit pairs
 * are kept; a column's alignment exponent sits up to two binades above its
 * largest, so that it rarely has to grow).  Each product then carries an
 * error below 2^-101 max|x| max|y| (integer limbs) or 2^-96 max|x| max|y|
 * (tensor-core digits), the sums of the kept products are exact, and every
 * result is rounded once.  Exact sums are
 * associative: the order of the partial sums does not matter, and the same
 * inputs give bitwise the same results on every run.  A bounded wait inside
 * the tensor-core kernels that runs out (2 s) turns the affected outputs
 * into NaN instead of hanging, and eo_device_status reports it. */

typedef enum {
  EO_OK = 0,
  EO_EINVAL = 1,      /* bad argument (size, leading dimension, NULL pointer, mode) */
  EO_ENOMEM = 2,      /* scratch allocation failed                                   */
  EO_ECUDA = 3,       /* a CUDA call or kernel launch failed (see eo_last_error)     */
  EO_ETIMEOUT = 4,    /* a bounded wait expired (eo_device_status, eo_server_wait)    */
  EO_EUNSUPPORTED = 5 /* valid but not implemented combination                       */
} eo_status;

typedef struct eo_ctx eo_ctx;

/* Create a context on CUDA device `device` (made current for the call).
 * The context starts on the legacy default stream. */
EO_API eo_status eo_create(eo_ctx** ctx, int device);
EO_API eo_status eo_destroy(eo_ctx* ctx);
/* Borrow a cudaStream_t for all later calls (NULL = default stream). */
EO_API eo_status eo_set_stream(eo_ctx* ctx, void* cuda_stream);
/* Text of the last error on this context ("" if none).  Owned by the context. */
EO_API const char* eo_last_error(const eo_ctx* ctx);
EO_API int eo_version(void);
/* Number of kernels this context has launched so far (diagnostics). */
EO_API uint64_t eo_kernel_launches(const eo_ctx* ctx);
/* Device-side failure record (no counterpart in the paper).  Every wait
 * inside the tensor-core kernels (TMA arrival, MMA completion, converted
 * digits) is bounded (2 s); a wait that runs out makes its kernel finish
 * early with NaN outputs and records the expiry in a word on the device.
 * eo_device_status waits for the context's stream, then returns EO_ETIMEOUT
 * (with a message in eo_last_error) if such a record exists on the
 * context's device, clearing it, and EO_OK otherwise.  The record is per
 * device, shared by every context on it.
 * eo_selftest_wait_timeout launches, on the context's stream, one kernel
 * whose single thread waits on an mbarrier that nothing completes, bounded
 * by `seconds` (0 < seconds <= 2): it exercises the same bounded-wait path,
 * so the next eo_device_status reports EO_ETIMEOUT; the context stays
 * usable. */
EO_API eo_status eo_device_status(eo_ctx* ctx);
EO_API eo_status eo_selftest_wait_timeout(eo_ctx* ctx, double seconds);

/*
 * Gram product G = X^T Y (kx-by-ky), the matrix-matrix product that carries
 * most of the arithmetic of phase II (Sec. 4.2, M = Y~^T Y~) and, with
 * Y = X and X = W, the W^T X of phase I.
 *   X: n-by-kx, Y: n-by-ky (Y == NULL: Y = X and ky must equal kx; G is then
 *   symmetric and both triangles are written).  FP64 data, or float data in
 *   EO_F32 mode.  G_hi (required) / G_lo: kx-by-ky with leading dimension ldg.
 * EO_DD: every G_ij is the double-double rounding of the sum of the exact
 * products (error below 2^-104 |G_ij| + n 2^-96 max|x_i| max|y_j|, see the
 * accuracy note above); results are bitwise reproducible.
 */
EO_API eo_status eo_gram(eo_ctx* ctx, int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y, int64_t ldy,
                  double* G_hi, double* G_lo, int ldg, eo_prec prec);

/*
 * Phase I projection against an orthonormal basis V (Sec. 4.2:
 * Y~ = (I - W W^T) X), optionally with the phase-II Gram matrix of the result.
 *   V: n-by-kv, Y: n-by-k (FP64).  C = V^T Y is written to C_hi/C_lo (kv-by-k,
 *   ldc; C_hi may be NULL).  Yout (n-by-k, ldyo) receives Y - V C, rounded
 *   once to FP64; Yout may equal Y (in place) but must not otherwise overlap
 *   it.  If M_hi != NULL, M = Yout^T Yout of the rounded result (k-by-k, ldm)
 *   is computed too: in EO_FP64 and EO_DD_EFT in the same pass over the data
 *   as the projection (the paper fuses these two kernels), in EO_DD by a
 *   second tensor-core Gram pass over Yout (the exact fused form does not fit
 *   one SM's tensor memory next to the projection's accumulators).
 * EO_F32 is not supported (EO_EUNSUPPORTED).
 */
EO_API eo_status eo_project(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                     int64_t ldy, double* Yout, int64_t ldyo, double* C_hi, double* C_lo, int ldc, double* M_hi,
                     double* M_lo, int ldm, eo_prec prec);

/*
 * The second half of phase I for a given C (Sec. 4.2: Y~ = X - W (W^T X)):
 * Yout = Y - V C with C = C_hi + C_lo (kv-by-k, ldc; C_lo may be NULL), and,
 * if M_hi != NULL, M = Yout^T Yout of the rounded result.  eo_project is
 * eo_gram(V, Y) followed by this call; calling the two separately lets a
 * caller reuse or inspect C.  Layout, aliasing and modes as in eo_project.
 */
EO_API eo_status eo_project_apply(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k,
                                  const double* Y, int64_t ldy, double* Yout, int64_t ldyo, const double* C_hi,
                                  const double* C_lo, int ldc, double* M_hi, double* M_lo, int ldm, eo_prec prec);

/*
 * Cholesky QR (Sec. 4.2: M = R^T R, Z = R^{-1}, Y = Y~ Z): X <- Q in place.
 *   X: n-by-k (FP64, or float in EO_F32 mode), ldx.
 *   M_hi/M_lo: optional Gram matrix of X for the first pass (as produced by
 *   eo_project's fused pass); NULL = compute it.
 *   R_hi/R_lo: optional k-by-k outputs (ldr): upper-triangular R with positive
 *   diagonal and X_in = Q R (R is the product of the passes' factors).
 *   passes: 1 or 2, or 0 = automatic (a second pass runs, on the device, when
 *   the first factor's diagonal ratio max R_ii / min R_ii exceeds 1e4 in
 *   EO_FP64/EO_F32 or 1e7 in EO_DD).
 *   info_dev: optional device int: 0 on success, j >= 1 if the j-th pivot of a
 *   pass was not positive (X then keeps the last completed pass), -1 if M had a
 *   NaN or Inf.
 */
EO_API eo_status eo_cholqr(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi, const double* M_lo,
                    int ldm, double* R_hi, double* R_lo, int ldr, int passes, eo_prec prec, int* info_dev);

/*
 * Pivoted, partial CholQR (Sec. 4.2: the Cholesky factorization of phase II
 * may be pivoted and partial, which makes it rank-revealing): X <- Q in
 * place.  Pass 1 factors M = X^T X with diagonal pivoting -- each step takes
 * the largest remaining diagonal entry (lowest index on ties) -- and stops
 * at the numerical rank r, when that entry is not above tol times the
 * largest diagonal entry of M (tol < 0 selects k * 2^-104 in EO_DD,
 * k * 2^-52 in EO_FP64 and EO_DD_EFT); then X <- X P [R11^{-1}, 0; 0, 0]:
 * Q's first r columns are orthonormal and span X's numerical range, the
 * others are zero.  Pass 2 (passes = 2, or passes = 0 and the pivoted
 * diagonal ratio R_11 / R_rr above 1e7 in EO_DD, 1e4 otherwise) repeats the
 * Cholesky on the leading r columns without pivoting.
 *   X: n-by-k FP64, ldx.  R_hi/R_lo: optional k-by-k outputs (ldr): upper
 *   trapezoidal, rows >= r zero, X(:, perm) = Q R up to rounding.
 *   perm_dev: optional device int[k], the pivot order (X's column perm[j]
 *   was factored at step j).  rank_dev: optional device int, r (-1 if M had
 *   a NaN or Inf).  info_dev: optional device int, 0, -1 (NaN or Inf: X is
 *   left as it was) or j >= 1 if the second pass broke down at column j (X
 *   keeps the first pass).  EO_F32 is not supported.
 */
EO_API eo_status eo_cholqr_piv(eo_ctx* ctx, int64_t n, int k, double* X, int64_t ldx, double* R_hi, double* R_lo,
                               int ldr, double tol, int passes, eo_prec prec, int* perm_dev, int* rank_dev,
                               int* info_dev);

/*
 * SVQB (Sec. 4.2: M = U Lambda U^T, Y = Y~ Z): X <- X Z in place with the
 * symmetric Z = U Lambda^{-1/2} U^T = M^{-1/2}, the solution of
 * min ||Z - I||_F subject to Z^T M Z = I (the Procrustes argument of the same
 * section).  Eigenvalues at or below tol * lambda_max are treated as zero
 * (Z uses the pseudo-inverse square root, and the result spans the numerical
 * range of X); tol < 0 selects k * 2^-52 (FP64, F32) or k * 2^-104 (DD).
 *   M_hi/M_lo: optional Gram matrix for the first pass (NULL = compute).
 *   Z_hi/Z_lo: optional k-by-k output (ldz), the product of the passes' Z.
 *   passes: 1 or 2 (0 = automatic as in eo_cholqr, from lambda_max/lambda_min).
 *   rank_dev: optional device int, the number of eigenvalues kept in the
 *   last pass, or -1 if M had a NaN or Inf.
 */
EO_API eo_status eo_svqb(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi, const double* M_lo,
                  int ldm, double* Z_hi, double* Z_lo, int ldz, double tol, int passes, eo_prec prec, int* rank_dev);

/*
 * SVQB in its rotated form (Sec. 4.2 with the scaling of the SVQB of
 * Stathopoulos and Wu, 2002): one pass of X <- X Z with
 * Z = D U Lambda^{-1/2}, where D = diag(M)^{-1/2} (d_i = 0 where M_ii <= 0)
 * and D M D = U Lambda U^T.  The columns of Z follow the eigenvalues in
 * ascending order (equal ones by index), each eigenvector's largest-magnitude
 * entry (lowest row on ties) is positive, and the columns of eigenvalues at
 * or below tol * lambda_max (of D M D) are zero.  Z^T M Z is the identity on
 * the kept columns; unlike eo_svqb's Z, this one is not symmetric and is not
 * the Frobenius-nearest to I, and Q spans the same space with its columns
 * rotated.  Arguments, tol < 0, layout, modes and rank_dev as in eo_svqb;
 * Z_hi/Z_lo (optional, ldz) receive Z.
 */
EO_API eo_status eo_svqb_rotated(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi,
                                 const double* M_lo, int ldm, double* Z_hi, double* Z_lo, int ldz, double tol,
                                 eo_prec prec, int* rank_dev);

/*
 * Iterated two-phase orthogonalization (Sec. 4.2: the two phases are
 * repeated in turn, with a rank-revealing factorization in phase II, which
 * makes the method robust; the runtime figure repeats them until both
 * measures fall below epsilon = 1e-10).  Each iteration runs phase I
 * (C = V^T Y, Y <- Y - V C) and measures ||C||_F and ||M - I||_F with
 * M = Y^T Y of the projected block (the Frobenius norm bounds the 2-norm from
 * above, so a stop certifies ||V^T Y||_2 <= eps and ||Y^T Y - I||_2 <= eps
 * for the C and M computed); when both are <= eps the iteration stops there,
 * otherwise phase II applies SVQB (Z = M^{-1/2} with eigenvalue cut tol, as
 * in eo_svqb) and the next iteration follows.  Y (n-by-k, FP64) is updated
 * in place; V (n-by-kv) must be orthonormal.  All max_iter iterations
 * (1..16) are enqueued at once and skipped on the device after convergence.
 *   iters_dev: optional device int, the number of SVQB updates applied before
 *   convergence was seen, or -max_iter if it was not seen.
 *   rank_dev: optional device int, the rank of the last SVQB applied (k when
 *   none was needed).
 * EO_F32 is not supported.
 */
EO_API eo_status eo_orthogonalize(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, double* Y,
                                  int64_t ldy, double eps, int max_iter, double tol, eo_prec prec, int* iters_dev,
                                  int* rank_dev);

/*
 * B-inner products (Sec. 4.2, closing remark: the technique extends to
 * <x, y>_B = x^T B y, as needed for generalized eigenproblems).  B is
 * symmetric positive definite and is never applied here: the caller passes
 * P = B X next to X (the product with B is the caller's, e.g. a sparse
 * matrix-vector product).  The Gram matrix is M = (X^T P + P^T X) / 2 (the
 * two triangles of X^T P differ only by the rounding of P), and every
 * transform Z applied to X is applied to P as well, so on return P = B Q up
 * to rounding and Q^T B Q = I.  Layout, passes, modes and outputs as in
 * eo_cholqr / eo_svqb / eo_project; X and BX (Y and BY) must not alias.
 *   eo_cholqr_b:  X <- Q, BX <- BX R^{-1} per pass; R_hi/R_lo, info_dev.
 *   eo_svqb_b:    X <- X Z, BX <- BX Z with Z = M^{-1/2}; Z_hi/Z_lo, rank_dev.
 *   eo_project_b: against a B-orthonormal W given with BW = B W:
 *                 C = BW^T Y, Y <- Y - W C, BY <- BY - BW C (in place), and
 *                 optionally M = sym(Y^T BY) of the results.  FP64 data only.
 */
EO_API eo_status eo_cholqr_b(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, void* BX, int64_t ldbx,
                             double* R_hi, double* R_lo, int ldr, int passes, eo_prec prec, int* info_dev);
EO_API eo_status eo_svqb_b(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, void* BX, int64_t ldbx,
                           double* Z_hi, double* Z_lo, int ldz, double tol, int passes, eo_prec prec, int* rank_dev);
EO_API eo_status eo_project_b(eo_ctx* ctx, int64_t n, int kv, const double* W, int64_t ldw, const double* BW,
                              int64_t ldbw, int k, double* Y, int64_t ldy, double* BY, int64_t ldby, double* C_hi,
                              double* C_lo, int ldc, double* M_hi, double* M_lo, int ldm, eo_prec prec);

/*
 * Batched orthogonalization (no counterpart in the paper, whose solvers
 * orthogonalize one block at a time): many independent blocks of uneven n and
 * k, each orthogonalized by the kernels of one eo_svqb (EO_BATCH_SVQB) or
 * eo_cholqr (EO_BATCH_CHOLQR) call with the same tol, passes and prec,
 * captured once into a CUDA graph and run by one graph launch.  With the
 * default launch shapes (EO_BATCH_NO_TUNE, and always outside EO_DD) every
 * block's result is bitwise that of the single call.  Tuned shapes split a
 * block's rows into other chunks; each chunk aligns its sums to its own
 * exponents, so the results move within the EO_DD error bound (last bits of
 * the low parts) and are again bitwise reproducible for that shape.  A
 * block's shape depends only on its own (k, n) and the context's tuned caps,
 * never on the other blocks: a result is the same alone and in any mix.
 *
 * eo_batch_create checks the blocks, picks the launch shapes, spreads the
 * blocks over `branches` concurrent graph branches (0 = min(nblocks, 16);
 * at most 64), allocates one device workspace per block (about 200 KB) and
 * captures the graph.  It launches nothing on the context's stream, but in
 * EO_DD it may run the autotuner first (below), which launches and
 * synchronizes on a private stream.  The blocks' pointers are captured: the
 * batch must be destroyed before any block's memory is freed.
 *   blocks: host array of nblocks descriptors (read during the call only).
 *   out_dev: optional device int[nblocks]: per block the rank (SVQB) or the
 *   info (CholQR) of the single call.
 *   flags: EO_BATCH_NO_TUNE = default launch shapes, no autotuning;
 *   EO_BATCH_CHAINS = each block's whole sequence on its branch (default:
 *   by phase -- the blocks' Gram matrices of a pass on the branches, then all
 *   their k-by-k factorizations in one launch of one CTA per block, then the
 *   updates on the branches; the factorizations, which run on one SM each,
 *   then spread over every SM).  Both give the same results.
 * eo_batch_run enqueues one launch of the graph on the context's stream; it
 * may be called any number of times (each run orthogonalizes the blocks'
 * current contents in place).  eo_batch_destroy waits for the context's
 * stream and frees the batch.
 *
 * Autotuner (EO_DD): the Gram and update kernels of a block run with a cap on
 * their CTAs, picked per (k, floor(log2 n)) for n >= 4096 by timing both
 * kernels on a synthetic n-by-k buffer for a coarse set of caps and then
 * around the best, keeping the cap with the least SM time (CTAs x duration)
 * and preferring more CTAs within 5 %.  Tuned caps are kept in the context;
 * eo_tune_cache(ctx, path) also loads them from, and saves new ones to, a
 * text file (one line per key, tagged with the device name; NULL = memory
 * only).
 */
typedef struct eo_block {
  int64_t n;      /* rows (>= 0)                                             */
  int k;          /* columns, 1..EO_KMAX                                     */
  void* X;        /* device, column-major n-by-k (float* in EO_F32), in place */
  int64_t ldx;    /* >= max(1, n)                                            */
  double* Z_hi;   /* optional k-by-k output: Z (SVQB) or R (CholQR)          */
  double* Z_lo;   /* optional low part                                       */
  int ldz;        /* >= k when Z_hi or Z_lo is given                         */
} eo_block;

typedef enum { EO_BATCH_SVQB = 0, EO_BATCH_CHOLQR = 1 } eo_batch_method;
#define EO_BATCH_NO_TUNE 1
#define EO_BATCH_CHAINS 2

typedef struct eo_batch eo_batch;

EO_API eo_status eo_tune_cache(eo_ctx* ctx, const char* path);
EO_API eo_status eo_batch_create(eo_ctx* ctx, int nblocks, const eo_block* blocks, eo_batch_method method,
                                 double tol, int passes, eo_prec prec, int* out_dev, int branches, int flags,
                                 eo_batch** batch);
EO_API eo_status eo_batch_run(eo_batch* batch);
EO_API eo_status eo_batch_destroy(eo_batch* batch);
/* CTA caps chosen for a block (0 = default shape). */
EO_API eo_status eo_batch_tile(const eo_batch* batch, int block, int* gram_ctas, int* row_ctas);
/* Passes each block took in the last run (1 or 2) into host int[nblocks];
 * waits for the context's stream. */
EO_API eo_status eo_batch_passes(eo_batch* batch, int* passes_host);
/* Jacobi sweeps of each block's last SVQB eigensolve in the last run (0 for
 * CholQR; at most 40) into host int[nblocks]; waits for the context's stream. */
EO_API eo_status eo_batch_sweeps(eo_batch* batch, int* sweeps_host);
/* Kernels one eo_batch_run launches (-1 for NULL), and the graph's branches. */
EO_API int64_t eo_batch_kernels(const eo_batch* batch);
EO_API int eo_batch_branches(const eo_batch* batch);

/*
 * Request server (no counterpart in the paper): many concurrent eigensolves
 * keep their bases V resident on the device and submit blocks Y to be
 * orthogonalized against them -- Yout = Y - V (V^T Y) followed by the
 * compensated CholQR of Yout with the automatic second pass, as
 * eo_project(..., M) + eo_cholqr(..., M, passes = 0, EO_DD) would do.
 *
 * A server thread admits queued requests onto `slots` streams (each with
 * its own workspace, reserved up front) in submission order, one request at
 * a time per basis, as soon as a slot is free and the device-memory budget
 * allows: registered bases (n kv 8 bytes) and the slots' workspaces stay
 * charged; a running request is charged for its block (n k 8 bytes, twice
 * when Yout != Y).  Requests that arrive while others run join as slots and
 * memory free up, and their kernels overlap on the GPU.  The first queued
 * request that does not fit stops admission until memory frees (no
 * overtaking on memory); a request blocked by its basis is passed over.
 * Every slot uses the default launch shapes, so a result is bitwise the same
 * alone and in any mix.
 *
 * eo_server_create: budget in bytes; slots in [1, 256]; starts the server
 *   thread.  The context only reports errors; it is not used for work.
 * eo_server_add_basis: registers V (device, n-by-kv, ldv; owned by the
 *   caller, unchanged while the server lives); EO_ENOMEM if it does not fit
 *   the budget.  May synchronize (it grows the slots' scratch).
 * eo_server_submit: queues a request; thread-safe and non-blocking.  Y and
 *   Yout: device n-by-k blocks (Yout may equal Y); R_hi/R_lo (k-by-k, ldr),
 *   info_dev: optional outputs as in eo_cholqr.  EO_ENOMEM if the block can
 *   never fit next to the resident bases.
 * eo_server_wait: blocks until the request is done (EO_ETIMEOUT after
 *   timeout_s seconds); *status = EO_OK or EO_ECUDA; *latency_ms = time from
 *   submission to the end of its last kernel.
 * eo_server_poll: up to max_out completed requests not yet reported, with
 *   their latency and time spent queued (ms).
 * eo_server_stats: resident bytes, peak in-flight bytes, peak requests
 *   running at once, requests queued and running now, kernels launched by
 *   the slots so far (any pointer may be NULL).
 * eo_server_destroy: stops the thread, waits for the slots, frees them.
 */
typedef struct eo_server eo_server;
EO_API eo_status eo_server_create(eo_ctx* ctx, size_t hbm_budget, int slots, eo_server** server);
EO_API eo_status eo_server_destroy(eo_server* server);
EO_API eo_status eo_server_add_basis(eo_server* server, int64_t n, int kv, const double* V, int64_t ldv,
                                     int* basis_id);
EO_API eo_status eo_server_submit(eo_server* server, int basis_id, int k, const double* Y, int64_t ldy, double* Yout,
                                  int64_t ldyo, double* R_hi, double* R_lo, int ldr, int* info_dev, int64_t* req_id);
EO_API eo_status eo_server_wait(eo_server* server, int64_t req_id, double timeout_s, int* status, double* latency_ms);
EO_API eo_status eo_server_poll(eo_server* server, int max_out, int64_t* ids, double* latency_ms, double* queue_ms,
                                int* statuses, int* n_out);
EO_API eo_status eo_server_stats(eo_server* server, size_t* resident, size_t* peak_inflight, int* peak_running,
                                 int* queued, int* running, uint64_t* kernels);
/* The admission policy alone, in a discrete-event simulation on the host (no
 * GPU): request i arrives at arrival[i] on basis[i], is charged bytes[i] and
 * runs for duration[i] once admitted; start[i] receives its admission time,
 * or -1 if it can never fit.  Returns the peak number running at once, or -1
 * on bad arguments. */
EO_API int eo_admission_simulate(size_t budget, int slots, size_t resident_bytes, int nreq, const int* basis,
                                 const int64_t* bytes, const double* arrival, const double* duration, double* start);

/*
 * Allocation-free compensated Gram product (no counterpart in the paper).
 *
 * eo_gram_dd_noalloc computes the same G = X^T Y as eo_gram(..., EO_DD) for
 * callers that cannot allocate device memory when they need it: a component
 * whose GPU memory is wholly owned by another allocator, or a latency-critical
 * loop that must not call cudaMalloc/cudaFree (which may synchronize the
 * device).  It needs no context and allocates nothing: its scratch is a
 * fixed array of EO_NOALLOC_SCRATCH_BYTES inside the library, held on every
 * GPU that loads the library until the process exits.
 *   X, Y, G_hi, G_lo, lds: as in eo_gram (Y == NULL: Y = X); FP64 data.
 *   kx, ky must not exceed EO_NOALLOC_KMAX, and n must not exceed
 *   EO_NOALLOC_NMAX (152 row chunks of at most 2^22 rows: the partial sums of
 *   more chunks would not fit the array); larger sizes return EO_EINVAL
 *   before anything is launched.
 *   cuda_stream: the cudaStream_t to run on (NULL = default stream); the
 *   current CUDA device is used.
 * The first call on each device looks up the array's device address (with
 * that device current), and so does the first call after the device's
 * context has been re-created (e.g. by cudaDeviceReset, after which the
 * array may sit elsewhere); make those calls before any stream capture.
 * Every call shares the one array, so calls whose work overlaps on the GPU
 * (different streams, or other host threads) race and give wrong results;
 * serialize them.  Returns EO_OK, EO_EINVAL or EO_ECUDA.
 */
#define EO_NOALLOC_KMAX 16
#define EO_NOALLOC_NMAX (152ll << 22)
#define EO_NOALLOC_SCRATCH_BYTES (152u * EO_NOALLOC_KMAX * EO_NOALLOC_KMAX * 32u)
EO_API eo_status eo_gram_dd_noalloc(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y,
                                    int64_t ldy, double* G_hi, double* G_lo, int ldg, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* EO_H */
