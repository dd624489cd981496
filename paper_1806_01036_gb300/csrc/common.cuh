// common.cuh — declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dd.cuh"
#include "eo.h"

namespace eo {

// Arithmetic of the FP64-pipe kernels (gram.cu, project.cu, update.cu,
// small.cu).  EO_DD_EFT runs them with MODE_DD; EO_DD uses the integer
// fixed-point kernels (fxgram.cu, fxrow.cu) for every sum over n rows.
enum Mode : int { MODE_FP64 = EO_FP64, MODE_DD = EO_DD, MODE_F32 = EO_F32 };

constexpr int KMAX = EO_KMAX;

// Dynamic shared memory limit of a kernel: always the device's opt-in
// maximum less its static shared memory, so that launches of one kernel with different sizes (several in
// one CUDA graph, say) never run under a smaller limit set for another.
int dyn_smem_limit();
template <class K>
cudaError_t set_dyn_smem(K kernel, size_t need) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const int lim = dyn_smem_limit() - (int)fa.sharedSizeBytes;  // the opt-in maximum covers static + dynamic
  if (lim <= 0 || need > (size_t)lim) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

// Device-resident status of one call.  gate[2p] enables the Gram and the
// small factorization of pass p, gate[2p+1] the streaming update of pass p;
// the factorization of pass p sets the gates of what follows, so a call never
// returns to the host between passes.
struct DevStatus {
  int info;
  int rank;
  int iters;
  int sweeps;  // Jacobi sweeps of the last SVQB eigensolve (0: none ran)
  int gate[64];
  int perm[64];  // pivot order of a pivoted Cholesky (eo_cholqr_piv)
};

// Gate layout of eo_orthogonalize (iteration i < kMaxIter): the projection,
// Gram and convergence test of iteration i run when gate[kItRun + i] != 0,
// its SVQB when gate[kItSvqb + i] != 0, its update when gate[kItUpd + i] != 0.
constexpr int kMaxIter = 16;
constexpr int kItRun = 0, kItSvqb = 16, kItUpd = 32;

// Device workspace for the k-by-k matrices of one call (FP64 hi/lo arrays,
// column-major with leading dimension KMAX).
struct SmallWs {
  double Mh[KMAX * KMAX], Ml[KMAX * KMAX];  // Gram matrix of the current pass
  double Zh[KMAX * KMAX], Zl[KMAX * KMAX];  // transform of the current pass
  double Th[KMAX * KMAX], Tl[KMAX * KMAX];  // accumulated R (CholQR) or Z (SVQB)
};

// ----------------------------------------------------------- Gram kernels
// Number of per-CTA partial results the Gram launch will produce and the
// scratch it needs (bytes) for a kx-by-ky Gram over n rows.
int gram_num_parts(int64_t n, int kx, int ky, bool sym);
size_t gram_scratch_bytes(int64_t n, int kx, int ky, bool sym);

// G = X^T Y (Y == X when sym).  X, Y are double* (or float* in MODE_F32).
// The kx-by-ky result goes to (G_hi, G_lo, ldg); G_lo may be null.
// gate: optional device flag; the kernels do nothing when *gate == 0.
cudaError_t launch_gram(Mode mode, int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y,
                        int64_t ldy, bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                        cudaStream_t st);

// --------------------------------------------------- projection kernels
size_t project_scratch_bytes(int64_t n, int kv, int k);
// Yout = Y - V C with C = (C_hi + C_lo) (kv-by-k, ldc), and, if M_hi is not
// null, M = Yout^T Yout accumulated in the same pass.
cudaError_t launch_project_fused(Mode mode, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                                 int64_t ldy, double* Yout, int64_t ldyo, const double* C_hi, const double* C_lo,
                                 int ldc, void* scratch, double* M_hi, double* M_lo, int ldm, const int* gate,
                                 cudaStream_t st);

// ------------------------------------------------------- update kernels
// X <- X Z for Z = (Zh + Zl) (k-by-k, ld KMAX); tri: Z upper triangular.
cudaError_t launch_update(Mode mode, int64_t n, int k, void* X, int64_t ldx, const double* Zh, const double* Zl,
                          bool tri, const int* gate, cudaStream_t st);

// ------------------------------------- exact fixed-point (EO_DD) kernels
// Partial Gram entry of one row chunk: an exact integer w (128 bits) with
// value w * 2^s, and a flag for non-finite inputs.
struct __align__(16) FxPart {
  long long wl, wh;
  int s, flag;
  long long pad;
};
// Sum the row-chunk partials of every entry exactly and round once: entry
// (i, j) of the kx-by-ky product into G(i, jo + j) (G_hi/G_lo, ldg).  sym:
// the product is columns jo .. jo + ky - 1 of a symmetric G; only entries
// with i <= jo + j are summed, each also written to G(jo + j, i).
cudaError_t launch_fx_reduce(int kx, int ky, bool sym, int nchunks, const FxPart* parts, double* G_hi, double* G_lo,
                             int ldg, const int* gate, cudaStream_t st, int jo = 0);
// The same product on the tcgen05 tensor cores (umma_gram.cu); same partial format.
// ctas > 0 caps the CTAs of the partial-sum launch (a launch shape picked by
// the batch autotuner); 0 = one CTA per SM.  The scratch sizes below hold for
// every cap.
size_t umma_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym);
cudaError_t launch_umma_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                             bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                             cudaStream_t st, int ctas = 0);
size_t fx_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym);
// CTAs of the partial-sum launch of each engine under a cap (0 = none; the
// largest launch of a product run as column strips).
int umma_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas);
// Kernels launch_umma_gram launches for these operands: 2 (partial sums and
// their reduction) per launch, 2 per column strip of a symmetric product
// with more than 16 columns.
int umma_gram_launches(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                       bool sym);
// The same exact sums for FP32 operands (the EO_F32 mode), each value
// widened to FP64 exactly: G_hi = the sum rounded once (G_lo its low part).
bool umma_gram_f32_supported(const float* X, const float* Y, int kx, int ky, bool sym);
cudaError_t launch_umma_gram_f32(int64_t n, int kx, const float* X, int64_t ldx, int ky, const float* Y,
                                 int64_t ldy, bool sym, void* scratch, double* G_hi, double* G_lo, int ldg,
                                 const int* gate, cudaStream_t st);
int fx_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas);
cudaError_t launch_fx_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st, int ctas = 0);
// Row products of the compensated mode on the tcgen05 tensor cores
// (umma_rowprod.cu): Out = Yin - A B (update = false) or Out = A B (update =
// true), A n-by-kin, B kin-by-kout double-double (column j at Bh + j ldb);
// kin <= 64, kout <= 16 (umma_rowprod_supported); Out may be A (in place).
// ctas > 0 caps the CTAs of the launch (0 = one per SM).
bool umma_rowprod_supported(int kin, int kout);
// Bounded device-side waits that ran out (tensor-core kernels): each unit's
// record, read and cleared (synchronous); and a one-thread kernel whose wait
// on an mbarrier that nothing completes runs out after limit_ns.
cudaError_t umma_gram_take_wait_record(unsigned* out);
cudaError_t umma_rowprod_take_wait_record(unsigned* out);
cudaError_t umma_wait_selftest(unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_umma_rowprod(bool update, int64_t n, int kin, const double* A, int64_t lda, int kout,
                                const double* Bh, const double* Bl, int ldb, bool tri, const double* Yin,
                                int64_t ldyin, double* Out, int64_t ldo, const int* gate, cudaStream_t st,
                                int ctas = 0);
// CTAs of an X Z launch (n-by-k) under a cap (0 = none).
int fx_update_ctas(int64_t n, int k, int ctas);
// Device scratch that lets an update with k > 16 run on the tensor cores
// (groups of 16 output columns; 0 when not needed).
size_t fx_update_tmp_bytes(int64_t n, int k);
// X <- X Z in place (Z: k-by-k double-double, leading dimension KMAX); ctas as
// above.  With k > 16 the tensor-core groups need tmp_bytes >= 
// fx_update_tmp_bytes(n, k) of scratch at tmp; otherwise the integer limbs run.
cudaError_t launch_fx_update(int64_t n, int k, double* X, int64_t ldx, const double* Zh, const double* Zl, bool tri,
                             const int* gate, cudaStream_t st, int ctas = 0, void* tmp = nullptr,
                             size_t tmp_bytes = 0);
// Kernels one launch_fx_update / launch_fx_project call launches.
int fx_update_launches(int64_t n, int k, size_t tmp_bytes);
int fx_project_launches(int64_t n, int kv, int k);
// Yout = Y - V C (C: kv-by-k double-double with leading dimension ldc).
cudaError_t launch_fx_project(int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y, int64_t ldy,
                              double* Yout, int64_t ldyo, const double* C_hi, const double* C_lo, int ldc,
                              const int* gate, cudaStream_t st);

// ------------------------------------------------ small k-by-k kernels
// Gates of one small factorization: it runs when *run != 0 and sets *upd
// (run the update that follows) and, if next is not null, *next (run the
// next pass).
struct SmallGates {
  const int* run;
  int* upd;
  int* next;
};

cudaError_t launch_status_init(DevStatus* s, int k, cudaStream_t st);
// M <- (M + M^T) / 2 in double-double (k-by-k, leading dimension ld; Ml may
// be null), when *gate != 0 (gate may be null).
cudaError_t launch_symmetrize(int k, double* Mh, double* Ml, int ld, const int* gate, cudaStream_t st);
// One CholQR factorization step of pass `pass` (0 or 1): M -> R, Z = R^{-1},
// T <- R T.  passes: 1, 2 or 0 (automatic).
cudaError_t launch_chol_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                              double* R_hi, double* R_lo, int ldr, DevStatus* s, SmallGates g, int pass, int passes,
                              int* info_user, cudaStream_t st);
cudaError_t launch_svqb_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                              double* Z_hi, double* Z_lo, int ldz, double tol, DevStatus* s, SmallGates g, int pass,
                              int passes, int* rank_user, cudaStream_t st, bool rotated = false);
// Pivoted, partial Cholesky of the pass's Gram matrix (one CTA): pass 0
// pivots on the largest remaining diagonal entry and stops at the numerical
// rank (remaining diagonal not above tol * the largest diagonal of M),
// Z = P [R11^{-1}, 0; 0, 0] (ws->Z) and R (ws->T); pass 1 factors the
// leading rank-by-rank block without pivoting, Z = [R2^{-1}, 0; 0, 0],
// R <- R2 R.  Rank and pivots go to the status (and the optional user
// outputs); info = -1 for a NaN or Inf, j >= 1 for a breakdown of pass 1.
cudaError_t launch_pivchol_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                                 double* R_hi, double* R_lo, int ldr, double tol, DevStatus* s, SmallGates g,
                                 int pass, int passes, int* info_user, int* rank_user, int* perm_user,
                                 cudaStream_t st);
// Many independent factorizations in one launch (one CTA per job): the
// Gram matrix of job j is in jobs[j].ws->Mh/Ml (leading dimension KMAX) and
// its gates in jobs[j].st (pass p as in the single launches); tol < 0 is
// replaced by the default of the job's k on the host.
struct SmallJob {
  int k;
  SmallWs* ws;
  DevStatus* st;
  double *Oh, *Ol;  // optional R (CholQR) or Z (SVQB) output
  int ldo;
  double tol;       // SVQB eigenvalue cut
  int* out;         // optional info (CholQR) or rank (SVQB)
};
double svqb_default_tol(Mode mode, int k);
cudaError_t launch_status_init_batched(const SmallJob* jobs, int njobs, cudaStream_t st);
cudaError_t launch_small_batched(bool chol, Mode mode, int njobs, int kmax, const SmallJob* jobs, int pass,
                                 int passes, cudaStream_t st);

// Convergence test of iteration `iter` of eo_orthogonalize: converged when
// max |C_ij| <= eps and max |M_ij - delta_ij| <= eps (C kv-by-k, M k-by-k,
// hi + lo).  Sets the SVQB/update gates of this iteration and the run gate of
// the next one, and the iteration count (negative when max_iter iterations
// did not converge).
cudaError_t launch_converge(const int* run, const double* Ch, const double* Cl, int ldc, int kv, int k,
                            const double* Mh, const double* Ml, int ldm, double eps, DevStatus* s, int iter,
                            int max_iter, int* iters_user, int* rank_user, cudaStream_t st);

}  // namespace eo
