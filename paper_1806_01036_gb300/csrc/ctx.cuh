// ctx.cuh — the context behind the C-ABI handle and the pieces that api.cu
// and batch.cu share: error reporting, scratch memory, and the enqueue of one
// orthogonalization sequence (Sec. 4.2, phase II: Gram matrix, factorization,
// update) on explicit device resources.
#pragma once

#include <map>
#include <string>

#include "common.cuh"

namespace eo {

// Launch shape of one block's streaming kernels: CTA caps of the Gram
// partial-sum launch and of the row-product (update) launch; 0 = default
// (one CTA per SM).  Chosen per (k, n bucket, mode) by the batch autotuner.
struct Tile {
  int gram = 0;
  int row = 0;
};

struct TuneKey {
  int k, bucket, prec;
  bool operator<(const TuneKey& o) const {
    if (k != o.k) return k < o.k;
    if (bucket != o.bucket) return bucket < o.bucket;
    return prec < o.prec;
  }
};

}  // namespace eo

struct eo_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  uint64_t launches = 0;
  std::string err;
  std::string tune_path;                      // on-disk cache of tuned tiles ("" = in memory only)
  std::map<eo::TuneKey, eo::Tile> tuned;      // tuned tiles of this device
};

namespace eo {

constexpr uint64_t kGramLaunches = 2;  // partial sums + fixed-order reduction

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

eo_status fail(eo_ctx* c, eo_status s, const char* fmt, const char* a = "", long long b = 0);
eo_status cuda_fail(eo_ctx* c, const char* where, cudaError_t e);
bool valid_prec(int p);
// Grows the context's scratch to hold parts_bytes of partial sums (may synchronize its stream).
eo_status reserve_scratch(eo_ctx* c, size_t parts_bytes);
// Mode of the FP64-pipe kernels for a precision (EO_DD_EFT runs them in DD).
inline Mode pipe_mode(eo_prec p) { return p == EO_DD_EFT ? MODE_DD : (Mode)p; }

// Compensated Gram product on the engine its shape suits (tensor cores or
// integer limbs); ctas caps the partial-sum CTAs (0 = default).
size_t dd_gram_scratch(int64_t n, int kx, int ky, bool sym);
int dd_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas);
cudaError_t launch_dd_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st, int ctas = 0);

// One CholQR (chol) or SVQB sequence on X (n-by-k): status init, then per
// pass the Gram matrix (unless given), the small factorization and the update.
struct OrthArgs {
  bool chol;
  int64_t n;
  int k;
  void* X;
  int64_t ldx;
  const double *M_hi, *M_lo;  // optional Gram matrix of the first pass
  int ldm;
  double *O_hi, *O_lo;        // optional R (CholQR) or Z (SVQB) output
  int ldo;
  double tol;
  int passes;
  eo_prec prec;
  int* out_dev;               // info (CholQR) or rank (SVQB)
  // B-inner product <x, y>_B = x^T B y: P = B X (n-by-k, ldp) is given, the
  // Gram matrix is the symmetric part of X^T P, and P is updated with X.
  void* P = nullptr;
  int64_t ldp = 0;
  // SVQB only: Z = D U Lambda^{-1/2} (D = diag(M)^{-1/2}) instead of M^{-1/2}
  bool rotated = false;
};
struct OrthRes {
  DevStatus* st;
  SmallWs* ws;
  void* parts;        // Gram partials, and the scratch of the updates: orth_scratch() bytes
  cudaStream_t stream;
  Tile tile;
  size_t parts_bytes = 0;  // its size (0: too small for the tensor-core updates of k > 16)
};
size_t orth_scratch(int64_t n, int k, eo_prec prec, bool b_inner = false);
// Enqueues the sequence; on a CUDA error returns it and names the step in *where.
cudaError_t enqueue_orth(const OrthArgs& a, const OrthRes& r, uint64_t* launches, const char** where);
// One step of pass p of the sequence (the status must have been initialized).
enum class OrthStep { kGram = 0, kSmall = 1, kUpdate = 2 };
cudaError_t enqueue_orth_step(const OrthArgs& a, const OrthRes& r, int p, OrthStep step, uint64_t* launches);

}  // namespace eo

#define EO_CHECK(cond, code, ...)                     \
  do {                                                \
    if (!(cond)) return fail(ctx, code, __VA_ARGS__); \
  } while (0)

#define EO_CUDA(expr, where)                                 \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, where, e_); \
  } while (0)
