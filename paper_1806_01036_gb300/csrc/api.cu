// api.cu — the C-ABI of include/eo.h: context, argument checks, scratch
// memory, and the launch sequences of eo_gram / eo_project / eo_cholqr /
// eo_svqb (arXiv:1806.01036, Sec. 4.2: phase I projection, phase II Gram,
// factorization of the Gram matrix and the final multiplication Y~ Z).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "ctx.cuh"

namespace eo {

eo_status fail(eo_ctx* c, eo_status s, const char* fmt, const char* a, long long b) {
  if (c) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, a, b);
    c->err = buf;
  }
  return s;
}

eo_status cuda_fail(eo_ctx* c, const char* where, cudaError_t e) {
  if (c) c->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // a failed attribute call or launch must not surface in the next call
  return EO_ECUDA;
}

bool valid_prec(int p) { return p == EO_FP64 || p == EO_DD || p == EO_F32 || p == EO_DD_EFT; }

int dyn_smem_limit() {
  static int cache[64] = {0};  // per device; concurrent first calls store the same value
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    dev = 0;
  }
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 227 * 1024;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Scratch layout: [DevStatus][SmallWs][C hi/lo (KMAX x KMAX)][partials ...]
constexpr size_t kOffStatus = 0;
constexpr size_t kOffWs = align_up(sizeof(DevStatus));
constexpr size_t kOffC = kOffWs + align_up(sizeof(SmallWs));
constexpr size_t kOffParts = kOffC + align_up(2 * sizeof(double) * KMAX * KMAX);

eo_status ensure_scratch(eo_ctx* c, size_t parts_bytes) {
  const size_t need = kOffParts + align_up(std::max<size_t>(parts_bytes, kAlign));
  if (need <= c->scratch_bytes) return EO_OK;
  if (c->scratch) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, "scratch resize (sync)", e);
    cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
  }
  const size_t grown = need + need / 4;
  cudaError_t e = cudaMalloc(&c->scratch, grown);
  if (e != cudaSuccess) {
    c->scratch = nullptr;
    cudaGetLastError();
    return fail(c, EO_ENOMEM, "cannot allocate %s%lld bytes of scratch", "", (long long)grown);
  }
  c->scratch_bytes = grown;
  return EO_OK;
}

}  // namespace

eo_status reserve_scratch(eo_ctx* c, size_t parts_bytes) { return ensure_scratch(c, parts_bytes); }

namespace {

DevStatus* status_of(eo_ctx* c) { return reinterpret_cast<DevStatus*>(static_cast<char*>(c->scratch) + kOffStatus); }
SmallWs* ws_of(eo_ctx* c) { return reinterpret_cast<SmallWs*>(static_cast<char*>(c->scratch) + kOffWs); }
double* c_hi_of(eo_ctx* c) { return reinterpret_cast<double*>(static_cast<char*>(c->scratch) + kOffC); }
double* c_lo_of(eo_ctx* c) { return c_hi_of(c) + KMAX * KMAX; }
void* parts_of(eo_ctx* c) { return static_cast<char*>(c->scratch) + kOffParts; }

__global__ void copy_small_kernel(int rows, int cols, const double* sh, const double* sl, int lds, double* dh,
                                  double* dl, int ldd) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows * cols; t += gridDim.x * blockDim.x) {
    const int i = t % rows, j = t / rows;
    if (dh) dh[(size_t)j * ldd + i] = sh[(size_t)j * lds + i];
    if (dl) dl[(size_t)j * ldd + i] = sl[(size_t)j * lds + i];
  }
}

}  // namespace

// Engine of a compensated Gram product: the tcgen05 digit engine
// (umma_gram.cu) once one side has more than 8 columns, the integer limbs
// (fxgram.cu) below (measured, symmetric, 4e6 rows: k = 4 0.26 ms on the
// limbs vs 0.51 ms on the tensor cores, k = 8 0.53 vs 0.51, k = 12 0.91 vs
// 0.55).  EO_DD_GRAM_ENGINE=int|umma overrides the choice (both engines give
// results within the same bound).
static bool use_umma_gram(int kx, int ky) {
  const char* e = getenv("EO_DD_GRAM_ENGINE");
  if (e && e[0] == 'u') return true;
  if (e && e[0] == 'i') return false;
  return std::max(kx, ky) > 8;
}

// Kernels one launch_dd_gram call launches.
static uint64_t dd_gram_launches(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y,
                                 int64_t ldy, bool sym) {
  return use_umma_gram(kx, sym ? kx : ky) ? (uint64_t)umma_gram_launches(n, kx, X, ldx, ky, Y, ldy, sym)
                                          : kGramLaunches;
}

size_t dd_gram_scratch(int64_t n, int kx, int ky, bool sym) {
  return std::max(fx_gram_scratch_bytes(n, kx, ky, sym), umma_gram_scratch_bytes(n, kx, ky, sym));
}

cudaError_t launch_dd_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st, int ctas) {
  if (use_umma_gram(kx, sym ? kx : ky))
    return launch_umma_gram(n, kx, X, ldx, ky, Y, ldy, sym, scratch, G_hi, G_lo, ldg, gate, st, ctas);
  return launch_fx_gram(n, kx, X, ldx, ky, Y, ldy, sym, scratch, G_hi, G_lo, ldg, gate, st, ctas);
}

int dd_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas) {
  return use_umma_gram(kx, sym ? kx : ky) ? umma_gram_ctas(n, kx, ky, sym, ctas) : fx_gram_ctas(n, kx, ky, sym, ctas);
}

// EO_F32 Gram products with 16 or more columns on one side run on the
// tensor-core digit engine (exact sums of the FP32 products, rounded once:
// at least as accurate as FP64 accumulation, and faster than summing on the
// FP64 pipe); narrower ones, and operands it cannot copy, sum their exact
// products in FP64.  The low parts are written as zero either way.
static bool f32_on_digits(const void* X, const void* Y, int kx, int ky, bool sym) {
  const char* e = getenv("EO_F32_GRAM_ENGINE");
  if (e && e[0] == 'f') return false;  // "fp64": the FP64-pipe sums
  return std::max(kx, sym ? kx : ky) >= 16 &&
         umma_gram_f32_supported(static_cast<const float*>(X), static_cast<const float*>(Y), kx, ky, sym);
}

size_t f32_gram_scratch(int64_t n, int kx, int ky, bool sym) {
  return std::max(gram_scratch_bytes(n, kx, ky, sym), umma_gram_scratch_bytes(n, kx, ky, sym));
}

cudaError_t launch_f32_gram(int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y, int64_t ldy,
                            bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                            cudaStream_t st) {
  if (!f32_on_digits(X, Y, kx, ky, sym))
    return launch_gram(MODE_F32, n, kx, X, ldx, ky, Y, ldy, sym, scratch, G_hi, G_lo, ldg, gate, st);
  cudaError_t e = launch_umma_gram_f32(n, kx, static_cast<const float*>(X), ldx, ky, static_cast<const float*>(Y),
                                       ldy, sym, scratch, G_hi, nullptr, ldg, gate, st);
  if (e == cudaSuccess && G_lo)
    e = cudaMemset2DAsync(G_lo, (size_t)ldg * sizeof(double), 0, (size_t)kx * sizeof(double), (size_t)(sym ? kx : ky),
                          st);
  return e;
}

size_t orth_scratch(int64_t n, int k, eo_prec prec, bool b_inner) {
  size_t s = prec == EO_DD ? dd_gram_scratch(n, k, k, true)
                           : (prec == EO_F32 ? f32_gram_scratch(n, k, k, true) : gram_scratch_bytes(n, k, k, true));
  if (b_inner) s = std::max(s, prec == EO_DD ? dd_gram_scratch(n, k, k, false) : gram_scratch_bytes(n, k, k, false));
  if (prec == EO_DD) s = std::max(s, fx_update_tmp_bytes(n, k));  // the partials are consumed before the update
  return s;
}

cudaError_t enqueue_orth_step(const OrthArgs& a, const OrthRes& r, int p, OrthStep step, uint64_t* launches) {
  const bool fx = a.prec == EO_DD;
  const Mode mode = pipe_mode(a.prec);
  const Mode small_mode = mode == MODE_DD ? MODE_DD : MODE_FP64;
  DevStatus* st = r.st;
  SmallWs* ws = r.ws;
  const int npass = a.passes == 1 ? 1 : 2;
  cudaError_t e = cudaSuccess;
  switch (step) {
    case OrthStep::kGram: {
      if (p == 0 && a.M_hi) return cudaSuccess;  // the caller's Gram matrix
      const bool b = a.P != nullptr;             // X^T P, then its symmetric part
      const void* Y = b ? a.P : a.X;
      const int64_t ldy = b ? a.ldp : a.ldx;
      if (fx) {
        e = launch_dd_gram(a.n, a.k, static_cast<const double*>(a.X), a.ldx, a.k, static_cast<const double*>(Y), ldy,
                           !b, r.parts, ws->Mh, ws->Ml, KMAX, &st->gate[2 * p], r.stream, r.tile.gram);
      } else if (a.prec == EO_F32) {
        e = launch_f32_gram(a.n, a.k, a.X, a.ldx, a.k, Y, ldy, !b, r.parts, ws->Mh, ws->Ml, KMAX, &st->gate[2 * p],
                            r.stream);
      } else {
        e = launch_gram(mode, a.n, a.k, a.X, a.ldx, a.k, Y, ldy, !b, r.parts, ws->Mh, ws->Ml, KMAX, &st->gate[2 * p],
                        r.stream);
      }
      *launches += fx ? dd_gram_launches(a.n, a.k, static_cast<const double*>(a.X), a.ldx, a.k,
                                         static_cast<const double*>(Y), ldy, !b)
                      : kGramLaunches;
      if (e == cudaSuccess && b) {
        e = launch_symmetrize(a.k, ws->Mh, ws->Ml, KMAX, &st->gate[2 * p], r.stream);
        *launches += 1;
      }
      return e;
    }
    case OrthStep::kSmall: {
      const bool given = p == 0 && a.M_hi;
      const double* mh = given ? a.M_hi : ws->Mh;
      const double* ml = given ? a.M_lo : ws->Ml;
      const int ld = given ? a.ldm : KMAX;
      const SmallGates gates{&st->gate[2 * p], &st->gate[2 * p + 1], p + 1 < npass ? &st->gate[2 * p + 2] : nullptr};
      e = a.chol ? launch_chol_small(small_mode, a.k, mh, ml, ld, ws, a.O_hi, a.O_lo, a.ldo, st, gates, p, a.passes,
                                     a.out_dev, r.stream)
                 : launch_svqb_small(small_mode, a.k, mh, ml, ld, ws, a.O_hi, a.O_lo, a.ldo, a.tol, st, gates, p,
                                     a.passes, a.out_dev, r.stream, a.rotated);
      *launches += 1;
      return e;
    }
    case OrthStep::kUpdate:
      for (int t = 0; t < (a.P ? 2 : 1) && e == cudaSuccess; ++t) {  // X, then P with the same Z
        void* A = t ? a.P : a.X;
        const int64_t lda = t ? a.ldp : a.ldx;
        e = fx ? launch_fx_update(a.n, a.k, static_cast<double*>(A), lda, ws->Zh, ws->Zl, a.chol,
                                  &st->gate[2 * p + 1], r.stream, r.tile.row, r.parts, r.parts_bytes)
               : launch_update(mode, a.n, a.k, A, lda, ws->Zh, ws->Zl, a.chol, &st->gate[2 * p + 1], r.stream);
        *launches += fx ? fx_update_launches(a.n, a.k, r.parts_bytes) : 1;
      }
      return e;
  }
  return cudaErrorInvalidValue;
}

cudaError_t enqueue_orth(const OrthArgs& a, const OrthRes& r, uint64_t* launches, const char** where) {
  cudaError_t e = launch_status_init(r.st, a.k, r.stream);
  *launches += 1;
  if (e != cudaSuccess) {
    *where = "status init";
    return e;
  }
  const int npass = a.passes == 1 ? 1 : 2;
  static const char* names[3] = {"Gram", "factorization", "update"};
  for (int p = 0; p < npass; ++p)
    for (OrthStep step : {OrthStep::kGram, OrthStep::kSmall, OrthStep::kUpdate}) {
      e = enqueue_orth_step(a, r, p, step, launches);
      if (e != cudaSuccess) {
        *where = names[(int)step];
        return e;
      }
    }
  return cudaSuccess;
}

}  // namespace eo

namespace eo {
namespace {

// Y - V C (and optionally M = Yout^T Yout) for a C already in device memory.
eo_status apply_projection(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                           int64_t ldy, double* Yout, int64_t ldyo, const double* ch, const double* cl, int ldc,
                           double* M_hi, double* M_lo, int ldm, eo_prec prec, const int* gate = nullptr) {
  if (prec == EO_DD) {
    EO_CUDA(launch_fx_project(n, kv, V, ldv, k, Y, ldy, Yout, ldyo, ch, cl, ldc, gate, ctx->stream), "eo_project");
    ctx->launches += fx_project_launches(n, kv, k);
    if (M_hi) {
      EO_CUDA(launch_dd_gram(n, k, Yout, ldyo, k, Yout, ldyo, true, parts_of(ctx), M_hi, M_lo, ldm, gate,
                             ctx->stream),
              "eo_project (Gram)");
      ctx->launches += dd_gram_launches(n, k, Yout, ldyo, k, Yout, ldyo, true);
    }
  } else {
    const Mode mode = pipe_mode(prec);
    EO_CUDA(launch_project_fused(mode, n, kv, V, ldv, k, Y, ldy, Yout, ldyo, ch, mode == MODE_DD ? cl : nullptr, ldc,
                                 parts_of(ctx), M_hi, M_lo, ldm, gate, ctx->stream),
            "eo_project (fused pass)");
    ctx->launches += M_hi ? 2 : 1;
  }
  return EO_OK;
}

size_t apply_scratch(int64_t n, int kv, int k, eo_prec prec) {
  return prec == EO_DD ? dd_gram_scratch(n, k, k, true) : project_scratch_bytes(n, kv, k);
}

template <bool CHOL>
eo_status orth_common(eo_ctx* ctx, const char* name, int64_t n, int k, void* X, int64_t ldx, const double* M_hi,
                      const double* M_lo, int ldm, double* O_hi, double* O_lo, int ldo, double tol, int passes,
                      eo_prec prec, int* out_dev, void* P = nullptr, int64_t ldp = 0, bool rotated = false) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "%s: bad precision mode %lld", name, (long long)prec);
  EO_CHECK(n >= 0 && k >= 1 && k <= KMAX, EO_EINVAL, "%s: bad sizes (n=%lld)", name, (long long)n);
  EO_CHECK(X != nullptr || n == 0, EO_EINVAL, "%s: null X", name);
  EO_CHECK(ldx >= std::max<int64_t>(1, n), EO_EINVAL, "%s: ldx too small%lld", name, (long long)ldx);
  EO_CHECK(!M_hi || ldm >= k, EO_EINVAL, "%s: ldm too small%lld", name, (long long)ldm);
  EO_CHECK(!(O_hi || O_lo) || ldo >= k, EO_EINVAL, "%s: output leading dimension too small%lld", name, (long long)ldo);
  EO_CHECK(passes >= 0 && passes <= 2, EO_EINVAL, "%s: passes must be 0, 1 or 2 (%lld)", name, (long long)passes);
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "%s: cannot select device", name);
  eo_status s = ensure_scratch(ctx, orth_scratch(n, k, prec, P != nullptr));
  if (s != EO_OK) return s;
  OrthArgs a{CHOL, n, k, X, ldx, M_hi, M_lo, ldm, O_hi, O_lo, ldo, tol, passes, prec, out_dev};
  a.P = P;
  a.ldp = ldp;
  a.rotated = rotated;
  OrthRes r{status_of(ctx), ws_of(ctx), parts_of(ctx), ctx->stream, Tile{}};
  r.parts_bytes = ctx->scratch_bytes - kOffParts;
  const char* where = "";
  cudaError_t e = enqueue_orth(a, r, &ctx->launches, &where);
  if (e != cudaSuccess) return cuda_fail(ctx, (std::string(name) + " (" + where + ")").c_str(), e);
  return EO_OK;
}

}  // namespace
}  // namespace eo

using namespace eo;

extern "C" {

int eo_version(void) { return 1; }

eo_status eo_create(eo_ctx** out, int device) {
  if (!out) return EO_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return EO_ECUDA;
  }
  eo_ctx* c = new eo_ctx();
  c->device = device;
  *out = c;
  return EO_OK;
}

eo_status eo_destroy(eo_ctx* ctx) {
  if (!ctx) return EO_EINVAL;
  {
    DeviceGuard g(ctx->device);
    if (ctx->scratch) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->scratch);
    }
  }
  delete ctx;
  return EO_OK;
}

eo_status eo_set_stream(eo_ctx* ctx, void* stream) {
  if (!ctx) return EO_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return EO_OK;
}

const char* eo_last_error(const eo_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t eo_kernel_launches(const eo_ctx* ctx) { return ctx ? ctx->launches : 0; }

eo_status eo_device_status(eo_ctx* ctx) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_device_status: cannot select device%s", "");
  EO_CUDA(cudaStreamSynchronize(ctx->stream), "eo_device_status (sync)");
  unsigned a = 0, b = 0;
  EO_CUDA(umma_gram_take_wait_record(&a), "eo_device_status (Gram record)");
  EO_CUDA(umma_rowprod_take_wait_record(&b), "eo_device_status (row-product record)");
  if (a || b) return fail(ctx, EO_ETIMEOUT, "a bounded device-side wait ran out%s (%lld): its outputs are NaN", "",
                          (long long)((a ? 1 : 0) | (b ? 2 : 0)));
  return EO_OK;
}

eo_status eo_selftest_wait_timeout(eo_ctx* ctx, double seconds) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(seconds > 0.0 && seconds <= 2.0, EO_EINVAL, "eo_selftest_wait_timeout: seconds must be in (0, 2]%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_selftest_wait_timeout: cannot select device%s", "");
  EO_CUDA(umma_wait_selftest((unsigned long long)(seconds * 1e9), ctx->stream), "eo_selftest_wait_timeout");
  ctx->launches += 1;
  return EO_OK;
}

eo_status eo_gram(eo_ctx* ctx, int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y, int64_t ldy,
                  double* G_hi, double* G_lo, int ldg, eo_prec prec) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  const bool sym = Y == nullptr;
  if (sym) {
    ky = kx;
    ldy = ldx;
  }
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_gram: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(n >= 0 && kx >= 1 && kx <= KMAX && ky >= 1 && ky <= KMAX, EO_EINVAL, "eo_gram: bad sizes%s (n=%lld)", "",
           (long long)n);
  EO_CHECK((X != nullptr || n == 0) && G_hi != nullptr, EO_EINVAL, "eo_gram: null pointer%s", "");
  EO_CHECK(ldx >= std::max<int64_t>(1, n) && ldy >= std::max<int64_t>(1, n) && ldg >= kx, EO_EINVAL,
           "eo_gram: leading dimension too small%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_gram: cannot select device%s", "");
  if (prec == EO_DD) {
    eo_status s = ensure_scratch(ctx, dd_gram_scratch(n, kx, ky, sym));
    if (s != EO_OK) return s;
    EO_CUDA(launch_dd_gram(n, kx, static_cast<const double*>(X), ldx, ky, static_cast<const double*>(sym ? X : Y),
                           ldy, sym, parts_of(ctx), G_hi, G_lo, ldg, nullptr, ctx->stream),
            "eo_gram");
    ctx->launches += dd_gram_launches(n, kx, static_cast<const double*>(X), ldx, ky,
                                      static_cast<const double*>(sym ? X : Y), ldy, sym);
    return EO_OK;
  } else if (prec == EO_F32) {
    eo_status s = ensure_scratch(ctx, f32_gram_scratch(n, kx, ky, sym));
    if (s != EO_OK) return s;
    EO_CUDA(launch_f32_gram(n, kx, X, ldx, ky, sym ? X : Y, ldy, sym, parts_of(ctx), G_hi, G_lo, ldg, nullptr,
                            ctx->stream),
            "eo_gram");
  } else {
    eo_status s = ensure_scratch(ctx, gram_scratch_bytes(n, kx, ky, sym));
    if (s != EO_OK) return s;
    EO_CUDA(launch_gram(pipe_mode(prec), n, kx, X, ldx, ky, sym ? X : Y, ldy, sym, parts_of(ctx), G_hi, G_lo, ldg,
                        nullptr, ctx->stream),
            "eo_gram");
  }
  ctx->launches += kGramLaunches;
  return EO_OK;
}

eo_status eo_project(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                     int64_t ldy, double* Yout, int64_t ldyo, double* C_hi, double* C_lo, int ldc, double* M_hi,
                     double* M_lo, int ldm, eo_prec prec) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_project: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(prec != EO_F32, EO_EUNSUPPORTED, "eo_project: FP32 inputs are not supported%s", "");
  EO_CHECK(n >= 0 && kv >= 1 && kv <= KMAX && k >= 1 && k <= KMAX, EO_EINVAL, "eo_project: bad sizes%s", "");
  EO_CHECK((V && Y && Yout) || n == 0, EO_EINVAL, "eo_project: null pointer%s", "");
  const int64_t mn = std::max<int64_t>(1, n);
  EO_CHECK(ldv >= mn && ldy >= mn && ldyo >= mn, EO_EINVAL, "eo_project: leading dimension too small%s", "");
  EO_CHECK(!C_hi || ldc >= kv, EO_EINVAL, "eo_project: ldc too small%s", "");
  EO_CHECK(!M_hi || ldm >= k, EO_EINVAL, "eo_project: ldm too small%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_project: cannot select device%s", "");
  const bool fx = prec == EO_DD;
  const size_t need = fx ? std::max(dd_gram_scratch(n, kv, k, false), dd_gram_scratch(n, k, k, true))
                         : std::max(gram_scratch_bytes(n, kv, k, false), project_scratch_bytes(n, kv, k));
  eo_status s = ensure_scratch(ctx, need);
  if (s != EO_OK) return s;
  double* ch = c_hi_of(ctx);
  double* cl = c_lo_of(ctx);
  const Mode mode = pipe_mode(prec);
  if (fx)
    EO_CUDA(launch_dd_gram(n, kv, V, ldv, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, nullptr, ctx->stream),
            "eo_project (V^T Y)");
  else
    EO_CUDA(launch_gram(mode, n, kv, V, ldv, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, nullptr, ctx->stream),
            "eo_project (V^T Y)");
  ctx->launches += kGramLaunches;
  if (C_hi || C_lo) {
    copy_small_kernel<<<4, 256, 0, ctx->stream>>>(kv, k, ch, cl, KMAX, C_hi, C_lo, ldc);
    EO_CUDA(cudaGetLastError(), "eo_project (copy C)");
    ctx->launches += 1;
  }
  return apply_projection(ctx, n, kv, V, ldv, k, Y, ldy, Yout, ldyo, ch, cl, KMAX, M_hi, M_lo, ldm, prec);
}

eo_status eo_project_apply(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                           int64_t ldy, double* Yout, int64_t ldyo, const double* C_hi, const double* C_lo, int ldc,
                           double* M_hi, double* M_lo, int ldm, eo_prec prec) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_project_apply: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(prec != EO_F32, EO_EUNSUPPORTED, "eo_project_apply: FP32 inputs are not supported%s", "");
  EO_CHECK(n >= 0 && kv >= 1 && kv <= KMAX && k >= 1 && k <= KMAX, EO_EINVAL, "eo_project_apply: bad sizes%s", "");
  EO_CHECK((V && Y && Yout) || n == 0, EO_EINVAL, "eo_project_apply: null pointer%s", "");
  EO_CHECK(C_hi != nullptr, EO_EINVAL, "eo_project_apply: C_hi is required%s", "");
  const int64_t mn = std::max<int64_t>(1, n);
  EO_CHECK(ldv >= mn && ldy >= mn && ldyo >= mn, EO_EINVAL, "eo_project_apply: leading dimension too small%s", "");
  EO_CHECK(ldc >= kv, EO_EINVAL, "eo_project_apply: ldc too small%s", "");
  EO_CHECK(!M_hi || ldm >= k, EO_EINVAL, "eo_project_apply: ldm too small%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_project_apply: cannot select device%s", "");
  eo_status s = ensure_scratch(ctx, apply_scratch(n, kv, k, prec));
  if (s != EO_OK) return s;
  return apply_projection(ctx, n, kv, V, ldv, k, Y, ldy, Yout, ldyo, C_hi, C_lo, ldc, M_hi, M_lo, ldm, prec);
}


eo_status eo_cholqr(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi, const double* M_lo,
                    int ldm, double* R_hi, double* R_lo, int ldr, int passes, eo_prec prec, int* info_dev) {
  return orth_common<true>(ctx, "eo_cholqr", n, k, X, ldx, M_hi, M_lo, ldm, R_hi, R_lo, ldr, 0.0, passes, prec,
                           info_dev);
}

eo_status eo_svqb(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi, const double* M_lo,
                  int ldm, double* Z_hi, double* Z_lo, int ldz, double tol, int passes, eo_prec prec, int* rank_dev) {
  return orth_common<false>(ctx, "eo_svqb", n, k, X, ldx, M_hi, M_lo, ldm, Z_hi, Z_lo, ldz, tol, passes, prec,
                            rank_dev);
}

eo_status eo_svqb_rotated(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, const double* M_hi, const double* M_lo,
                          int ldm, double* Z_hi, double* Z_lo, int ldz, double tol, eo_prec prec, int* rank_dev) {
  return orth_common<false>(ctx, "eo_svqb_rotated", n, k, X, ldx, M_hi, M_lo, ldm, Z_hi, Z_lo, ldz, tol, 1, prec,
                            rank_dev, nullptr, 0, true);
}

eo_status eo_cholqr_piv(eo_ctx* ctx, int64_t n, int k, double* X, int64_t ldx, double* R_hi, double* R_lo, int ldr,
                        double tol, int passes, eo_prec prec, int* perm_dev, int* rank_dev, int* info_dev) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_cholqr_piv: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(prec != EO_F32, EO_EUNSUPPORTED, "eo_cholqr_piv: FP32 inputs are not supported%s", "");
  EO_CHECK(n >= 0 && k >= 1 && k <= KMAX, EO_EINVAL, "eo_cholqr_piv: bad sizes%s (n=%lld)", "", (long long)n);
  EO_CHECK(X != nullptr || n == 0, EO_EINVAL, "eo_cholqr_piv: null X%s", "");
  EO_CHECK(ldx >= std::max<int64_t>(1, n), EO_EINVAL, "eo_cholqr_piv: ldx too small%s %lld", "", (long long)ldx);
  EO_CHECK(!(R_hi || R_lo) || ldr >= k, EO_EINVAL, "eo_cholqr_piv: ldr too small%s %lld", "", (long long)ldr);
  EO_CHECK(passes >= 0 && passes <= 2, EO_EINVAL, "eo_cholqr_piv: passes must be 0, 1 or 2%s (%lld)", "",
           (long long)passes);
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_cholqr_piv: cannot select device%s", "");
  eo_status s = ensure_scratch(ctx, orth_scratch(n, k, prec, false));
  if (s != EO_OK) return s;
  const bool fx = prec == EO_DD;
  const Mode mode = pipe_mode(prec);
  const Mode small_mode = mode == MODE_DD ? MODE_DD : MODE_FP64;
  if (tol < 0.0) tol = k * (small_mode == MODE_DD ? 0x1p-104 : 0x1p-52);
  DevStatus* st = status_of(ctx);
  SmallWs* ws = ws_of(ctx);
  const size_t parts_bytes = ctx->scratch_bytes - kOffParts;
  EO_CUDA(launch_status_init(st, k, ctx->stream), "eo_cholqr_piv (status)");
  ctx->launches += 1;
  const int npass = passes == 1 ? 1 : 2;
  for (int p = 0; p < npass; ++p) {
    const int* run = &st->gate[2 * p];
    if (fx)
      EO_CUDA(launch_dd_gram(n, k, X, ldx, k, X, ldx, true, parts_of(ctx), ws->Mh, ws->Ml, KMAX, run, ctx->stream),
              "eo_cholqr_piv (Gram)");
    else
      EO_CUDA(launch_gram(mode, n, k, X, ldx, k, X, ldx, true, parts_of(ctx), ws->Mh, ws->Ml, KMAX, run,
                          ctx->stream),
              "eo_cholqr_piv (Gram)");
    const SmallGates gates{run, &st->gate[2 * p + 1], p + 1 < npass ? &st->gate[2 * p + 2] : nullptr};
    EO_CUDA(launch_pivchol_small(small_mode, k, ws->Mh, ws->Ml, KMAX, ws, R_hi, R_lo, ldr, tol, st, gates, p, passes,
                                 info_dev, rank_dev, perm_dev, ctx->stream),
            "eo_cholqr_piv (factorization)");
    // pass 0: Z = P [R11^{-1}, 0; 0, 0] is a full matrix; pass 1: upper triangular
    const bool tri = p == 1;
    if (fx)
      EO_CUDA(launch_fx_update(n, k, X, ldx, ws->Zh, ws->Zl, tri, &st->gate[2 * p + 1], ctx->stream, 0, parts_of(ctx),
                               parts_bytes),
              "eo_cholqr_piv (update)");
    else
      EO_CUDA(launch_update(mode, n, k, X, ldx, ws->Zh, ws->Zl, tri, &st->gate[2 * p + 1], ctx->stream),
              "eo_cholqr_piv (update)");
    ctx->launches += (fx ? dd_gram_launches(n, k, X, ldx, k, X, ldx, true) : kGramLaunches) + 1 +
                     (fx ? fx_update_launches(n, k, parts_bytes) : 1);
  }
  return EO_OK;
}

eo_status eo_cholqr_b(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, void* BX, int64_t ldbx, double* R_hi,
                      double* R_lo, int ldr, int passes, eo_prec prec, int* info_dev) {
  if (!ctx) return EO_EINVAL;
  EO_CHECK(BX != nullptr || n == 0, EO_EINVAL, "eo_cholqr_b: null BX%s", "");
  EO_CHECK(ldbx >= std::max<int64_t>(1, n), EO_EINVAL, "eo_cholqr_b: ldbx too small%s", "");
  EO_CHECK(BX != X || n == 0, EO_EINVAL, "eo_cholqr_b: BX must not alias X (pass a copy for B = I)%s", "");
  return orth_common<true>(ctx, "eo_cholqr_b", n, k, X, ldx, nullptr, nullptr, 0, R_hi, R_lo, ldr, 0.0, passes, prec,
                           info_dev, BX, ldbx);
}

eo_status eo_svqb_b(eo_ctx* ctx, int64_t n, int k, void* X, int64_t ldx, void* BX, int64_t ldbx, double* Z_hi,
                    double* Z_lo, int ldz, double tol, int passes, eo_prec prec, int* rank_dev) {
  if (!ctx) return EO_EINVAL;
  EO_CHECK(BX != nullptr || n == 0, EO_EINVAL, "eo_svqb_b: null BX%s", "");
  EO_CHECK(ldbx >= std::max<int64_t>(1, n), EO_EINVAL, "eo_svqb_b: ldbx too small%s", "");
  EO_CHECK(BX != X || n == 0, EO_EINVAL, "eo_svqb_b: BX must not alias X (pass a copy for B = I)%s", "");
  return orth_common<false>(ctx, "eo_svqb_b", n, k, X, ldx, nullptr, nullptr, 0, Z_hi, Z_lo, ldz, tol, passes, prec,
                            rank_dev, BX, ldbx);
}

eo_status eo_project_b(eo_ctx* ctx, int64_t n, int kv, const double* W, int64_t ldw, const double* BW, int64_t ldbw,
                       int k, double* Y, int64_t ldy, double* BY, int64_t ldby, double* C_hi, double* C_lo, int ldc,
                       double* M_hi, double* M_lo, int ldm, eo_prec prec) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_project_b: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(prec != EO_F32, EO_EUNSUPPORTED, "eo_project_b: FP32 inputs are not supported%s", "");
  EO_CHECK(n >= 0 && kv >= 1 && kv <= KMAX && k >= 1 && k <= KMAX, EO_EINVAL, "eo_project_b: bad sizes%s", "");
  EO_CHECK((W && BW && Y && BY) || n == 0, EO_EINVAL, "eo_project_b: null pointer%s", "");
  EO_CHECK(Y != BY || n == 0, EO_EINVAL, "eo_project_b: BY must not alias Y%s", "");
  const int64_t mn = std::max<int64_t>(1, n);
  EO_CHECK(ldw >= mn && ldbw >= mn && ldy >= mn && ldby >= mn, EO_EINVAL,
           "eo_project_b: leading dimension too small%s", "");
  EO_CHECK(!(C_hi || C_lo) || ldc >= kv, EO_EINVAL, "eo_project_b: ldc too small%s", "");
  EO_CHECK(!M_hi || ldm >= k, EO_EINVAL, "eo_project_b: ldm too small%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_project_b: cannot select device%s", "");
  const bool fx = prec == EO_DD;
  const size_t need = fx ? std::max(dd_gram_scratch(n, kv, k, false), dd_gram_scratch(n, k, k, false))
                         : std::max({gram_scratch_bytes(n, kv, k, false), gram_scratch_bytes(n, k, k, false),
                                     project_scratch_bytes(n, kv, k)});
  eo_status s = ensure_scratch(ctx, need);
  if (s != EO_OK) return s;
  double* ch = c_hi_of(ctx);
  double* cl = c_lo_of(ctx);
  const Mode mode = pipe_mode(prec);
  // C = (B W)^T Y
  if (fx)
    EO_CUDA(launch_dd_gram(n, kv, BW, ldbw, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, nullptr, ctx->stream),
            "eo_project_b (BW^T Y)");
  else
    EO_CUDA(launch_gram(mode, n, kv, BW, ldbw, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, nullptr, ctx->stream),
            "eo_project_b (BW^T Y)");
  ctx->launches += kGramLaunches;
  if (C_hi || C_lo) {
    copy_small_kernel<<<4, 256, 0, ctx->stream>>>(kv, k, ch, cl, KMAX, C_hi, C_lo, ldc);
    EO_CUDA(cudaGetLastError(), "eo_project_b (copy C)");
    ctx->launches += 1;
  }
  // Y <- Y - W C and BY <- BY - BW C, in place
  s = apply_projection(ctx, n, kv, W, ldw, k, Y, ldy, Y, ldy, ch, cl, KMAX, nullptr, nullptr, 0, prec);
  if (s == EO_OK) s = apply_projection(ctx, n, kv, BW, ldbw, k, BY, ldby, BY, ldby, ch, cl, KMAX, nullptr, nullptr, 0,
                                       prec);
  if (s != EO_OK || !M_hi) return s;
  // M = the symmetric part of Y^T (BY)
  if (fx)
    EO_CUDA(launch_dd_gram(n, k, Y, ldy, k, BY, ldby, false, parts_of(ctx), M_hi, M_lo, ldm, nullptr, ctx->stream),
            "eo_project_b (Y^T BY)");
  else
    EO_CUDA(launch_gram(mode, n, k, Y, ldy, k, BY, ldby, false, parts_of(ctx), M_hi, M_lo, ldm, nullptr, ctx->stream),
            "eo_project_b (Y^T BY)");
  EO_CUDA(launch_symmetrize(k, M_hi, M_lo, ldm, nullptr, ctx->stream), "eo_project_b (symmetrize)");
  ctx->launches += kGramLaunches + 1;
  return EO_OK;
}

eo_status eo_orthogonalize(eo_ctx* ctx, int64_t n, int kv, const double* V, int64_t ldv, int k, double* Y,
                           int64_t ldy, double eps, int max_iter, double tol, eo_prec prec, int* iters_dev,
                           int* rank_dev) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_orthogonalize: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(prec != EO_F32, EO_EUNSUPPORTED, "eo_orthogonalize: FP32 inputs are not supported%s", "");
  EO_CHECK(n >= 0 && kv >= 1 && kv <= KMAX && k >= 1 && k <= KMAX, EO_EINVAL, "eo_orthogonalize: bad sizes%s", "");
  EO_CHECK((V && Y) || n == 0, EO_EINVAL, "eo_orthogonalize: null pointer%s", "");
  const int64_t mn = std::max<int64_t>(1, n);
  EO_CHECK(ldv >= mn && ldy >= mn, EO_EINVAL, "eo_orthogonalize: leading dimension too small%s", "");
  EO_CHECK(max_iter >= 1 && max_iter <= kMaxIter, EO_EINVAL, "eo_orthogonalize: max_iter must be in [1, %lld]", "",
           (long long)kMaxIter);
  EO_CHECK(eps >= 0.0, EO_EINVAL, "eo_orthogonalize: eps must be >= 0%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_orthogonalize: cannot select device%s", "");
  const bool fx = prec == EO_DD;
  const size_t need = fx ? std::max({dd_gram_scratch(n, kv, k, false), dd_gram_scratch(n, k, k, true),
                                     fx_update_tmp_bytes(n, k)})
                         : std::max(gram_scratch_bytes(n, kv, k, false), project_scratch_bytes(n, kv, k));
  eo_status s = ensure_scratch(ctx, need);
  if (s != EO_OK) return s;
  DevStatus* st = status_of(ctx);
  SmallWs* ws = ws_of(ctx);
  double* ch = c_hi_of(ctx);
  double* cl = c_lo_of(ctx);
  const Mode small_mode = pipe_mode(prec) == MODE_DD ? MODE_DD : MODE_FP64;
  EO_CUDA(launch_status_init(st, k, ctx->stream), "eo_orthogonalize");
  ctx->launches += 1;
  for (int it = 0; it < max_iter; ++it) {
    const int* run = &st->gate[kItRun + it];
    // phase I: C = V^T Y, Y <- Y - V C (in place), M = Y^T Y
    if (fx)
      EO_CUDA(launch_dd_gram(n, kv, V, ldv, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, run, ctx->stream),
              "eo_orthogonalize (V^T Y)");
    else
      EO_CUDA(launch_gram(pipe_mode(prec), n, kv, V, ldv, k, Y, ldy, false, parts_of(ctx), ch, cl, KMAX, run,
                          ctx->stream),
              "eo_orthogonalize (V^T Y)");
    ctx->launches += kGramLaunches;
    s = apply_projection(ctx, n, kv, V, ldv, k, Y, ldy, Y, ldy, ch, cl, KMAX, ws->Mh, ws->Ml, KMAX, prec, run);
    if (s != EO_OK) return s;
    // converged when both V^T Y and Y^T Y - I are below eps: stop here
    EO_CUDA(launch_converge(run, ch, cl, KMAX, kv, k, ws->Mh, ws->Ml, KMAX, eps, st, it, max_iter, iters_dev,
                            rank_dev, ctx->stream),
            "eo_orthogonalize (test)");
    // phase II: SVQB of the projected block
    const SmallGates gates{&st->gate[kItSvqb + it], &st->gate[kItUpd + it], nullptr};
    EO_CUDA(launch_svqb_small(small_mode, k, ws->Mh, ws->Ml, KMAX, ws, nullptr, nullptr, KMAX, tol, st, gates, 0, 1,
                              rank_dev, ctx->stream),
            "eo_orthogonalize (SVQB)");
    if (fx)
      EO_CUDA(launch_fx_update(n, k, Y, ldy, ws->Zh, ws->Zl, false, &st->gate[kItUpd + it], ctx->stream, 0,
                               parts_of(ctx), ctx->scratch_bytes - kOffParts),
              "eo_orthogonalize (update)");
    else
      EO_CUDA(launch_update(pipe_mode(prec), n, k, Y, ldy, ws->Zh, ws->Zl, false, &st->gate[kItUpd + it],
                            ctx->stream),
              "eo_orthogonalize (update)");
    ctx->launches += 2 + (fx ? fx_update_launches(n, k, ctx->scratch_bytes - kOffParts) : 1);  // test, SVQB, update
  }
  return EO_OK;
}

}  // extern "C"
