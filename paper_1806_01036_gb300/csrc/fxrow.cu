// fxrow.cu — row-wise products of the compensated mode with exact
// fixed-point accumulation (fx.cuh):
//   fx_update:   Y = Y~ Z, the final multiplication of phase II
//                (arXiv:1806.01036, Sec. 4.2; Z = R^{-1} upper triangular for
//                CholQR, the symmetric M^{-1/2} for SVQB);
//   fx_project:  Y~ = Y - V C, the phase I projection with C = V^T Y.
// Z (or C) is a double-double k-by-k (kv-by-k) matrix; each of its columns
// is aligned to its largest exponent once per CTA.  Each row of the streamed
// matrix (Y~ or V) is aligned to its own largest exponent.  A thread owns one
// row and four output columns; it forms the four sums of exact limb products
// and rounds each once to FP64 (for the projection, after subtracting the
// sum from y exactly in integer arithmetic).
#include <algorithm>

#include "common.cuh"
#include "fx.cuh"

namespace eo {
namespace {

using namespace fx;

constexpr int kThreads = 256;
constexpr int JG = 4;  // output columns per thread

// Limbs of the columns of a double-double matrix B (rows x cols, leading
// dimension ldb, hi/lo arrays), each column aligned to its largest exponent:
// Bl[j * rows + i], Eb[j] (>= 2048 when the column holds an Inf or NaN).
__device__ void load_small_limbs(int rows, int cols, const double* Bh, const double* Bl_, int ldb, int4* Bl, int* Eb) {
  for (int j = threadIdx.x; j < cols; j += blockDim.x) {
    int e = 0;
    for (int i = 0; i < rows; ++i) {
      e = max(e, align_exp(Bh[(size_t)j * ldb + i]));
      if (Bl_ && align_exp(Bl_[(size_t)j * ldb + i]) == 2047) e = 2047;
    }
    Eb[j] = e + 1;  // one binade of headroom: |h + l| may round up past the largest h
  }
  __syncthreads();
  for (int t = threadIdx.x; t < rows * cols; t += blockDim.x) {
    const int i = t % rows, j = t / rows;
    const double h = Bh[(size_t)j * ldb + i];
    const double l = Bl_ ? Bl_[(size_t)j * ldb + i] : 0.0;
    const Limbs L = to_limbs_dd(h, l, Eb[j]);
    Bl[(size_t)j * rows + i] = make_int4(L.v[0], L.v[1], L.v[2], L.v[3]);
  }
  __syncthreads();
}

// Rows of a panel: P rows, with limbs of the streamed matrix (cols columns)
// aligned per row.  Shared layout: Sl[c * P + r] (int4), Er[r].
template <int MODE_UPDATE>
__global__ void __launch_bounds__(kThreads, 2)
    fx_rowprod_kernel(int64_t n, int kin, const double* A, int64_t lda, int kout, const double* Bh, const double* Bl,
                      int ldb, int tri, const double* Yin, int64_t ldyin, double* Out, int64_t ldo, int P,
                      int lgP, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int4* Blimb = reinterpret_cast<int4*>(smem_raw);                 // kout * kin
  int4* Sl = Blimb + (size_t)kout * kin;                              // kin * P
  int* Eb = reinterpret_cast<int*>(Sl + (size_t)kin * P);             // kout
  int* Er = Eb + kout;                                                // P
  load_small_limbs(kin, kout, Bh, Bl, ldb, Blimb, Eb);

  const int ngroups = (kout + JG - 1) / JG;
  const int tid = threadIdx.x;
  const int my_r = tid & (P - 1), my_g = tid >> lgP;  // P * ngroups <= blockDim
  const bool active = my_g < ngroups;
  const int j0 = my_g * JG;
  const int parts = kThreads / P;  // threads per row in the exponent scan
  const int64_t stride = (int64_t)gridDim.x * P;

  for (int64_t pr = (int64_t)blockIdx.x * P; pr < n; pr += stride) {
    const int rows = (int)min((int64_t)P, n - pr);
    if (tid < P) Er[tid] = 0;
    __syncthreads();
    // row exponents: `parts` threads per row, strided over columns (loads
    // coalesced along rows; every load of the panel precedes every store of it,
    // so the update may run in place)
    if (my_g < parts && my_r < rows) {
      int m = 0;
      for (int c = my_g; c < kin; c += parts) m = max(m, align_exp(A[(size_t)c * lda + pr + my_r]));
      atomicMax(&Er[my_r], m);
    }
    __syncthreads();
    for (int e = tid; e < kin * P; e += kThreads) {  // second read of the panel: from L1/L2
      const int c = e >> lgP, r = e & (P - 1);
      const Limbs L = r < rows ? to_limbs(A[(size_t)c * lda + pr + r], max(Er[r], 1)) : Limbs{{0, 0, 0, 0}};
      Sl[e] = make_int4(L.v[0], L.v[1], L.v[2], L.v[3]);
    }
    __syncthreads();
    if (active && my_r < rows) {
      long long acc[JG][4];
#pragma unroll
      for (int q = 0; q < JG; ++q)
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[q][d] = 0;
      const int iend = tri ? min(kin, j0 + JG) : kin;  // Z is upper triangular for CholQR
      for (int i = 0; i < iend; ++i) {
        const int4 a = Sl[(size_t)i * P + my_r];
#pragma unroll
        for (int q = 0; q < JG; ++q) {
          const int j = min(j0 + q, kout - 1);
          mac4(acc[q], a, Blimb[(size_t)j * kin + i]);
        }
      }
      const int64_t r = pr + my_r;
#pragma unroll
      for (int q = 0; q < JG; ++q) {
        const int j = j0 + q;
        if (j < kout) {
          const i128 w = acc_to_w(acc[q]);
          const int S = max(Er[my_r], 1) + Eb[j] - kScaleOffset;
          double out;
          if (MODE_UPDATE)
            out = w_to_double(w, S);
          else
            out = sub_round(Yin[(size_t)j * ldyin + r], w, S);
          if (Er[my_r] >= 2047 || Eb[j] >= 2048) out = __longlong_as_double(0x7ff8000000000000ll);  // Inf/NaN input
          Out[(size_t)j * ldo + r] = out;
        }
      }
    }
    __syncthreads();
  }
}

// The general exact rounding (the rare inputs the branch-free forms leave),
// out of line.
__device__ __noinline__ double fx_round_general(int update, double y, i128 w, int S) {
  return update ? w_to_double(w, S) : sub_round(y, w, S);
}

// Narrow row products (kin <= KIN <= 8): a thread holds its row's values in
// registers, loaded one row ahead, and forms up to four outputs of it; the
// threads of a row's output groups are adjacent lanes of one warp, so the
// row's exponent needs no shared memory and the kernel no block barrier
// after the small matrix's limbs are set up.  The sums, their order and the
// rounding are those of fx_rowprod_kernel (bitwise the same outputs).  In
// place (update): every lane's loads of a row precede the warp's stores to
// it (the __syncwarp at the end of each step).
template <int MODE_UPDATE, int KIN>
__global__ void __launch_bounds__(kThreads, 2)
    fx_rowreg_kernel(int64_t n, int kin, const double* A, int64_t lda, int kout, const double* Bh, const double* Bl,
                     int ldb, int tri, const double* Yin, int64_t ldyin, double* Out, int64_t ldo, int lgng,
                     const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int4* Blimb = reinterpret_cast<int4*>(smem_raw);                 // kout * kin
  int* Eb = reinterpret_cast<int*>(Blimb + (size_t)kout * kin);    // kout
  load_small_limbs(kin, kout, Bh, Bl, ldb, Blimb, Eb);

  const int lane = threadIdx.x & 31;
  const int g = lane & ((1 << lgng) - 1);     // output group of this lane: outputs 4g .. 4g + 3
  const int rpw = 32 >> lgng;                 // rows per warp and step
  const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t slots = (int64_t)gridDim.x * (kThreads / 32) * rpw;  // rows per step of the grid
  const int j0 = JG * g;
  const bool active = j0 < kout;
  const int iend = tri ? min(kin, j0 + JG) : kin;  // Z is upper triangular for CholQR
  auto load_row = [&](int64_t r, double (&v)[KIN]) {
#pragma unroll
    for (int i = 0; i < KIN; ++i) v[i] = (i < kin && r < n) ? A[(size_t)i * lda + r] : 0.0;
  };
  int64_t w0 = warp * rpw;  // first row of this warp's step (uniform over the warp)
  double v[KIN];
  load_row(w0 + (lane >> lgng), v);
  __syncwarp();  // every lane's loads of the first step's rows precede its stores
  for (; w0 < n; w0 += slots) {
    const int64_t r = w0 + (lane >> lgng);
    double vn[KIN];
    load_row(r + slots, vn);  // the row of the next step, in flight during this one
    int e = 0;
#pragma unroll
    for (int i = 0; i < KIN; ++i) e = max(e, align_exp(v[i]));
    const int Er = max(e, 1);
    if (active && r < n) {
      long long acc[JG][4];
#pragma unroll
      for (int q = 0; q < JG; ++q)
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[q][d] = 0;
#pragma unroll
      for (int i = 0; i < KIN; ++i) {
        if (i < iend) {
          const Limbs L = to_limbs(v[i], Er);
          const int4 a = make_int4(L.v[0], L.v[1], L.v[2], L.v[3]);
#pragma unroll
          for (int q = 0; q < JG; ++q) mac4(acc[q], a, Blimb[(size_t)min(j0 + q, kout - 1) * kin + i]);
        }
      }
#pragma unroll
      for (int q = 0; q < JG; ++q) {
        const int j = j0 + q;
        if (j < kout) {
          const i128 w = acc_to_w(acc[q]);
          const int S = Er + Eb[j] - kScaleOffset;
          const double y = MODE_UPDATE ? 0.0 : Yin[(size_t)j * ldyin + r];
          bool ok;
          double out = MODE_UPDATE ? w_to_double_fast(w, S, ok) : sub_round_fast(y, w, S, ok);
          if (!ok) out = fx_round_general(MODE_UPDATE, y, w, S);
          if (e >= 2047 || Eb[j] >= 2048) out = __longlong_as_double(0x7ff8000000000000ll);  // Inf/NaN input
          Out[(size_t)j * ldo + r] = out;
        }
      }
    }
    __syncwarp();  // every lane's loads of this step's rows precede the next step's stores
#pragma unroll
    for (int i = 0; i < KIN; ++i) v[i] = vn[i];
  }
}

constexpr int kRegKin = 8;  // widest kin of fx_rowreg_kernel

int reg_groups_log2(int kout) {
  const int ng = (kout + JG - 1) / JG;
  int lg = 0;
  while ((1 << lg) < ng) ++lg;
  return lg;
}

bool use_rowreg(int kin, int kout) { return kin <= kRegKin && reg_groups_log2(kout) <= 3; }

int grid_reg(int64_t n, int kout, int ctas) {
  const int64_t rows_per_block = (int64_t)(kThreads / 32) * (32 >> reg_groups_log2(kout));
  const int64_t need = (n + rows_per_block - 1) / rows_per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, ctas > 0 ? ctas : 152 * 4));
}

constexpr size_t kSmemBudget = 110 * 1024;  // two CTAs per SM

int rows_per_panel(int kin, int kout) {
  const int ngroups = (kout + JG - 1) / JG;
  int P = 16;  // a power of two with P * ngroups <= kThreads
  while (P * 2 * ngroups <= kThreads) P *= 2;
  // shared memory: B's limbs, the panel's limbs and values, exponents
  const size_t fixed = sizeof(int4) * (size_t)kout * kin + sizeof(int) * kout;
  const size_t per_row = sizeof(int4) * (size_t)kin + sizeof(int);
  const int cap = (int)((kSmemBudget - fixed) / per_row);
  while (P > 16 && P > cap) P /= 2;
  return P;
}

size_t smem_bytes(int kin, int kout, int P) {
  return sizeof(int4) * ((size_t)kout * kin + (size_t)kin * P) + sizeof(int) * (kout + P);
}

int grid_of(int64_t n, int P, int ctas) {
  const int64_t panels = (n + P - 1) / P;
  return (int)std::max<int64_t>(1, std::min<int64_t>(panels, ctas > 0 ? ctas : 152 * 2));
}

cudaError_t launch_rowprod(bool update, int64_t n, int kin, const double* A, int64_t lda, int kout, const double* Bh,
                           const double* Bl, int ldb, bool tri, const double* Yin, int64_t ldyin, double* Out,
                           int64_t ldo, const int* gate, cudaStream_t st, int ctas = 0) {
  if (use_rowreg(kin, kout)) {
    const int lgng = reg_groups_log2(kout);
    const size_t smem = sizeof(int4) * (size_t)kout * kin + sizeof(int) * kout;
    const int blocks = grid_reg(n, kout, ctas);
    auto kern = update ? (kin <= 4 ? fx_rowreg_kernel<1, 4> : fx_rowreg_kernel<1, 8>)
                       : (kin <= 4 ? fx_rowreg_kernel<0, 4> : fx_rowreg_kernel<0, 8>);
    kern<<<blocks, kThreads, smem, st>>>(n, kin, A, lda, kout, Bh, Bl, ldb, tri ? 1 : 0, update ? nullptr : Yin,
                                         update ? 0 : ldyin, Out, ldo, lgng, gate);
    return cudaGetLastError();
  }
  const int P = rows_per_panel(kin, kout);
  int lgP = 0;
  while ((1 << lgP) < P) ++lgP;
  const size_t smem = smem_bytes(kin, kout, P);
  const int blocks = grid_of(n, P, ctas);
  cudaError_t e;
  if (update) {
    e = set_dyn_smem(fx_rowprod_kernel<1>, smem);
    if (e != cudaSuccess) return e;
    fx_rowprod_kernel<1><<<blocks, kThreads, smem, st>>>(n, kin, A, lda, kout, Bh, Bl, ldb, tri ? 1 : 0, nullptr, 0,
                                                         Out, ldo, P, lgP, gate);
  } else {
    e = set_dyn_smem(fx_rowprod_kernel<0>, smem);
    if (e != cudaSuccess) return e;
    fx_rowprod_kernel<0><<<blocks, kThreads, smem, st>>>(n, kin, A, lda, kout, Bh, Bl, ldb, 0, Yin, ldyin, Out, ldo,
                                                         P, lgP, gate);
  }
  return cudaGetLastError();
}

}  // namespace

// Both row products go to the tensor-core engine (umma_rowprod.cu) when their
// sizes fit it (kin <= 64, kout <= 16), to the integer limbs otherwise;
// EO_DD_ROW_ENGINE=int forces the integer limbs.
// Columns [0, cols) of dst <- src (n rows), when *gate != 0.
__global__ void copy_cols_kernel(int64_t n, int cols, const double* __restrict__ src, int64_t lds,
                                 double* __restrict__ dst, int64_t ldd, const int* gate) {
  if (gate && *gate == 0) return;
  const int64_t total = n * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    dst[j * ldd + i] = src[j * lds + i];
  }
}

size_t fx_update_tmp_bytes(int64_t n, int k) {
  if (k <= 16 || umma_rowprod_supported(k, k) || !umma_rowprod_supported(k, 16)) return 0;
  return (size_t)n * 16 * ((k + 15) / 16 - 1) * sizeof(double);
}

int fx_update_launches(int64_t n, int k, size_t tmp_bytes) {
  if (umma_rowprod_supported(k, k)) return n > 0 ? 1 : 0;
  const size_t need = fx_update_tmp_bytes(n, k);
  if (n > 0 && need > 0 && tmp_bytes >= need) return (k + 15) / 16 + 1;
  return 1;
}

int fx_project_launches(int64_t n, int kv, int k) {
  if (umma_rowprod_supported(kv, k)) return n > 0 ? 1 : 0;
  if (umma_rowprod_supported(kv, 16)) return n > 0 ? (k + 15) / 16 : 0;
  return 1;
}

int fx_update_ctas(int64_t n, int k, int ctas) {
  if (umma_rowprod_supported(k, k) || fx_update_tmp_bytes(n, k) > 0) {
    const int64_t ntiles = (n + 127) / 128;  // 128-row tiles of the tensor-core engine
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, ctas > 0 ? ctas : 152));
  }
  if (use_rowreg(k, k)) return grid_reg(n, k, ctas);
  return grid_of(n, rows_per_panel(k, k), ctas);
}

cudaError_t launch_fx_update(int64_t n, int k, double* X, int64_t ldx, const double* Zh, const double* Zl, bool tri,
                             const int* gate, cudaStream_t st, int ctas, void* tmp, size_t tmp_bytes) {
  if (umma_rowprod_supported(k, k))
    return launch_umma_rowprod(true, n, k, X, ldx, k, Zh, Zl, KMAX, tri, nullptr, 0, X, ldx, gate, st, ctas);
  const size_t need = fx_update_tmp_bytes(n, k);
  if (n > 0 && need > 0 && tmp && tmp_bytes >= need) {
    // groups of 16 output columns on the tensor cores: every group reads all
    // k columns of X, so all but the last write to tmp, the last runs in
    // place (a tile's loads precede its stores), and tmp is copied back
    const int G = (k + 15) / 16;
    double* T = static_cast<double*>(tmp);
    for (int g = 0; g < G; ++g) {
      const int c0 = 16 * g, kc = std::min(16, k - c0);
      const bool last = g == G - 1;
      double* out = last ? X + (size_t)c0 * ldx : T + (size_t)c0 * n;
      // a column slice of a triangular Z is not triangular in its own indices:
      // pass it whole (its zero entries cost nothing extra)
      cudaError_t e = launch_umma_rowprod(true, n, k, X, ldx, kc, Zh + (size_t)c0 * KMAX, Zl + (size_t)c0 * KMAX,
                                          KMAX, false, nullptr, 0, out, last ? ldx : n, gate, st, ctas);
      if (e != cudaSuccess) return e;
    }
    const int64_t total = n * 16 * (G - 1);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
    copy_cols_kernel<<<blocks, 256, 0, st>>>(n, 16 * (G - 1), T, n, X, ldx, gate);
    return cudaGetLastError();
  }
  return launch_rowprod(true, n, k, X, ldx, k, Zh, Zl, KMAX, tri, nullptr, 0, X, ldx, gate, st, ctas);
}

cudaError_t launch_fx_project(int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y, int64_t ldy,
                              double* Yout, int64_t ldyo, const double* C_hi, const double* C_lo, int ldc,
                              const int* gate, cudaStream_t st) {
  if (umma_rowprod_supported(kv, k))
    return launch_umma_rowprod(false, n, kv, V, ldv, k, C_hi, C_lo, ldc, false, Y, ldy, Yout, ldyo, gate, st);
  if (umma_rowprod_supported(kv, 16)) {
    // groups of 16 columns: each reads V and its own columns of Y and writes
    // the same columns of Yout, so groups never disturb one another (in place too)
    for (int c0 = 0; c0 < k; c0 += 16) {
      const int kc = std::min(16, k - c0);
      cudaError_t e = launch_umma_rowprod(false, n, kv, V, ldv, kc, C_hi + (size_t)c0 * ldc,
                                          C_lo ? C_lo + (size_t)c0 * ldc : nullptr, ldc, false, Y + (size_t)c0 * ldy,
                                          ldy, Yout + (size_t)c0 * ldyo, ldyo, gate, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return launch_rowprod(false, n, kv, V, ldv, k, C_hi, C_lo, ldc, false, Y, ldy, Yout, ldyo, gate, st);
}

}  // namespace eo
