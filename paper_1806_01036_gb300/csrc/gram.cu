// gram.cu — Gram products G = X^T Y over tall-skinny blocks.
//
// arXiv:1806.01036, Sec. 4.2: phase II builds M = Y~^T Y~, "the bulk of
// computation", and phase I needs W^T X; both are sums over the n rows of
// products of two columns.  In EO_DD mode each sum is accumulated with the
// Ogita-Rump-Oishi Dot2 step (TwoProd + TwoSum, FP64-pipe error-free
// transformations) as the paper's DD kernels do with AVX2 + FMA.
//
// Structure (deterministic for a given (n, kx, ky, mode)):
//   1. gram_partial: CTA b owns a contiguous chunk of rows.  Its warps own
//      TxT tiles of G; the lanes of a warp (and of the warps sharing a tile)
//      split the rows of the chunk.  Lane sums are combined by a fixed xor
//      butterfly, warps by a fixed-order loop, and the CTA's partial tile is
//      stored to scratch at parts[b][entry].
//   2. gram_reduce: one warp per output entry sums the partials in the fixed
//      order p = lane, lane+32, ... followed by the same butterfly, and writes
//      hi (and lo) of the result, mirroring the symmetric case.
#include <algorithm>

#include "common.cuh"

namespace eo {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int MODE>
struct Acc;

template <>
struct Acc<MODE_DD> {
  dd v;
  __device__ void zero() { v = dd{0.0, 0.0}; }
  __device__ void mac(double a, double b) { dd_fma_acc(v, a, b); }
  __device__ void add(dd o) { v = dd_add(dd_norm(v), dd_norm(o)); }
  __device__ dd get() const { return dd_norm(v); }
};

template <int MODE>
struct Acc {  // FP64 and F32 modes: plain FP64 accumulation with fma
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void mac(double a, double b) { v = __fma_rn(a, b, v); }
  __device__ void add(dd o) { v = __dadd_rn(v, o.hi); }
  __device__ dd get() const { return dd{v, 0.0}; }
};

__device__ __forceinline__ dd shfl_xor_dd(dd v, int m) {
  return dd{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// Tile t of the tile grid (nti x ntj); in the symmetric case only tiles with
// ti <= tj exist and they are numbered row by row.
__device__ __forceinline__ void tile_coords(int t, int nti, int ntj, int sym, int& ti, int& tj) {
  if (!sym) {
    ti = t / ntj;
    tj = t % ntj;
    return;
  }
  int row = 0;
  while (t >= ntj - row) {
    t -= ntj - row;
    ++row;
  }
  ti = row;
  tj = row + t;
}

template <int MODE, typename T, int TS>
__global__ void __launch_bounds__(kThreads) gram_partial_kernel(int64_t n, int kx, const T* __restrict__ X, int64_t ldx,
                                                                int ky, const T* __restrict__ Y, int64_t ldy, int sym,
                                                                int ntiles, dd* __restrict__ parts, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ dd red[kWarps][TS * TS];
  const int nti = (kx + TS - 1) / TS, ntj = (ky + TS - 1) / TS;
  const int t0 = blockIdx.y * kWarps;
  const int ctiles = min(kWarps, ntiles - t0);
  const int wpt = kWarps / ctiles;  // warps sharing one tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my = warp / wpt, sub = warp % wpt;
  const bool active = my < ctiles;

  const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = min(n, r0 + rpc);

  int ti = 0, tj = 0;
  if (active) tile_coords(t0 + my, nti, ntj, sym, ti, tj);
  const int i0 = ti * TS, j0 = tj * TS;

  Acc<MODE> acc[TS][TS];
#pragma unroll
  for (int a = 0; a < TS; ++a)
#pragma unroll
    for (int b = 0; b < TS; ++b) acc[a][b].zero();

  if (active) {
    const T* xc[TS];
    const T* yc[TS];
#pragma unroll
    for (int a = 0; a < TS; ++a) {
      xc[a] = X + (size_t)min(i0 + a, kx - 1) * ldx;
      yc[a] = Y + (size_t)min(j0 + a, ky - 1) * ldy;
    }
    const int stride = wpt * 32;
    for (int64_t r = r0 + sub * 32 + lane; r < r1; r += stride) {
      double xv[TS], yv[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) {
        xv[a] = (double)__ldg(xc[a] + r);
        yv[a] = (double)__ldg(yc[a] + r);
      }
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) acc[a][b].mac(xv[a], yv[b]);
    }
  }

  // Lane butterfly (fixed pattern), then warps of the same tile in order.
#pragma unroll
  for (int a = 0; a < TS; ++a)
#pragma unroll
    for (int b = 0; b < TS; ++b) {
      dd v = acc[a][b].get();
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        dd o = shfl_xor_dd(v, m);
        if (MODE == MODE_DD)
          v = dd_add(v, o);
        else
          v.hi = __dadd_rn(v.hi, o.hi);
      }
      if (lane == 0) red[warp][a * TS + b] = v;
    }
  __syncthreads();
  if (active && sub == 0) {
    const int E = kx * ky;
    for (int e = lane; e < TS * TS; e += 32) {
      dd v = red[warp][e];
      for (int s = 1; s < wpt; ++s) {
        dd o = red[warp + s][e];
        if (MODE == MODE_DD)
          v = dd_add(v, o);
        else
          v.hi = __dadd_rn(v.hi, o.hi);
      }
      const int i = i0 + e / TS, j = j0 + e % TS;
      if (i < kx && j < ky) parts[(size_t)blockIdx.x * E + (size_t)j * kx + i] = v;
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) gram_reduce_kernel(int kx, int ky, int sym, int nparts,
                                                               const dd* __restrict__ parts, double* G_hi,
                                                               double* G_lo, int ldg, const int* gate) {
  if (gate && *gate == 0) return;
  const int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int E = kx * ky;
  if (warp >= E) return;
  const int i = warp % kx, j = warp / kx;
  if (sym && i > j) return;  // the upper triangle is mirrored below
  dd v = dd{0.0, 0.0};
  for (int p = lane; p < nparts; p += 32) {
    dd o = parts[(size_t)p * E + warp];
    if (MODE == MODE_DD)
      v = dd_add(v, o);
    else
      v.hi = __dadd_rn(v.hi, o.hi);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    dd o = shfl_xor_dd(v, m);
    if (MODE == MODE_DD)
      v = dd_add(v, o);
    else
      v.hi = __dadd_rn(v.hi, o.hi);
  }
  if (lane == 0) {
    if (MODE == MODE_DD) v = fast_two_sum(v.hi, v.lo);
    G_hi[(size_t)j * ldg + i] = v.hi;
    if (G_lo) G_lo[(size_t)j * ldg + i] = (MODE == MODE_DD) ? v.lo : 0.0;
    if (sym && i != j) {
      G_hi[(size_t)i * ldg + j] = v.hi;
      if (G_lo) G_lo[(size_t)i * ldg + j] = (MODE == MODE_DD) ? v.lo : 0.0;
    }
  }
}

int tile_size(int kx, int ky) {
  int k = std::max(kx, ky);
  return k >= 4 ? 4 : (k >= 2 ? 2 : 1);
}

int num_tiles(int kx, int ky, bool sym) {
  int ts = tile_size(kx, ky);
  int nti = (kx + ts - 1) / ts, ntj = (ky + ts - 1) / ts;
  return sym ? nti * (nti + 1) / 2 : nti * ntj;
}

template <int MODE, typename T, int TS>
cudaError_t launch_t(int64_t n, int kx, const T* X, int64_t ldx, int ky, const T* Y, int64_t ldy, bool sym, dd* parts,
                     int nparts, double* G_hi, double* G_lo, int ldg, const int* gate, cudaStream_t st) {
  const int ntiles = num_tiles(kx, ky, sym);
  dim3 grid(nparts, (ntiles + kWarps - 1) / kWarps);
  gram_partial_kernel<MODE, T, TS><<<grid, kThreads, 0, st>>>(n, kx, X, ldx, ky, Y, ldy, sym ? 1 : 0, ntiles, parts,
                                                              gate);
  const int E = kx * ky;
  const int rblocks = (E * 32 + kThreads - 1) / kThreads;
  gram_reduce_kernel<MODE><<<rblocks, kThreads, 0, st>>>(kx, ky, sym ? 1 : 0, nparts, parts, G_hi, G_lo, ldg, gate);
  return cudaGetLastError();
}

template <int MODE, typename T>
cudaError_t launch_m(int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y, int64_t ldy, bool sym,
                     dd* parts, int nparts, double* G_hi, double* G_lo, int ldg, const int* gate, cudaStream_t st) {
  const T* x = static_cast<const T*>(X);
  const T* y = static_cast<const T*>(Y);
  switch (tile_size(kx, ky)) {
    case 4: return launch_t<MODE, T, 4>(n, kx, x, ldx, ky, y, ldy, sym, parts, nparts, G_hi, G_lo, ldg, gate, st);
    case 2: return launch_t<MODE, T, 2>(n, kx, x, ldx, ky, y, ldy, sym, parts, nparts, G_hi, G_lo, ldg, gate, st);
    default: return launch_t<MODE, T, 1>(n, kx, x, ldx, ky, y, ldy, sym, parts, nparts, G_hi, G_lo, ldg, gate, st);
  }
}

}  // namespace

int gram_num_parts(int64_t n, int kx, int ky, bool sym) {
  const int ntiles = num_tiles(kx, ky, sym);
  const int gy = (ntiles + kWarps - 1) / kWarps;
  // about four resident CTAs per SM over the whole grid; at least 256 rows each
  int64_t by_rows = (n + 255) / 256;
  int target = std::max(1, (152 * 4) / gy);
  return (int)std::max<int64_t>(1, std::min<int64_t>(by_rows, target));
}

size_t gram_scratch_bytes(int64_t n, int kx, int ky, bool sym) {
  return (size_t)gram_num_parts(n, kx, ky, sym) * (size_t)kx * ky * sizeof(dd);
}

cudaError_t launch_gram(Mode mode, int64_t n, int kx, const void* X, int64_t ldx, int ky, const void* Y, int64_t ldy,
                        bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                        cudaStream_t st) {
  dd* parts = static_cast<dd*>(scratch);
  const int np = gram_num_parts(n, kx, ky, sym);
  if (sym) {
    Y = X;
    ldy = ldx;
  }
  switch (mode) {
    case MODE_DD: return launch_m<MODE_DD, double>(n, kx, X, ldx, ky, Y, ldy, sym, parts, np, G_hi, G_lo, ldg, gate, st);
    case MODE_F32: return launch_m<MODE_F32, float>(n, kx, X, ldx, ky, Y, ldy, sym, parts, np, G_hi, G_lo, ldg, gate, st);
    default: return launch_m<MODE_FP64, double>(n, kx, X, ldx, ky, Y, ldy, sym, parts, np, G_hi, G_lo, ldg, gate, st);
  }
}

}  // namespace eo
