// fxgram.cu — Gram products G = X^T Y in the compensated mode with exact
// fixed-point accumulation (fx.cuh) on the integer pipe.
//
// arXiv:1806.01036, Sec. 4.2: M = Y~^T Y~ and W^T X, summed over the n rows.
//
// Grid: blockIdx.x = tile group (a GI x GJ block of 4x4 tiles of G),
//       blockIdx.y = row chunk.  Consecutive CTAs share their rows, so the
//       columns that several groups read are served from L2.
// Per row panel of P rows the CTA
//   1. loads its X and Y columns into shared memory and takes the largest
//      biased exponent of each column (the running alignment exponent of that
//      column only grows; when it grows, accumulators are shifted right),
//   2. converts every value to four 26-bit limbs against that exponent,
//   3. lets each warp (one 4x4 tile, lanes over rows) accumulate the ten limb
//      products per entry into 64-bit diagonal accumulators; every
//      kRowsPerDrain rows a lane's accumulators are reduced over the warp as
//      exact 128-bit integers into a per-warp shared total.
// The CTA's tile totals (exact integers, with the column exponents that
// scale them) go to scratch; fx_gram_reduce aligns them to the largest scale
// and sums them exactly in 256 bits, then rounds once to a double-double.
// No step depends on the order of the sums.
#include <algorithm>

#include "common.cuh"
#include "fx.cuh"

namespace eo {
namespace {

using namespace fx;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int TS = 4;                 // tile edge
constexpr int GI = 2, GJ = 4;         // tiles per group (GI * GJ == kWarps)
constexpr int NCX = GI * TS, NCY = GJ * TS, NC = NCX + NCY;
constexpr int P = 128;                // rows per panel
constexpr int kDrainPanels = kRowsPerDrain / (P / 32);  // panels between drains (1 warp per tile)

struct __align__(16) FxPart {
  long long wl, wh;
  int s, flag;
  long long pad;
};

__device__ __forceinline__ i128 make_i128(long long lo, long long hi) {
  return (i128)(((u128)(unsigned long long)hi << 64) | (u128)(unsigned long long)lo);
}

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int m) {
  long long lo = (long long)(unsigned long long)(u128)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, m);
  hi = __shfl_xor_sync(0xffffffffu, hi, m);
  return make_i128(lo, hi);
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += shfl_xor_i128(v, m);
  return v;
}

// Group g -> (gi, gj); in the symmetric case only groups that hold a tile
// with ti <= tj exist, numbered row by row.
__device__ __forceinline__ void group_coords(int g, int ngi, int ngj, int sym, int& gi, int& gj) {
  if (!sym) {
    gi = g / ngj;
    gj = g % ngj;
    return;
  }
  for (int a = 0; a < ngi; ++a)
    for (int b = 0; b < ngj; ++b) {
      if (a * GI <= b * GJ + GJ - 1) {
        if (g == 0) {
          gi = a;
          gj = b;
          return;
        }
        --g;
      }
    }
  gi = gj = 0;
}

__global__ void __launch_bounds__(kThreads, 1)
    fx_gram_partial_kernel(int64_t n, int kx, const double* __restrict__ X, int64_t ldx, int ky,
                           const double* __restrict__ Y, int64_t ldy, int sym, int ngi, int ngj,
                           int64_t rows_per_chunk, FxPart* __restrict__ parts, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int4 (*limb)[P] = reinterpret_cast<int4 (*)[P]>(smem_raw);                       // [NC][P]
  double (*pan)[P] = reinterpret_cast<double (*)[P]>(smem_raw + sizeof(int4) * NC * P);  // [NC][P]
  __shared__ int Erun[NC], pmax[NC], delta[NC];
  __shared__ i128 Wt[kWarps][TS * TS];
  __shared__ int flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int gi, gj;
  group_coords(blockIdx.x, ngi, ngj, sym, gi, gj);
  const int nti = (kx + TS - 1) / TS, ntj = (ky + TS - 1) / TS;
  const int x0 = gi * NCX, y0 = gj * NCY;
  const int ncx = max(0, min(NCX, kx - x0)), ncy = max(0, min(NCY, ky - y0));
  const int ncol = ncx + ncy;

  // active tiles of this group, in row-major order; warps are shared out evenly
  int nact = 0, my_li = -1, my_lj = -1;
  for (int li = 0; li < GI; ++li)
    for (int lj = 0; lj < GJ; ++lj) {
      const int ti = gi * GI + li, tj = gj * GJ + lj;
      if (ti < nti && tj < ntj && (!sym || ti <= tj)) ++nact;
    }
  const int wpt = nact ? kWarps / nact : 1;
  const int my_t = warp / wpt, sub = warp % wpt;
  {
    int c = 0;
    for (int li = 0; li < GI; ++li)
      for (int lj = 0; lj < GJ; ++lj) {
        const int ti = gi * GI + li, tj = gj * GJ + lj;
        if (ti < nti && tj < ntj && (!sym || ti <= tj)) {
          if (c == my_t) {
            my_li = li;
            my_lj = lj;
          }
          ++c;
        }
      }
  }
  const bool active = my_t < nact && my_li >= 0;

  if (tid < NC) {
    Erun[tid] = 0;
    pmax[tid] = 0;
  }
  if (tid == 0) flag = 0;
  for (int e = tid; e < kWarps * TS * TS; e += kThreads) Wt[e / (TS * TS)][e % (TS * TS)] = 0;

  long long acc[TS][TS][4];
#pragma unroll
  for (int a = 0; a < TS; ++a)
#pragma unroll
    for (int b = 0; b < TS; ++b)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[a][b][d] = 0;

  // local limb columns of this warp's tile (clamped; out-of-range entries are never stored)
  int xc[TS], yc[TS];
#pragma unroll
  for (int a = 0; a < TS; ++a) {
    xc[a] = min(max(my_li, 0) * TS + a, max(ncx - 1, 0));
    yc[a] = ncx + min(max(my_lj, 0) * TS + a, max(ncy - 1, 0));
  }
  __syncthreads();

  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  int panels = 0;

  auto drain = [&]() {
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        i128 w = warp_sum_i128(acc_to_w(acc[a][b]));
        if (lane == 0) Wt[warp][a * TS + b] += w;
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[a][b][d] = 0;
      }
  };

  for (int64_t pr = r0; pr < r1; pr += P) {
    const int rows = (int)min((int64_t)P, r1 - pr);
    // 1. load the panel and the largest exponent per column
    for (int e = tid; e < ncol * P; e += kThreads) {
      const int c = e / P, r = e % P;
      double v = 0.0;
      if (r < rows) v = c < ncx ? X[(size_t)(x0 + c) * ldx + pr + r] : Y[(size_t)(y0 + c - ncx) * ldy + pr + r];
      pan[c][r] = v;
      const int ae = align_exp(v);
      if (ae == 2047) flag = 1;
      const int m = __reduce_max_sync(0xffffffffu, ae);  // the 32 lanes share column c (P % 32 == 0)
      if (lane == 0) atomicMax(&pmax[c], m);
    }
    __syncthreads();
    if (tid < ncol) {
      const int en = max(Erun[tid], pmax[tid]);
      delta[tid] = Erun[tid] == 0 ? 0 : en - Erun[tid];
      Erun[tid] = en;
      pmax[tid] = 0;
    }
    __syncthreads();
    // rescale accumulators whose columns' exponents grew
    if (active) {
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) {
          const int sh = delta[xc[a]] + delta[yc[b]];
          if (sh > 0) {
            acc_shift(acc[a][b], sh);
            if (lane == 0) Wt[warp][a * TS + b] = w_shift(Wt[warp][a * TS + b], sh);
          }
        }
    }
    // 2. convert to limbs
    for (int e = tid; e < ncol * P; e += kThreads) {
      const int c = e / P, r = e % P;
      const Limbs L = to_limbs(pan[c][r], max(Erun[c], 1));
      limb[c][r] = make_int4(L.v[0], L.v[1], L.v[2], L.v[3]);
    }
    __syncthreads();
    // 3. limb products
    if (active) {
      for (int r = sub * 32 + lane; r < rows; r += wpt * 32) {
        int4 xl[TS], yl[TS];
#pragma unroll
        for (int a = 0; a < TS; ++a) {
          xl[a] = limb[xc[a]][r];
          yl[a] = limb[yc[a]][r];
        }
#pragma unroll
        for (int a = 0; a < TS; ++a)
#pragma unroll
          for (int b = 0; b < TS; ++b) mac4(acc[a][b], xl[a], yl[b]);
      }
      if (++panels == kDrainPanels * wpt) {
        drain();
        panels = 0;
      }
    }
    __syncthreads();
  }
  if (active) drain();
  __syncthreads();

  if (active && sub == 0 && lane < TS * TS) {
    const int a = lane / TS, b = lane % TS;
    i128 w = 0;
    for (int s = 0; s < wpt; ++s) w += Wt[warp + s][lane];
    const int i = x0 + my_li * TS + a, j = y0 + my_lj * TS + b;
    if (my_li * TS + a < ncx && my_lj * TS + b < ncy) {
      FxPart p;
      p.wl = (long long)(unsigned long long)(u128)w;
      p.wh = (long long)(w >> 64);
      p.s = max(Erun[xc[a]], 1) + max(Erun[yc[b]], 1) - kScaleOffset;
      p.flag = flag;
      p.pad = 0;
      parts[(size_t)blockIdx.y * ((size_t)kx * ky) + (size_t)j * kx + i] = p;
    }
  }
}

__device__ __forceinline__ void shfl_acc256(Acc256& a, int m) {
  Acc256 o;
  long long w0 = (long long)(unsigned long long)a.lo, w1 = (long long)(unsigned long long)(a.lo >> 64);
  long long w2 = (long long)(unsigned long long)(u128)a.hi, w3 = (long long)(a.hi >> 64);
  w0 = __shfl_xor_sync(0xffffffffu, w0, m);
  w1 = __shfl_xor_sync(0xffffffffu, w1, m);
  w2 = __shfl_xor_sync(0xffffffffu, w2, m);
  w3 = __shfl_xor_sync(0xffffffffu, w3, m);
  o.lo = ((u128)(unsigned long long)w1 << 64) | (u128)(unsigned long long)w0;
  o.hi = make_i128(w2, w3);
  a.add(o);
}

__global__ void __launch_bounds__(kThreads) fx_gram_reduce_kernel(int kx, int ky, int sym, int nchunks,
                                                                  const FxPart* __restrict__ parts, double* G_hi,
                                                                  double* G_lo, int ldg, const int* gate) {
  if (gate && *gate == 0) return;
  const int e = (blockIdx.x * kThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int E = kx * ky;
  if (e >= E) return;
  const int i = e % kx, j = e / kx;
  if (sym && i > j) return;
  int smax = -1 << 30, fl = 0;
  for (int c = lane; c < nchunks; c += 32) {
    const FxPart& p = parts[(size_t)c * E + e];
    if (p.wl != 0 || p.wh != 0) smax = max(smax, p.s);
    fl |= p.flag;
  }
  smax = __reduce_max_sync(0xffffffffu, smax);
  fl = __reduce_or_sync(0xffffffffu, fl);
  Acc256 acc;
  acc.zero();
  for (int c = lane; c < nchunks; c += 32) {
    const FxPart& p = parts[(size_t)c * E + e];
    if (p.wl != 0 || p.wh != 0) acc.add(w_shift(make_i128(p.wl, p.wh), smax - p.s));
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) shfl_acc256(acc, m);
  if (lane == 0) {
    double hi = 0.0, lo = 0.0;
    if (fl) {
      hi = lo = __longlong_as_double(0x7ff8000000000000ll);
    } else if (smax > (-1 << 30)) {
      int extra = 0;
      const i128 w = acc.narrow(extra);
      w_to_dd(w, smax + extra, hi, lo);
    }
    G_hi[(size_t)j * ldg + i] = hi;
    if (G_lo) G_lo[(size_t)j * ldg + i] = lo;
    if (sym && i != j) {
      G_hi[(size_t)i * ldg + j] = hi;
      if (G_lo) G_lo[(size_t)i * ldg + j] = lo;
    }
  }
}

int num_groups(int kx, int ky, bool sym) {
  const int nti = (kx + TS - 1) / TS, ntj = (ky + TS - 1) / TS;
  const int ngi = (nti + GI - 1) / GI, ngj = (ntj + GJ - 1) / GJ;
  if (!sym) return ngi * ngj;
  int g = 0;
  for (int a = 0; a < ngi; ++a)
    for (int b = 0; b < ngj; ++b)
      if (a * GI <= b * GJ + GJ - 1) ++g;
  return g;
}

int num_chunks(int64_t n, int kx, int ky, bool sym) {
  const int g = num_groups(kx, ky, sym);
  const int64_t by_rows = (n + P - 1) / P;
  const int64_t want = (152 + g - 1) / g;  // one resident CTA per SM over the grid
  return (int)std::max<int64_t>(1, std::min(by_rows, want));
}

}  // namespace

size_t fx_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym) {
  return (size_t)num_chunks(n, kx, ky, sym) * (size_t)kx * ky * sizeof(FxPart);
}

cudaError_t launch_fx_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st) {
  if (sym) {
    Y = X;
    ldy = ldx;
    ky = kx;
  }
  const int nti = (kx + TS - 1) / TS, ntj = (ky + TS - 1) / TS;
  const int ngi = (nti + GI - 1) / GI, ngj = (ntj + GJ - 1) / GJ;
  const int groups = num_groups(kx, ky, sym);
  const int chunks = num_chunks(n, kx, ky, sym);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = std::max<int64_t>(P, (rpc + P - 1) / P * P);
  FxPart* parts = static_cast<FxPart*>(scratch);
  dim3 grid(groups, chunks);
  const size_t smem = (sizeof(int4) + sizeof(double)) * NC * P;
  cudaError_t e = cudaFuncSetAttribute(fx_gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fx_gram_partial_kernel<<<grid, kThreads, smem, st>>>(n, kx, X, ldx, ky, Y, ldy, sym ? 1 : 0, ngi, ngj, rpc, parts,
                                                    gate);
  const int E = kx * ky;
  fx_gram_reduce_kernel<<<(E * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(kx, ky, sym ? 1 : 0, chunks, parts,
                                                                                  G_hi, G_lo, ldg, gate);
  return cudaGetLastError();
}

}  // namespace eo
