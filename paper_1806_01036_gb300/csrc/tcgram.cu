// tcgram.cu — compensated Gram products G = X^T Y on the tensor cores.
//
// arXiv:1806.01036, Sec. 4.2: M = Y~^T Y~ and W^T X summed over n rows with
// increased precision.  The sums are exact, as in fx.cuh, but the digit
// products run on the FP16 tensor cores instead of the integer pipe:
//
//  * each column value x of a row panel is aligned to its column's running
//    exponent A and held as X = floor(|x| 2^(1127 - A)) < 2^105, cut into 15
//    digits of 7 bits, X = sum_k D_k 2^(98 - 7k);
//  * a digit is stored as the FP16 number +-D_k 2^-24 (its bit pattern is the
//    digit itself with the value's sign; an FP16 subnormal), so every product
//    of two digits is exact and lands on the grid 2^-48;
//  * for each digit diagonal d = k + l <= 14 the tensor cores accumulate
//    S_d = sum over rows and over k + l = d of D_k(x) E_l(y) in FP32; with at
//    most 15 digit pairs of magnitude <= 127^2 per row, a 32-row panel keeps
//    |S_d| < 2^24, so the FP32 sums are exact integers (times 2^-48);
//  * after each panel the 15 sums are combined exactly, sum_d S_d 2^(7(14-d)),
//    in 128-bit integers and added to the running total in the units of the
//    integer engine (value = W 2^(Ax + Ay - 2148)); the partials then go
//    through the same exact, order-free reduction (fx_gram_reduce).
//
// The digits dropped (d >= 15) weigh less than 2^-101 max|x| max|y| per row,
// the same as the integer engine.  MMA: mma.sync m16n8k16 (row.col, f16
// inputs, f32 accumulators); a warp owns one 16x8 output tile (16 columns of
// X by 8 of Y) and 15 accumulator fragments.
#include <algorithm>

#include "common.cuh"
#include "fx.cuh"

namespace eo {
namespace {

using namespace fx;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int TM = 16, TN = 8;  // output tile of one warp: TM columns of X by TN of Y
constexpr int NS = 15;          // digits per value
constexpr int P = 32;           // rows per panel (two k-steps of 16)
constexpr int kTileGroup = 8;   // tiles per CTA
constexpr int kOffsetDigits = 2148;

struct TcPlan {
  int ntx, nty, sym, ntiles, groups, tiles_per_group;
  int max_slots;  // columns held by a CTA (multiple of 8)
};

__host__ __device__ __forceinline__ bool tc_tile_needed(int tx, int ty, int sym) {
  return !sym || tx * TM <= ty * TN + TN - 1;
}

__host__ __device__ __forceinline__ void tc_nth_tile(int t, int ntx, int nty, int sym, int& tx, int& ty) {
  if (!sym) {
    tx = t / nty;
    ty = t % nty;
    return;
  }
  for (int a = 0; a < ntx; ++a) {
    const int first = (a * TM) / TN;  // first ty whose tile touches the upper triangle
    const int cnt = nty - first;
    if (t < cnt) {
      tx = a;
      ty = first + t;
      return;
    }
    t -= cnt;
  }
  tx = ty = 0;
}

// Column ranges of a group: X columns [xa, xb), Y columns [ya, yb) (rounded
// to whole tiles, possibly past the matrix edge: those slots hold zeros).
__host__ __device__ __forceinline__ void group_ranges(const TcPlan& p, int g, int& xa, int& xb, int& ya, int& yb,
                                                      int& T) {
  const int t0 = g * p.tiles_per_group;
  T = p.ntiles - t0 < p.tiles_per_group ? p.ntiles - t0 : p.tiles_per_group;
  int tx, ty;
  tc_nth_tile(t0, p.ntx, p.nty, p.sym, tx, ty);
  int lx = tx, hx = tx, ly = ty, hy = ty;
  for (int t = 1; t < T; ++t) {
    tc_nth_tile(t0 + t, p.ntx, p.nty, p.sym, tx, ty);
    lx = tx < lx ? tx : lx;
    hx = tx > hx ? tx : hx;
    ly = ty < ly ? ty : ly;
    hy = ty > hy ? ty : hy;
  }
  xa = lx * TM;
  xb = hx * TM + TM;
  ya = ly * TN;
  yb = hy * TN + TN;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned& r0, unsigned& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ __forceinline__ void mma16816(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Byte offset of the 16-byte chunk ch (rows 8ch .. 8ch+7) of column slot c in
// digit slice s: the chunk index is XOR-swizzled so that the eight rows an
// ldmatrix reads (eight consecutive slots, same chunk) fall on distinct banks.
__device__ __forceinline__ unsigned dig_off(int s, int c, int nslots, int ch) {
  return (unsigned)((((s * nslots + c) << 2) + (ch ^ ((c >> 1) & 3))) << 4);
}

// X = floor(|x| 2^(1127 - A)) as (hi, lo) 64-bit halves; A >= align_exp(x).
__device__ __forceinline__ void fixed105(double x, int A, unsigned long long& x1, unsigned long long& x0) {
  const unsigned hi = hi32(x), lo = lo32(x);
  int be = (hi >> 20) & 0x7ff;
  unsigned mh = hi & 0xfffffu;
  if (be) mh |= 0x100000u; else be = 1;
  const unsigned long long m = ((unsigned long long)mh << 32) | lo;
  const int t = 52 - (A - be);
  u128 X;
  if (t >= 0) X = (u128)m << t;
  else if (t > -64) X = (u128)(m >> (-t));
  else X = 0;
  x0 = (unsigned long long)X;
  x1 = (unsigned long long)(X >> 64);
}

template <int S>
__device__ __forceinline__ unsigned digit(unsigned long long x1, unsigned long long x0) {
  constexpr int q = 98 - 7 * S;
  if (q >= 64) return (unsigned)(x1 >> (q - 64)) & 127u;
  if (q > 57) return (unsigned)((x0 >> q) | (x1 << (64 - q))) & 127u;
  return (unsigned)(x0 >> q) & 127u;
}

template <int S>
__device__ __forceinline__ void store_digits(unsigned char* dig, int nslots, int c, int r, unsigned long long a1,
                                             unsigned long long a0, unsigned sa, unsigned long long b1,
                                             unsigned long long b0, unsigned sb) {
  if constexpr (S < NS) {
    const unsigned w = (digit<S>(a1, a0) | sa) | ((digit<S>(b1, b0) | sb) << 16);
    *reinterpret_cast<unsigned*>(dig + dig_off(S, c, nslots, r >> 3) + ((r & 7) << 1)) = w;
    store_digits<S + 1>(dig, nslots, c, r, a1, a0, sa, b1, b0, sb);
  }
}

// acc[d] += A_s B_t for all s + t = d <= 14, with B_t for t = 0..14 in b.
template <int S>
__device__ __forceinline__ void mma_slice(float (*acc)[4], unsigned a_base, int a_stride, const unsigned (*b)[2]) {
  if constexpr (S < NS) {
    unsigned a[4];
    ldsm_x4(a_base + S * a_stride, a[0], a[1], a[2], a[3]);
#pragma unroll
    for (int t = 0; t + S < NS; ++t) mma16816(acc[S + t], a, b[t]);
    mma_slice<S + 1>(acc, a_base, a_stride, b);
  }
}

__global__ void __launch_bounds__(kThreads, 2)
    tc_gram_partial_kernel(int64_t n, int kx, const double* __restrict__ X, int64_t ldx, int ky,
                           const double* __restrict__ Y, int64_t ldy, TcPlan plan, int64_t rows_per_chunk,
                           FxPart* __restrict__ parts, const int* gate) {
  if (gate && *gate == 0) return;
  const int sym = plan.sym;
  int xa, xb, ya, yb, T;
  group_ranges(plan, blockIdx.x, xa, xb, ya, yb, T);
  // slots: symmetric -> one run [ca, cb) of X's columns; otherwise X's then Y's
  const int ca = sym ? min(xa, ya) : 0, cb = sym ? max(xb, yb) : 0;
  const int nslots = sym ? cb - ca : (xb - xa) + (yb - ya);
  auto xslot = [&](int c) { return sym ? c - ca : c - xa; };
  auto yslot = [&](int c) { return sym ? c - ca : (xb - xa) + c - ya; };
  auto slot_col = [&](int sl, bool& isx) {  // slot -> (matrix, column)
    if (sym) {
      isx = true;
      return ca + sl;
    }
    isx = sl < xb - xa;
    return isx ? xa + sl : ya + sl - (xb - xa);
  };

  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = plan.max_slots;
  unsigned char* dig = smem_raw;  // NS * nslots * P halves; reused at the end for the cross-warp sums
  const size_t dig_bytes = max((size_t)NS * S * P * 2, (size_t)kWarps * 32 * 4 * sizeof(i128));
  double* stage = reinterpret_cast<double*>(dig + dig_bytes);  // S * P doubles
  int* Erun = reinterpret_cast<int*>(stage + (size_t)S * P);
  int* pmax = Erun + S;
  int* delta = pmax + S;
  __shared__ int flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wpt = kWarps / T;  // warps per tile (k-steps split among them)
  const int my_t = warp / wpt, ksub = warp % wpt;
  const bool active = my_t < T;
  int tx = 0, ty = 0;
  if (active) tc_nth_tile(blockIdx.x * plan.tiles_per_group + my_t, plan.ntx, plan.nty, sym, tx, ty);
  const int xs0 = xslot(tx * TM), ys0 = yslot(ty * TN);
  const int g = lane >> 2, tig = lane & 3;
  // the four accumulator elements of this lane: (X col, Y col) slots
  const int ex[4] = {xs0 + g, xs0 + g, xs0 + g + 8, xs0 + g + 8};
  const int ey[4] = {ys0 + 2 * tig, ys0 + 2 * tig + 1, ys0 + 2 * tig, ys0 + 2 * tig + 1};

  for (int c = tid; c < nslots; c += kThreads) {
    Erun[c] = 0;
    pmax[c] = 0;
  }
  if (tid == 0) flag = 0;

  float acc[NS][4];
#pragma unroll
  for (int d = 0; d < NS; ++d)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[d][q] = 0.f;
  i128 W[4] = {0, 0, 0, 0};

  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const int npan = r0 < r1 ? (int)((r1 - r0 + P - 1) / P) : 0;

  auto issue = [&](int p) {
    const int64_t pr = r0 + (int64_t)p * P;
    const int rows = (int)min((int64_t)P, r1 - pr);
    for (int e = tid; e < nslots * P; e += kThreads) {
      const int sl = e >> 5, r = e & (P - 1);
      bool isx;
      const int col = slot_col(sl, isx);
      double* dst = stage + e;
      if (r < rows && (isx ? col < kx : col < ky)) {
        cp_async8(dst, isx ? X + (size_t)col * ldx + pr + r : Y + (size_t)col * ldy + pr + r);
      } else {
        *dst = 0.0;
      }
    }
    cp_async_commit();
  };

  __syncthreads();
  if (npan > 0) issue(0);
  const unsigned dig_s = (unsigned)__cvta_generic_to_shared(dig);
  const int a_stride = nslots * P * 2;  // bytes between digit slices (dig_off's layout)
  for (int p = 0; p < npan; ++p) {
    cp_async_wait0();
    __syncthreads();
    for (int e = tid; e < nslots * P; e += kThreads) {  // largest exponent per column of the panel
      const int ae = align_exp(stage[e]);
      if (ae == 2047) flag = 1;
      const int m = __reduce_max_sync(0xffffffffu, ae);  // a warp's 32 values are one column (P == 32)
      if (lane == 0) atomicMax(&pmax[e >> 5], m);
    }
    __syncthreads();
    for (int c = tid; c < nslots; c += kThreads) {
      const int en = max(Erun[c], pmax[c]);
      delta[c] = Erun[c] == 0 ? 0 : en - Erun[c];
      Erun[c] = en;
      pmax[c] = 0;
    }
    __syncthreads();
    if (active) {  // divide running totals by 2^growth of their columns' exponents
#pragma unroll
      for (int q = 0; q < 4; ++q) W[q] = w_shift(W[q], delta[ex[q]] + delta[ey[q]]);
    }
    // digits: a thread takes two rows of one column per step
    for (int u = tid; u < nslots * (P / 2); u += kThreads) {
      const int c = u >> 4, r = (u & 15) << 1;
      const int A = max(Erun[c], 1);
      const double va = stage[(c << 5) + r], vb = stage[(c << 5) + r + 1];
      unsigned long long a1, a0, b1, b0;
      fixed105(va, A, a1, a0);
      fixed105(vb, A, b1, b0);
      const unsigned sa = (hi32(va) >> 31) << 15, sb = (hi32(vb) >> 31) << 15;
      store_digits<0>(dig, nslots, c, r, a1, a0, sa, b1, b0, sb);
    }
    __syncthreads();
    if (p + 1 < npan) issue(p + 1);  // the staging buffer is free again
    if (active) {
      for (int kk = ksub; kk < P / 16; kk += wpt) {
        // B fragments (Y digits) for all 15 slices: ldmatrix.x2 rows = 8 Y slots, chunk 2kk + (lane >> 3 & 1)
        unsigned b[NS][2];
        {
          const int n = lane & 7, kc = 2 * kk + ((lane >> 3) & 1);
          const unsigned base = dig_s + dig_off(0, ys0 + n, nslots, kc);
#pragma unroll
          for (int t = 0; t < NS; ++t) ldsm_x2(base + t * a_stride, b[t][0], b[t][1]);
        }
        // A fragments (X digits): ldmatrix.x4 rows = 16 X slots, chunks 2kk and 2kk + 1
        const int mrow = (lane & 7) + ((lane >> 3) & 1) * 8, kc = 2 * kk + (lane >> 4);
        const unsigned a_base = dig_s + dig_off(0, xs0 + mrow, nslots, kc);
        mma_slice<0>(acc, a_base, a_stride, b);
      }
      // drain the panel: S_d = acc * 2^48 (exact integers), W += floor(sum_d S_d 2^(7(14-d)) / 2^8)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        i128 h = 0;
#pragma unroll
        for (int d = 0; d < NS; ++d) {
          h = (h << 7) + (i128)__float2int_rn(acc[d][q] * 0x1p48f);
          acc[d][q] = 0.f;
        }
        W[q] += h >> 8;
      }
    }
  }
  __syncthreads();

  // sum the warps that share a tile (k-split) and write the partials
  i128* red = reinterpret_cast<i128*>(dig);  // reuse: kWarps * 32 * 4 entries
  if (active) {
#pragma unroll
    for (int q = 0; q < 4; ++q) red[((size_t)warp * 32 + lane) * 4 + q] = W[q];
  }
  __syncthreads();
  if (active && ksub == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      i128 w = 0;
      for (int s2 = 0; s2 < wpt; ++s2) w += red[((size_t)(warp + s2) * 32 + lane) * 4 + q];
      bool isx;
      const int i = slot_col(ex[q], isx);
      const int j = sym ? ca + ey[q] : ya + ey[q] - (xb - xa);
      if (i < kx && j < ky) {
        FxPart o;
        o.wl = (long long)(unsigned long long)(u128)w;
        o.wh = (long long)(w >> 64);
        o.s = max(Erun[ex[q]], 1) + max(Erun[ey[q]], 1) - kOffsetDigits;
        o.flag = flag;
        o.pad = 0;
        parts[(size_t)blockIdx.y * ((size_t)kx * ky) + (size_t)j * kx + i] = o;
      }
    }
  }
}

TcPlan make_plan(int kx, int ky, bool sym) {
  TcPlan p{};
  p.sym = sym ? 1 : 0;
  p.ntx = (kx + TM - 1) / TM;
  p.nty = (ky + TN - 1) / TN;
  int nt = 0;
  for (int a = 0; a < p.ntx; ++a)
    for (int b = 0; b < p.nty; ++b) nt += tc_tile_needed(a, b, p.sym) ? 1 : 0;
  p.ntiles = nt;
  p.groups = (nt + kTileGroup - 1) / kTileGroup;
  p.tiles_per_group = (nt + p.groups - 1) / p.groups;
  // wpt = kWarps / T must divide evenly enough: T in {1, 2, 4, 8} keeps every warp busy
  int worst = 0;
  for (int g = 0; g < p.groups; ++g) {
    int xa, xb, ya, yb, T;
    group_ranges(p, g, xa, xb, ya, yb, T);
    const int s = sym ? std::max(xb, yb) - std::min(xa, ya) : (xb - xa) + (yb - ya);
    worst = std::max(worst, s);
  }
  p.max_slots = worst;
  return p;
}

size_t plan_smem(const TcPlan& p) {
  const size_t digits = (size_t)NS * p.max_slots * P * 2;
  const size_t red = (size_t)kWarps * 32 * 4 * sizeof(i128);
  return std::max(digits, red) + (size_t)p.max_slots * P * sizeof(double) + 3 * sizeof(int) * p.max_slots;
}

int num_chunks(int64_t n, const TcPlan& p) {
  const int64_t by_rows = (n + P - 1) / P;
  const int64_t want = (2 * 152 + p.groups - 1) / p.groups;  // two resident CTAs per SM
  return (int)std::max<int64_t>(1, std::min(by_rows, want));
}

}  // namespace

size_t tc_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym) {
  if (sym) ky = kx;
  return (size_t)num_chunks(n, make_plan(kx, ky, sym)) * (size_t)kx * ky * sizeof(FxPart);
}

cudaError_t launch_tc_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st) {
  if (sym) {
    Y = X;
    ldy = ldx;
    ky = kx;
  }
  const TcPlan plan = make_plan(kx, ky, sym);
  const int chunks = num_chunks(n, plan);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = std::max<int64_t>(P, (rpc + P - 1) / P * P);
  FxPart* parts = static_cast<FxPart*>(scratch);
  const size_t smem = plan_smem(plan);
  cudaError_t e = cudaFuncSetAttribute(tc_gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.groups, chunks);
  tc_gram_partial_kernel<<<grid, kThreads, smem, st>>>(n, kx, X, ldx, ky, Y, ldy, plan, rpc, parts, gate);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_fx_reduce(kx, ky, sym, chunks, parts, G_hi, G_lo, ldg, gate, st);
}

}  // namespace eo
