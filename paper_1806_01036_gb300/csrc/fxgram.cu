// fxgram.cu — Gram products G = X^T Y in the compensated mode with exact
// fixed-point accumulation (fx.cuh) on the integer pipe.
//
// arXiv:1806.01036, Sec. 4.2: M = Y~^T Y~ and W^T X, summed over the n rows.
//
// The output is cut into 2x4 tiles (2 columns of X by 4 of Y); the tiles that
// are needed (all of them, or those touching the upper triangle when Y = X)
// are taken in row-major order and split into groups of at most
// 16 * 8 = 128 tiles.  Grid: blockIdx.x = group, blockIdx.y = row chunk, so
// consecutive CTAs share their rows (columns several groups read come from L2).
// Inside a CTA every tile owns R "row lanes" (R = 4..32 lanes of one warp, or
// several warps when the group has fewer than 16 tiles).  A CTA streams its
// chunk in panels of P rows:
//   * cp.async copies the next panel's columns into shared memory while the
//     current one is processed (double buffering);
//   * each column's running alignment exponent is raised to the panel's
//     largest exponent (accumulators are divided by 2^growth, exactly);
//   * every column value is converted once to four 26-bit limbs;
//   * every thread accumulates the ten leading limb products of its tile's
//     eight entries over its rows in 64-bit diagonal accumulators, and every
//     kRowsPerDrain rows these are summed over the tile's row lanes, exactly,
//     into 128-bit totals in shared memory.
// The CTA's totals (exact integers plus the column exponents that scale them)
// go to scratch; fx_gram_reduce aligns them to the largest scale, sums them
// exactly in 256 bits and rounds once to a double-double.  No result depends
// on the order of any sum.
#include <algorithm>

#include "common.cuh"
#include "fx.cuh"

namespace eo {
namespace {

using namespace fx;

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int TI = 2, TJ = 4;       // tile: TI columns of X by TJ columns of Y
constexpr int kMaxTiles = 128;      // tiles per CTA (8 per warp)
constexpr size_t kSmemBudget = 200 * 1024;


// Launch geometry shared by host and device.
struct GramPlan {
  int nti, ntj;      // tile grid
  int sym;
  int ntiles;        // needed tiles
  int groups;        // CTAs per row chunk
  int tiles_per_group;
  int P;             // rows per panel (a power of two, >= 32)
  int lgP;           // log2(P)
  int max_slots;     // columns held per CTA (bound)
};

__host__ __device__ __forceinline__ bool tile_needed(int ti, int tj, int sym) {
  return !sym || ti * TI <= tj * TJ + TJ - 1;
}

// Row-major index -> coordinates of the t-th needed tile.
__host__ __device__ __forceinline__ void nth_tile(int t, int nti, int ntj, int sym, int& ti, int& tj) {
  if (!sym) {
    ti = t / ntj;
    tj = t % ntj;
    return;
  }
  for (int a = 0; a < nti; ++a) {
    const int first = (a * TI) / TJ;  // first tj with a tile touching the upper triangle
    const int cnt = ntj - first;
    if (t < cnt) {
      ti = a;
      tj = first + t;
      return;
    }
    t -= cnt;
  }
  ti = tj = 0;
}

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

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

__global__ void __launch_bounds__(kThreads, 1)
    fx_gram_partial_kernel(int64_t n, int kx, const double* __restrict__ X, int64_t ldx, int ky,
                           const double* __restrict__ Y, int64_t ldy, GramPlan plan, int64_t rows_per_chunk,
                           FxPart* __restrict__ parts, const int* gate) {
  if (gate && *gate == 0) return;
  const int P = plan.P, lgP = plan.lgP;
  const int sym = plan.sym;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: limbs [slots][P] int4 | panel 2 x [slots][P] double | Wt [max(tiles,16)][8] i128 | ints
  const int S = plan.max_slots;
  int4* limb = reinterpret_cast<int4*>(smem_raw);
  double* pan = reinterpret_cast<double*>(limb + (size_t)S * P);
  i128* Wt = reinterpret_cast<i128*>(pan + 2 * (size_t)S * P);
  int* Erun = reinterpret_cast<int*>(Wt + (size_t)kMaxTiles * TI * TJ);
  int* pmax = Erun + S;
  int* delta = pmax + S;
  __shared__ int flag;

  const int tid = threadIdx.x, lane = tid & 31;
  // tiles of this group and the column ranges they read
  const int t0 = blockIdx.x * plan.tiles_per_group;
  const int T = min(plan.tiles_per_group, plan.ntiles - t0);
  int xa, xb, ya, yb;  // X columns [xa, xb), Y columns [ya, yb)
  {
    int ti, tj;
    nth_tile(t0, plan.nti, plan.ntj, sym, ti, tj);
    int ti_lo = ti, ti_hi = ti, tj_lo = tj, tj_hi = tj;
    for (int t = 1; t < T; ++t) {
      nth_tile(t0 + t, plan.nti, plan.ntj, sym, ti, tj);
      ti_lo = min(ti_lo, ti);
      ti_hi = max(ti_hi, ti);
      tj_lo = min(tj_lo, tj);
      tj_hi = max(tj_hi, tj);
    }
    xa = ti_lo * TI;
    xb = min(kx, ti_hi * TI + TI);
    ya = tj_lo * TJ;
    yb = min(ky, tj_hi * TJ + TJ);
  }
  // shared-memory slots: symmetric -> one run of columns [ca, cb) of X;
  // otherwise the X columns followed by the Y columns
  const int ca = sym ? min(xa, ya) : 0, cb = sym ? max(xb, yb) : 0;
  const int nslots = sym ? cb - ca : (xb - xa) + (yb - ya);
  auto xslot = [&](int c) { return sym ? c - ca : c - xa; };
  auto yslot = [&](int c) { return sym ? c - ca : (xb - xa) + c - ya; };

  // thread -> (tile, row lane)
  // row lanes per tile: a power of two (4..32) inside a warp when the group has
  // at least kWarps tiles, otherwise whole warps
  int Rl;
  if (T >= kWarps) {
    const int R = 32 / ((T + kWarps - 1) / kWarps);  // >= 4 for T <= kMaxTiles
    Rl = 32;
    while (Rl > R) Rl >>= 1;
  } else {
    Rl = 32 * (kWarps / T);
  }
  const int my_t = tid / Rl, rl = tid % Rl;
  const bool active = my_t < T;
  int ti = 0, tj = 0;
  if (active) nth_tile(t0 + my_t, plan.nti, plan.ntj, sym, ti, tj);
  const int rot = Rl < 8 ? (my_t * Rl) & (P - 1) : 0;  // spreads the tiles of a warp over the banks

  int xs[TI], ys[TJ];
#pragma unroll
  for (int a = 0; a < TI; ++a) xs[a] = xslot(min(ti * TI + a, kx - 1));
#pragma unroll
  for (int b = 0; b < TJ; ++b) ys[b] = yslot(min(tj * TJ + b, ky - 1));

  for (int c = tid; c < nslots; c += kThreads) {
    Erun[c] = 0;
    pmax[c] = 0;
  }
  if (tid == 0) flag = 0;
  for (int e = tid; e < kMaxTiles * TI * TJ; e += kThreads) Wt[e] = 0;

  long long acc[TI][TJ][4];
#pragma unroll
  for (int a = 0; a < TI; ++a)
#pragma unroll
    for (int b = 0; b < TJ; ++b)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[a][b][d] = 0;

  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const int npan = r0 < r1 ? (int)((r1 - r0 + P - 1) / P) : 0;

  auto issue = [&](int p, int buf) {
    const int64_t pr = r0 + (int64_t)p * P;
    const int rows = (int)min((int64_t)P, r1 - pr);
    double* dst0 = pan + (size_t)buf * S * P;
    for (int e = tid; e < nslots * P; e += kThreads) {
      const int c = e >> lgP, r = e & (P - 1);
      double* dst = dst0 + e;
      if (r < rows) {
        const double* src;
        if (sym) src = X + (size_t)(ca + c) * ldx + pr + r;
        else if (c < xb - xa) src = X + (size_t)(xa + c) * ldx + pr + r;
        else src = Y + (size_t)(ya + c - (xb - xa)) * ldy + pr + r;
        cp_async8(dst, src);
      } else {
        *dst = 0.0;
      }
    }
    cp_async_commit();
  };

  // Sum a tile's accumulators over its row lanes into Wt (exact).  Called by
  // every thread (idle threads hold zeros) so that the shuffles see full warps.
  auto drain = [&]() {
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
      for (int b = 0; b < TJ; ++b) {
        i128 w = acc_to_w(acc[a][b]);
        const int width = Rl < 32 ? Rl : 32;
        for (int m = width >> 1; m >= 1; m >>= 1) w += shfl_xor_i128(w, m);
        if (active) {
          if (Rl <= 32) {
            if (rl == 0) Wt[my_t * TI * TJ + a * TJ + b] += w;
          } else if (lane == 0) {  // several warps per tile: one slot per warp
            Wt[(tid >> 5) * TI * TJ + a * TJ + b] += w;
          }
        }
#pragma unroll
        for (int d = 0; d < 4; ++d) acc[a][b][d] = 0;
      }
  };
  const int rows_per_lane_panel = (P + Rl - 1) / Rl;
  const int drain_every = max(1, kRowsPerDrain / rows_per_lane_panel);

  __syncthreads();
  if (npan > 0) issue(0, 0);
  if (npan > 1) issue(1, 1);
  int since_drain = 0;
  for (int p = 0; p < npan; ++p) {
    const int buf = p & 1;
    const double* cur = pan + (size_t)buf * S * P;
    const int rows = (int)min((int64_t)P, r1 - (r0 + (int64_t)p * P));
    if (p + 1 < npan) cp_async_wait1(); else cp_async_wait0();
    __syncthreads();
    for (int e = tid; e < nslots * P; e += kThreads) {  // largest exponent per column
      const int ae = align_exp(cur[e]);
      if (ae == 2047) flag = 1;
      const int m = __reduce_max_sync(0xffffffffu, ae);  // a warp's 32 values share one column (P % 32 == 0)
      if (lane == 0) atomicMax(&pmax[e >> lgP], m);
    }
    __syncthreads();
    for (int c = tid; c < nslots; c += kThreads) {
      const int en = max(Erun[c], pmax[c]);
      delta[c] = Erun[c] == 0 ? 0 : en - Erun[c];
      Erun[c] = en;
      pmax[c] = 0;
    }
    __syncthreads();
    if (active) {  // divide accumulators by 2^growth of their columns' exponents
#pragma unroll
      for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) {
          const int sh = delta[xs[a]] + delta[ys[b]];
          if (sh > 0) {
            acc_shift(acc[a][b], sh);
            const int slot = Rl <= 32 ? (rl == 0 ? my_t : -1) : (lane == 0 ? (tid >> 5) : -1);
            if (slot >= 0) Wt[slot * TI * TJ + a * TJ + b] = w_shift(Wt[slot * TI * TJ + a * TJ + b], sh);
          }
        }
    }
    for (int e = tid; e < nslots * P; e += kThreads) {
      const Limbs L = to_limbs(cur[e], max(Erun[e >> lgP], 1));
      limb[e] = make_int4(L.v[0], L.v[1], L.v[2], L.v[3]);
    }
    __syncthreads();
    if (p + 2 < npan) issue(p + 2, buf);  // this panel buffer is free again
    if (active) {
      const int rot_p = rot % rows;
      for (int k = rl; k < rows; k += Rl) {
        int r = k + rot_p;
        if (r >= rows) r -= rows;
        int4 xl[TI], yl[TJ];
#pragma unroll
        for (int a = 0; a < TI; ++a) xl[a] = limb[(size_t)xs[a] * P + r];
#pragma unroll
        for (int b = 0; b < TJ; ++b) yl[b] = limb[(size_t)ys[b] * P + r];
#pragma unroll
        for (int a = 0; a < TI; ++a)
#pragma unroll
          for (int b = 0; b < TJ; ++b) mac4(acc[a][b], xl[a], yl[b]);
      }
    }
    if (++since_drain == drain_every) {  // uniform over the CTA
      drain();
      since_drain = 0;
    }
  }
  drain();
  __syncthreads();

  // write the tile totals: entry e of tile t sums the slots of its warps
  for (int q = tid; q < T * TI * TJ; q += kThreads) {
    const int t = q / (TI * TJ), e = q % (TI * TJ);
    const int a = e / TJ, b = e % TJ;
    int qi, qj;
    nth_tile(t0 + t, plan.nti, plan.ntj, sym, qi, qj);
    const int i = qi * TI + a, j = qj * TJ + b;
    if (i >= kx || j >= ky) continue;
    i128 w = 0;
    if (Rl <= 32) {
      w = Wt[t * TI * TJ + e];
    } else {
      const int wpt = Rl / 32;
      for (int s = 0; s < wpt; ++s) w += Wt[(t * wpt + s) * TI * TJ + e];
    }
    FxPart o;
    o.wl = (long long)(unsigned long long)(u128)w;
    o.wh = (long long)(w >> 64);
    o.s = max(Erun[xslot(i)], 1) + max(Erun[yslot(j)], 1) - kScaleOffset;
    o.flag = flag;
    o.pad = 0;
    parts[(size_t)blockIdx.y * ((size_t)kx * ky) + (size_t)j * kx + i] = o;
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

constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) fx_gram_reduce_kernel(int kx, int ky, int sym, int nchunks,
                                                                     const FxPart* __restrict__ parts, double* G_hi,
                                                                     double* G_lo, int ldg, const int* gate,
                                                                     int jo) {
  if (gate && *gate == 0) return;
  const int e = (blockIdx.x * kRedThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int E = kx * ky;
  if (e >= E) return;
  const int i = e % kx, j = e / kx;
  if (sym && i > jo + j) return;  // X = Y: the upper triangle of G, mirrored below
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
    // entry (i, jo + j) of G; with X = Y its mirror (jo + j, i) too
    G_hi[(size_t)(jo + j) * ldg + i] = hi;
    if (G_lo) G_lo[(size_t)(jo + j) * ldg + i] = lo;
    if (sym && i != jo + j) {
      G_hi[(size_t)i * ldg + jo + j] = hi;
      if (G_lo) G_lo[(size_t)i * ldg + jo + j] = lo;
    }
  }
}

GramPlan make_plan(int kx, int ky, bool sym) {
  GramPlan p{};
  p.sym = sym ? 1 : 0;
  p.nti = (kx + TI - 1) / TI;
  p.ntj = (ky + TJ - 1) / TJ;
  int nt = 0;
  for (int a = 0; a < p.nti; ++a)
    for (int b = 0; b < p.ntj; ++b) nt += tile_needed(a, b, p.sym) ? 1 : 0;
  p.ntiles = nt;
  p.groups = (nt + kMaxTiles - 1) / kMaxTiles;
  p.tiles_per_group = (nt + p.groups - 1) / p.groups;
  // columns a group may hold (host-side bound: scan the groups)
  int worst = 0;
  for (int g = 0; g < p.groups; ++g) {
    const int t0 = g * p.tiles_per_group, T = std::min(p.tiles_per_group, nt - t0);
    int lo_i = 1 << 30, hi_i = -1, lo_j = 1 << 30, hi_j = -1;
    for (int t = 0; t < T; ++t) {
      int ti, tj;
      nth_tile(t0 + t, p.nti, p.ntj, p.sym, ti, tj);
      lo_i = std::min(lo_i, ti);
      hi_i = std::max(hi_i, ti);
      lo_j = std::min(lo_j, tj);
      hi_j = std::max(hi_j, tj);
    }
    const int xa = lo_i * TI, xb = std::min(kx, hi_i * TI + TI), ya = lo_j * TJ, yb = std::min(ky, hi_j * TJ + TJ);
    const int s = sym ? std::max(xb, yb) - std::min(xa, ya) : (xb - xa) + (yb - ya);
    worst = std::max(worst, s);
  }
  p.max_slots = worst;
  // rows per panel: a power of two >= 32 that fits the limbs and two panels
  // of values; up to 2048 rows when few columns are held, so that a group
  // with few tiles (all 512 threads on one tile: small k) still gives every
  // thread rows and amortizes the per-panel barriers
  const size_t fixed = sizeof(i128) * kMaxTiles * TI * TJ + 3 * sizeof(int) * worst + 64;
  int P = 2048;
  while (P > 32 && fixed + (size_t)worst * P * (sizeof(int4) + 2 * sizeof(double)) > kSmemBudget) P /= 2;
  p.P = P;
  p.lgP = 0;
  while ((1 << p.lgP) < P) ++p.lgP;
  return p;
}

size_t plan_smem(const GramPlan& p) {
  return sizeof(int4) * (size_t)p.max_slots * p.P + 2 * sizeof(double) * (size_t)p.max_slots * p.P +
         sizeof(i128) * kMaxTiles * TI * TJ + 3 * sizeof(int) * p.max_slots;
}

// Row chunks: one resident CTA per SM over the grid, and at most 2^22 rows per
// chunk (a 128-bit total then holds the sum of a chunk's products, each below
// 2^104 units, with room to spare).  ctas > 0 caps the CTAs (fewer chunks).
int num_chunks(int64_t n, const GramPlan& p, int ctas = 0) {
  const int64_t by_rows = (n + p.P - 1) / p.P;
  const int64_t want = (152 + p.groups - 1) / p.groups;
  const int64_t need = (n + (1ll << 22) - 1) >> 22;
  const int64_t c = std::max<int64_t>(1, std::min(by_rows, std::max(want, need)));
  if (ctas <= 0) return (int)c;
  const int64_t cap = std::max<int64_t>(1, ctas / p.groups);
  return (int)std::max<int64_t>(std::max<int64_t>(1, need), std::min(c, cap));
}

}  // namespace

cudaError_t launch_fx_reduce(int kx, int ky, bool sym, int nchunks, const FxPart* parts, double* G_hi, double* G_lo,
                             int ldg, const int* gate, cudaStream_t st, int jo) {
  const int E = kx * ky;
  fx_gram_reduce_kernel<<<(E * 32 + kRedThreads - 1) / kRedThreads, kRedThreads, 0, st>>>(
      kx, ky, sym ? 1 : 0, nchunks, parts, G_hi, G_lo, ldg, gate, jo);
  return cudaGetLastError();
}

size_t fx_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym) {
  if (sym) ky = kx;
  return (size_t)num_chunks(n, make_plan(kx, ky, sym)) * (size_t)kx * ky * sizeof(FxPart);
}

int fx_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas) {
  if (sym) ky = kx;
  const GramPlan plan = make_plan(kx, ky, sym);
  return plan.groups * num_chunks(n, plan, ctas);
}

cudaError_t launch_fx_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                           bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                           cudaStream_t st, int ctas) {
  if (sym) {
    Y = X;
    ldy = ldx;
    ky = kx;
  }
  const GramPlan plan = make_plan(kx, ky, sym);
  const int chunks = num_chunks(n, plan, ctas);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = std::max<int64_t>(plan.P, (rpc + plan.P - 1) / plan.P * plan.P);
  FxPart* parts = static_cast<FxPart*>(scratch);
  dim3 grid(plan.groups, chunks);
  const size_t smem = plan_smem(plan);
  cudaError_t e = set_dyn_smem(fx_gram_partial_kernel, smem);
  if (e != cudaSuccess) return e;
  fx_gram_partial_kernel<<<grid, kThreads, smem, st>>>(n, kx, X, ldx, ky, Y, ldy, plan, rpc, parts, gate);
  const int E = kx * ky;
  fx_gram_reduce_kernel<<<(E * 32 + kRedThreads - 1) / kRedThreads, kRedThreads, 0, st>>>(
      kx, ky, sym ? 1 : 0, chunks, parts, G_hi, G_lo, ldg, gate, 0);
  return cudaGetLastError();
}

}  // namespace eo
