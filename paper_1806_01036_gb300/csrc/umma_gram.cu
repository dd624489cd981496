// umma_gram.cu — compensated Gram products G = X^T Y on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// arXiv:1806.01036, Sec. 4.2: M = Y~^T Y~ and W^T X summed over n rows with
// increased precision.  The sums are exact, as in fx.cuh; the digit products
// run on the tensor cores:
//
//  * each value x of a column is aligned to the column's alignment exponent
//    A and held as X = floor(|x| 2^(1127 - A)) < 2^105, written with 15
//    balanced digits, X = sum_s D_s 2^(98 - 7s), D_s in [-64, 63] (D_0 in
//    [-64, 128]; umma.cuh: the fields of X + sum_s 64 2^(98 - 7s), less 64);
//  * a digit is the FP16 integer sign(x) D_s, so every product of two digits
//    is an integer of at most 2^12 (2^14 for the two top digits) and FP32
//    sums of such products are exact while they stay within 2^24;
//  * a column's alignment exponent starts at the first panel's largest
//    exponent plus EO_GRAM_HEADROOM binades and grows (to the new largest
//    exponent plus the headroom) only when a value's exponent exceeds it:
//    with the headroom, later panels rarely raise it, and each raise costs a
//    full drain of the accumulators;
//  * digit slabs sit in shared memory in the canonical K-major layout (8x16-
//    byte core matrices; the K dimension is the row index of X and Y).  One
//    MMA multiplies J consecutive X slabs (M = 128 = J x kxp TMEM lanes) by
//    the Y slabs t = 0 .. T-1 (N = T x kyp) and writes at TMEM column offset
//    J q kyp, so the product of slabs s = Jq + j and t lands in column block
//    c = Jq + t of lane block j: column block c of lane block j collects the
//    digit diagonal d = c + j, and the 120 digit pairs with d <= 14 take
//    15 / J + 1 MMAs per 16 rows;
//  * every R rows (R such that no accumulator can exceed 2^24 in magnitude:
//    the largest per-row sum of digit-pair bounds that a column block
//    collects, group_bound below) the accumulators are read back
//    (tcgen05.ld), converted to integers, added to 32-bit running sums per
//    (lane, column) and set back to zero; a group of three column blocks
//    whose per-row bound is smaller is drained only every 2nd, 4th or 8th
//    time.  The running sums are folded into a 128-bit total W in the units
//    of the integer engine (value = W 2^(Ax + Ay - 2148)) every 8192 rows,
//    before an alignment exponent grows, and at the end.  The row-chunk
//    partials go through the same exact, order-free reduction
//    (fx_gram_reduce).
//
// Error per product x y: the dropped digit pairs (d >= 15) weigh less than
// 14.2 * 2^103 units^2 (units of 2^(Ax - 1127), 2^(Ay - 1127)), and a value
// more than 52 binades below A is truncated by less than one unit; with
// max|x| >= 2^(104 - h) units for a headroom h, the error is below
// 22.2 * 2^(2h - 105) max|x| max|y| (h = 2: 2^-96.5).  Pipeline per CTA (one
// per SM): TMA loads
// of the FP64 panels (128-byte swizzle, two panels ahead), conversion of
// panel p into one of two digit buffers while the tensor cores run panel
// p-1, one warp issuing the MMAs and committing them to an mbarrier per
// buffer.  Every wait is bounded; a wait that runs out marks the partials
// non-finite, so the result is NaN.  Inputs that TMA cannot address (a base
// address not 16-byte aligned or an odd leading dimension) are copied by the
// converter threads themselves with cp.async (the DIRECT variant).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "fx.cuh"
#include "umma.cuh"

namespace eo {
namespace {

using namespace fx;
using namespace umma;

// 19 converter warps and the MMA warp: five warps per SM sub-partition, so
// that each may hold 96 registers (a sixth warp on one of them caps every
// thread at 80, and the kernel spills).
#ifndef EO_GRAM_CONV_WARPS
#define EO_GRAM_CONV_WARPS 19
#endif
constexpr int kConvWarps = EO_GRAM_CONV_WARPS;  // staging and conversion (16 to 19)
constexpr int kDrainWarps = 16;  // the first 16 also drain TMEM: 4 per lane quarter
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kThreads = kConvThreads + 32;  // plus one MMA-issuing warp
static_assert(kConvWarps >= kDrainWarps, "every drain warp converts");
constexpr int kLanes = 128;   // MMA M = TMEM lanes
constexpr int kMaxItems = 3;  // items (two rows of one column) per thread and panel
constexpr int kOffsetDigits = 2148;
constexpr int kFoldRows = 8192;  // rows between folds of the 32-bit running sums
constexpr size_t kSmemCap = 225 * 1024;
// Binades of headroom above a column's largest exponent when its alignment
// exponent is set (see the error bound above).
#ifndef EO_GRAM_HEADROOM
#define EO_GRAM_HEADROOM 2
#endif

struct UPlan {
  int kxp, kyp, J, nq;  // X tile width (J = 128 / kxp lane blocks), Y tile width, MMAs per k-step
  int ntx, nty;         // tiles over X and Y columns
  int shared;           // X and Y are one matrix held once (symmetric, kx <= 16)
  int P;                // rows per panel (multiple of 16)
  int drain_panels;     // panels accumulated in TMEM between drains
  int fold_drains;      // drains between folds of the running sums
  int drain_log;        // 3 bits per group g of column blocks 3g..3g+2: log2 of the drains it may skip + 1
  int nslots;           // staged columns per CTA
  unsigned dig_bytes;   // one digit buffer (A part, then B part unless shared)
  unsigned a_bytes;     // A part of a digit buffer
  unsigned stage_bytes; // one staging buffer: P / 16 TMA boxes of X (16 rows x kxp), then of Y
};

// ------------------------------------------------------------ kernel
// Warps 0..kConvWarps-1 stage, scan and convert (named barrier 1), the
// first 16 of them also drain TMEM; warp kConvWarps issues the MMAs: per
// panel p it waits for ready[p & 1] (one arrival per converter thread: the
// digits of p are in buffer p & 1 and TMEM is drained if due), issues the
// MMAs and commits them to full[p & 1], which the converters wait on before
// they reuse the buffer (panel p + 2) or read TMEM.
// DIRECT: the operands cannot be read by TMA (a leading dimension that is
// not a whole number of 16-byte units, or a base that is not 16-byte
// aligned): every converter thread then copies its own items of panel p + 2
// into private shared-memory slots with 8-byte cp.async (zeros beyond the
// matrix) and reads them back at panel p; the rest is the same.
constexpr unsigned kDirectStageBytes = 2u * kMaxItems * kConvThreads * 16u;

// An FP32 value widened to FP64 exactly in integer arithmetic (the FP64
// conversion unit is slow on this GPU); zeros, subnormals, infinities and
// NaNs (the exponent field 0 or 255) take the conversion instruction.
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)f;
  return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)), (int)(b << 29));
}

// PAD: the tile has padded columns (beyond kx or ky, e.g. kx = 40 in a
// 64-column plan): their digits are zeroed once and never converted.
// T: the element type of X and Y; FP32 (the EO_F32 mode) only with DIRECT
// loads, every value widened to FP64 exactly as it is read.  KXPC, PC: the
// plan's X tile width and panel rows when known at compile time (the hot
// plans: slab strides become immediate store offsets), 0 = from the plan.
template <int KYP, bool DIRECT, bool PAD, typename T = double, int KXPC = 0, int PC = 0>
__global__ void __launch_bounds__(kThreads, 1)
    umma_gram_partial_kernel(int64_t n, int kx, const T* __restrict__ X, int64_t ldx, int ky,
                             const T* __restrict__ Y, int64_t ldy, UPlan pl, int64_t rows_per_chunk,
                             const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy,
                             FxPart* __restrict__ parts, const int* gate) {
  static_assert(sizeof(T) == 8 || DIRECT, "FP32 operands are copied by the converter threads");
  // The compile-time plans: (KXPC, PC) = (64, 32) with separate X and Y
  // (V^T Y, 64 + 16 columns) and (16, 128) with X = Y (symmetric, 16
  // columns); TMA loads, no padded columns.  Their items are numbered A
  // items first (kNA of them), then B items (kNB), so that whether an item
  // exists and which operand it belongs to is known per item slot at compile
  // time or is uniform over a warp.
  constexpr bool kHot = KXPC > 0;
  constexpr bool kHotShared = KXPC == 16;
  constexpr int kNA = kHot ? KXPC * PC / 2 : 0, kNB = kHot && !kHotShared ? KYP * PC / 2 : 0;
  static_assert(!kHot || ((KXPC == 64 && PC == 32) || (KXPC == 16 && PC == 128)), "compile-time plans");
  static_assert(!kHot || (!DIRECT && !PAD && KYP == 16), "compile-time plans load by TMA");
  static_assert(!kHot || (kNA + kNB <= kMaxItems * kConvThreads && kNA % 32 == 0 && kNB % 32 == 0),
                "compile-time plans: whole warps of items");
  if (gate && *gate == 0) return;
  // Y columns of one converter thread in a drain (four warps share a TMEM
  // lane quarter), handled NH times NY at a time
  constexpr int NYT = KYP * 4 / kDrainWarps;
  constexpr int NY = NYT < 4 ? NYT : 4;
  constexpr int NH = NYT / NY;
  const int kxp = KXPC ? KXPC : pl.kxp, P = PC ? PC : pl.P;
  const int nslots = KXPC ? (pl.shared ? KXPC : KXPC + KYP) : pl.nslots;
  const int tx = blockIdx.x / pl.nty, ty = blockIdx.x % pl.nty;
  const int x0 = tx * kxp, y0 = ty * KYP;  // first X / Y column of the tile
  const unsigned SBO = (unsigned)P * 16;   // bytes per 8-row group of a slab (P / 8 core matrices)

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base (the 128-byte swizzle of the TMA boxes is anchored there)
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* stage = smem;                                 // 2 staging buffers (TMA boxes; DIRECT: slots)
  const size_t stage_region = DIRECT ? max(2 * (size_t)pl.stage_bytes, (size_t)kDirectStageBytes)
                                     : 2 * (size_t)pl.stage_bytes;
  unsigned char* dig = stage + stage_region;                   // 2 digit buffers
  int* Erun = reinterpret_cast<int*>(dig + 2 * (size_t)pl.dig_bytes);
  int* pmax = Erun + 2 * nslots;  // three panels' column maxima (Erun: running exponents, two buffers)
  __shared__ __align__(8) unsigned long long full_bar[2], ready_bar[2], stage_bar[2];
  __shared__ unsigned tmem_base;
  __shared__ int flag, bad;
  // far[b]: the last panel in digit buffer b with an item off the near path
  // (its digit slabs 11..14 may be nonzero); written by the converters before
  // they mark the panel ready, read by the MMA warp after that
  __shared__ int far[2];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- set-up: TMEM (accumulators in columns 0..255, running sums in 256..511),
  // barriers, zero slabs, exponents
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base), 512);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&full_bar[b]), 1);
      mbar_init(smem_u32(&ready_bar[b]), kConvThreads);
      mbar_init(smem_u32(&stage_bar[b]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flag = 0;
    bad = 0;
    far[0] = far[1] = -1;
  }
  for (int c = tid; c < 5 * nslots; c += kThreads) Erun[c] = 0;  // Erun and pmax
  {  // slab 15 of every operand stays zero
    const unsigned za = (unsigned)kxp / 8u * SBO, zb = (unsigned)KYP / 8u * SBO;  // bytes of one slab
    for (int b = 0; b < 2; ++b) {
      unsigned* pa = reinterpret_cast<unsigned*>(dig + (size_t)b * pl.dig_bytes + 15u * za);
      for (unsigned e = tid; e < za / 4; e += kThreads) pa[e] = 0u;
      if (!pl.shared) {
        unsigned* pb = reinterpret_cast<unsigned*>(dig + (size_t)b * pl.dig_bytes + pl.a_bytes + 15u * zb);
        for (unsigned e = tid; e < zb / 4; e += kThreads) pb[e] = 0u;
      }
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = tmem_base;

  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min(n, r0 + rows_per_chunk);
  const int npan = r0 < r1 ? (int)((r1 - r0 + P - 1) / P) : 0;
  const unsigned dig_s = smem_u32(dig);
  const unsigned fb0 = smem_u32(&full_bar[0]), rb0 = smem_u32(&ready_bar[0]), sb0 = smem_u32(&stage_bar[0]);
  // TMA loads of panel p into staging buffer p & 1: P / 16 boxes of 16 rows per operand
  const unsigned xbox = (unsigned)kxp * 128u, ybox = (unsigned)KYP * 128u;
  auto load_panel = [&](int p) {
    const unsigned bar = sb0 + 8u * (unsigned)(p & 1);
    const unsigned dst = smem_u32(stage) + (unsigned)(p & 1) * pl.stage_bytes;
    const int xr = (int)(r0 + (int64_t)p * P);
    mbar_arrive_expect_tx(bar, pl.stage_bytes);
    for (int h = 0; h < P / 16; ++h) {
      tma_load_2d(dst + (unsigned)h * xbox, &tmx, xr + 16 * h, x0, bar);
      if (!pl.shared) tma_load_2d(dst + (unsigned)(P / 16) * xbox + (unsigned)h * ybox, &tmy, xr + 16 * h, y0, bar);
    }
  };
  if (!DIRECT && tid == 0) {
    for (int p = 0; p < 2 && p < npan; ++p) load_panel(p);
  }

  // the partial sums of this thread's lane: lane block jl (digit phase), X column xl
  const int Lq = (warp & 3) * 32, L = Lq + lane;
  const int jl = L >> (31 - __clz(kxp)), xl = L & (kxp - 1);
  const int yq = (warp >> 2) * NYT;  // first of this thread's NYT Y columns (drain warps)
  const bool drainer = warp < kDrainWarps;
  i128 W[NYT];
#pragma unroll
  for (int y = 0; y < NYT; ++y) W[y] = 0;

  if (warp == kConvWarps) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int p = 0;
      for (; p < npan; ++p) {
        const int db = p & 1;
        if (!mbar_wait(rb0 + 8u * db, (unsigned)(p >> 1) & 1u, &bad)) break;
        tc_fence_after();
        const unsigned abase = dig_s + (unsigned)db * pl.dig_bytes;
        const unsigned bbase = pl.shared ? abase : abase + pl.a_bytes;
        // every item of the panel on the near path: digit slabs 11..14 of
        // both operands are zero, and the MMAs that would only multiply them
        // are left out (exactly the same sums)
        const int ns = *reinterpret_cast<volatile int*>(&far[db]) == p ? NS : 11;
        for (int ks = 0; ks < P / 16; ++ks) {
          for (int q = 0; q < pl.nq; ++q) {
            if (pl.J * q >= ns) break;  // all of this MMA's X slabs are zero
            const int nt = min(NS - pl.J * q, ns);
            const int Tp = KYP == 16 ? nt : (nt + 1) & ~1;  // N a multiple of 16
            const unsigned long long ad =
                sdesc(abase + (unsigned)(pl.J * q * kxp / 8) * SBO + (unsigned)ks * 256u, 128u, SBO);
            const unsigned long long bd = sdesc(bbase + (unsigned)ks * 256u, 128u, SBO);
            mma_f16(taddr + (unsigned)(KYP * pl.J * q), ad, bd, idesc_f16(kLanes, KYP * Tp),
                    1u);  // the accumulators start at zero and drains zero them
          }
        }
        mma_commit(fb0 + 8u * db);
      }
      // the last committed MMAs finish before TMEM and shared memory are released
      if (p > 0) mbar_wait_final(fb0 + 8u * ((p - 1) & 1), (unsigned)((p - 1) >> 1) & 1u, &bad);
    }
    __syncwarp();
  } else {
    // ---------------- converters: staging, exponents, digits, drains
    const unsigned tacc = taddr + ((unsigned)Lq << 16) + (unsigned)yq;
    const unsigned tsum = tacc + 256u;
    if (drainer) {
      unsigned z[3][NY];
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int y = 0; y < NY; ++y) z[u][y] = 0u;
#pragma unroll
      for (int hh = 0; hh < NH; ++hh)
#pragma unroll
        for (int c0 = 0; c0 < NS; c0 += 3) {
          const unsigned ts = tsum + 4u * hh, ta = tacc + 4u * hh;
          tmem_st3<NY>(ts + c0 * KYP, ts + (c0 + 1) * KYP, ts + (c0 + 2) * KYP, z);
          tmem_st3<NY>(ta + c0 * KYP, ta + (c0 + 1) * KYP, ta + (c0 + 2) * KYP, z);
        }
      tmem_wait_st();
    }

    // TMEM accumulators -> TMEM running sums (column block c of lane block
    // jl: diagonal c + jl) for the groups of three column blocks G0 .. 4 (the
    // groups due at a drain are always such a suffix: a group's period is a
    // power of two no shorter than that of any later group); a drained
    // group's accumulators are set back to zero.  The loads of the next group
    // are in flight while a group is added.
    unsigned tacc_h = tacc, tsum_h = tsum;  // the NY columns being drained
    auto load = [&](int c0, unsigned (&v)[3][NY], unsigned (&sm)[3][NY]) {
      tmem_ld3x2_nowait<NY>(tacc_h + c0 * KYP, tacc_h + (c0 + 1) * KYP, tacc_h + (c0 + 2) * KYP, tsum_h + c0 * KYP,
                            tsum_h + (c0 + 1) * KYP, tsum_h + (c0 + 2) * KYP, v, sm);
    };
    auto add_store = [&](int c0, unsigned (&v)[3][NY], unsigned (&sm)[3][NY]) {
      // (column blocks with c + jl > 14 collect no kept diagonal: the fold skips them)
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int y = 0; y < NY; ++y) sm[u][y] += (unsigned)__float2int_rn(__uint_as_float(v[u][y]));
      tmem_st3<NY>(tsum_h + c0 * KYP, tsum_h + (c0 + 1) * KYP, tsum_h + (c0 + 2) * KYP, sm);
      tmem_zero3<NY>(tacc_h + c0 * KYP, tacc_h + (c0 + 1) * KYP, tacc_h + (c0 + 2) * KYP);
    };
    auto drain_from = [&](auto g0) {
      constexpr int G0 = decltype(g0)::value;
      unsigned va[3][NY], sa[3][NY], vb[3][NY], sb[3][NY];
      load(3 * G0, va, sa);
      tmem_wait_ld_regs<NY>(va, sa);
      if constexpr (G0 + 1 <= 4) load(3 * (G0 + 1), vb, sb);
      add_store(3 * G0, va, sa);
      if constexpr (G0 + 1 <= 4) {
        tmem_wait_ld_regs<NY>(vb, sb);
        if constexpr (G0 + 2 <= 4) load(3 * (G0 + 2), va, sa);
        add_store(3 * (G0 + 1), vb, sb);
      }
      if constexpr (G0 + 2 <= 4) {
        tmem_wait_ld_regs<NY>(va, sa);
        if constexpr (G0 + 3 <= 4) load(3 * (G0 + 3), vb, sb);
        add_store(3 * (G0 + 2), va, sa);
      }
      if constexpr (G0 + 3 <= 4) {
        tmem_wait_ld_regs<NY>(vb, sb);
        if constexpr (G0 + 4 <= 4) load(3 * (G0 + 4), va, sa);
        add_store(3 * (G0 + 3), vb, sb);
      }
      if constexpr (G0 + 4 <= 4) {
        tmem_wait_ld_regs<NY>(va, sa);
        add_store(3 * (G0 + 4), va, sa);
      }
      tmem_wait_st();
    };
    auto drain = [&](int g0) {
#pragma unroll
      for (int hh = 0; hh < NH; ++hh) {
        tacc_h = tacc + 4u * hh;
        tsum_h = tsum + 4u * hh;
        switch (g0) {
          case 0: drain_from(std::integral_constant<int, 0>{}); break;
          case 1: drain_from(std::integral_constant<int, 1>{}); break;
          case 2: drain_from(std::integral_constant<int, 2>{}); break;
          case 3: drain_from(std::integral_constant<int, 3>{}); break;
          case 4: drain_from(std::integral_constant<int, 4>{}); break;
          default: break;  // no group due
        }
      }
    };
    auto fold = [&]() {  // running sums -> W (units 2^(Ax + Ay - 2148)), sums back to zero
#pragma unroll
      for (int hh = 0; hh < NH; ++hh) {
        const unsigned ts = tsum + 4u * hh;
        i128 h[NY];
#pragma unroll
        for (int y = 0; y < NY; ++y) h[y] = 0;
#pragma unroll
        for (int c0 = 0; c0 < NS; c0 += 3) {
          unsigned sm[3][NY];
          tmem_ld3<NY>(ts + c0 * KYP, ts + (c0 + 1) * KYP, ts + (c0 + 2) * KYP, sm);
#pragma unroll
          for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int y = 0; y < NY; ++y)
              if (c0 + u + jl <= 14) h[y] = (h[y] << 7) + (i128)(int)sm[u][y];
#pragma unroll
          for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int y = 0; y < NY; ++y) sm[u][y] = 0u;
          tmem_st3<NY>(ts + c0 * KYP, ts + (c0 + 1) * KYP, ts + (c0 + 2) * KYP, sm);
        }
        tmem_wait_st();
#pragma unroll
        for (int y = 0; y < NY; ++y) W[hh * NY + y] += h[y] >> 8;
      }
    };

    // This thread's items (two rows of one column) of every panel: i = tid +
    // k * kConvThreads.  Within a warp, lanes l, l ^ 8, l ^ 16, l ^ 24 share a column,
    // the eight columns of a quarter warp read distinct 16-byte chunks of the
    // swizzled boxes, and the 32 digit words a warp stores per slab fill 128
    // contiguous bytes.  it_s: column << 16 | staging offset / 16; it_d:
    // digit offset | B operand << 31.
    // Item i of a panel goes to thread slot i % kConvThreads, slot k = i /
    // kConvThreads; thread tid holds slot titem, rotated so that the slots
    // past the last whole round of items (the third item of some threads)
    // fall to the converter warps that do not drain TMEM.  In the hot plans
    // the kNA items of the A operand come first and the kNB items of the B
    // operand after them (item_valid, item_b below).
    const int titem = (tid + 32 * (kConvWarps - kDrainWarps)) % kConvThreads;
    const int half = P >> 1, ncg = nslots >> 3;
    const int nitems = nslots * half;
    unsigned it_s[kMaxItems], it_d[kMaxItems];
#pragma unroll
    for (int k = 0; k < kMaxItems; ++k) {
      int c, rh, cl, rl;
      if constexpr (kHot) {
        // an empty slot (past the kNA + kNB items) takes item 0's column, so
        // that every column index stays below nslots
        const int i0 = titem + k * kConvThreads;
        const bool live = i0 < kNA + kNB;
        const bool kb = live && i0 >= kNA;
        const int i = kb ? i0 - kNA : (live ? i0 : 0);
        const int g = kb ? KYP / 8 : KXPC / 8;  // column groups of the operand
        cl = i & 7;
        rl = (i >> 3) & 3;
        c = ((i >> 5) % g) * 8 + cl + (kb ? KXPC : 0);
        rh = (i >> 5) / g;
      } else {
        const int i = titem + k * kConvThreads;
        cl = i & 7;
        rl = (i >> 3) & 3;
        c = ((i >> 5) % ncg) * 8 + cl;
        rh = (i >> 5) / ncg;
      }
      const int r = (rh * 4 + rl) * 2;
      const bool isb = !pl.shared && c >= kxp;
      const int lc = isb ? c - kxp : c;
      const unsigned so = (isb ? (unsigned)(P / 16) * xbox : 0u) + (unsigned)(r >> 4) * (isb ? ybox : xbox) +
                          (unsigned)lc * 128u + ((((unsigned)(r & 15) >> 1) ^ (unsigned)(lc & 7)) << 4);
      it_s[k] = ((unsigned)c << 16) | (so >> 4);
      it_d[k] = ((isb ? pl.a_bytes : 0u) + (unsigned)(lc >> 3) * SBO + (unsigned)rh * 128u +
                 (unsigned)(lc & 7) * 16u + (unsigned)rl * 4u) |
                ((unsigned)isb << 31);
      if constexpr (PAD) {  // bit 30: a padded column, whose digits stay zero
        if (titem + k * kConvThreads < nitems && !(isb ? y0 + lc < ky : x0 + lc < kx)) it_d[k] |= 1u << 30;
      }
    }
    // item k exists for this thread; it belongs to the B operand
    auto item_valid = [&](int k) -> bool {
      if constexpr (kHot) {
        if (k * kConvThreads >= kNA + kNB) return false;
        if ((k + 1) * kConvThreads <= kNA + kNB) return true;
        return titem + k * kConvThreads < kNA + kNB;
      } else {
        return titem + k * kConvThreads < nitems;
      }
    };
    auto item_b = [&](int k) -> bool {
      if constexpr (kHot) {
        if (kNB == 0 || (k + 1) * kConvThreads <= kNA) return false;
        if (k * kConvThreads >= kNA) return true;
        return titem + k * kConvThreads >= kNA;
      } else {
        return (it_d[k] >> 31) != 0u;
      }
    };
    const unsigned stride_a = (unsigned)kxp / 8u * SBO, stride_b = (unsigned)KYP / 8u * SBO;
    if constexpr (PAD) {  // the digit words of padded columns: zero once, in both buffers
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        if (it_d[k] & 0x40000000u) {
          for (int b = 0; b < 2; ++b) {
            unsigned char* d = dig + (size_t)b * pl.dig_bytes + (it_d[k] & 0x3fffffffu);
            const unsigned strd = (it_d[k] >> 31) ? stride_b : stride_a;
            for (int sl = 0; sl < NS; ++sl) *reinterpret_cast<unsigned*>(d + sl * strd) = 0u;
          }
        }
      }
    }

    // DIRECT: each item's column (null: zeros) and row offset in the panel
    const T* gcol[kMaxItems];
    int irow[kMaxItems];
    const unsigned slot0 = smem_u32(stage) + (unsigned)tid * 16u;
    // a copy of no bytes (a row past the chunk: the slot is zero-filled) names
    // the partials array as its source, an address that is always valid
    const T* zsrc = reinterpret_cast<const T*>(parts);
    auto prefetch = [&](int pp) {  // this thread's items of panel pp into slot buffer pp & 1
      const int64_t base = r0 + (int64_t)pp * P;
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        if (!gcol[k]) continue;
        const int64_t row = base + irow[k];
        const unsigned d = slot0 + (unsigned)(((pp & 1) * kMaxItems + k) * kConvThreads) * 16u;
        if constexpr (sizeof(T) == 8) {
          cp_async8z(d, row < r1 ? gcol[k] + row : zsrc, row < r1 ? 8u : 0u);
          cp_async8z(d + 8u, row + 1 < r1 ? gcol[k] + row + 1 : zsrc, row + 1 < r1 ? 8u : 0u);
        } else {
          cp_async4z(d, row < r1 ? gcol[k] + row : zsrc, row < r1 ? 4u : 0u);
          cp_async4z(d + 4u, row + 1 < r1 ? gcol[k] + row + 1 : zsrc, row + 1 < r1 ? 4u : 0u);
        }
      }
      cp_async_commit_group();
    };
    if constexpr (DIRECT) {
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        const int i = titem + k * kConvThreads;
        const int cl = i & 7, rl = (i >> 3) & 3, rest = i >> 5;
        const int c = (rest % ncg) * 8 + cl, rh = rest / ncg;
        const bool isb = !pl.shared && c >= kxp;
        const int lc = isb ? c - kxp : c, gc = isb ? y0 + lc : x0 + lc;
        const bool ok = i < nitems && gc < (isb ? ky : kx);
        gcol[k] = ok ? (isb ? Y + (size_t)gc * ldy : X + (size_t)gc * ldx) : nullptr;
        irow[k] = (rh * 4 + rl) * 2;
      }
      prefetch(0);
      prefetch(1);
    }

    // One barrier per panel.  The values of panel p are in registers and
    // the maxima of its columns complete in pmax[p % 3] when panel p begins
    // (both done during panel p-1): a converter aligns and converts p, drains
    // TMEM if due, marks p ready for the MMA warp, then reads and scans panel
    // p+1 while those MMAs run; the barrier that ends the panel completes
    // that scan.  The running exponents through panel q sit in Erun[q & 1],
    // the maxima of panel q in pmax[q % 3]; a buffer is rewritten only after
    // the barrier that follows its last read.
    auto stage_values = [&](int q, double2 (&v)[kMaxItems]) {  // this thread's items of panel q
      if constexpr (DIRECT) {
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // panel q's copies (q + 1's may be in flight)
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
          const unsigned char* slot = stage + ((size_t)((q & 1) * kMaxItems + k) * kConvThreads + tid) * 16u;
          if constexpr (sizeof(T) == 8) {
            v[k] = gcol[k] ? *reinterpret_cast<const double2*>(slot) : make_double2(0.0, 0.0);
          } else {
            const float2 f = gcol[k] ? *reinterpret_cast<const float2*>(slot) : make_float2(0.0f, 0.0f);
            v[k] = make_double2(widen(f.x), widen(f.y));
          }
        }
        prefetch(q + 2);  // into the slots just read (zeros past the chunk)
      } else {
        mbar_wait(sb0 + 8u * (unsigned)(q & 1), (unsigned)(q >> 1) & 1u, &bad);  // panel q staged
        const unsigned char* st = stage + (size_t)(q & 1) * pl.stage_bytes;
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k)
          v[k] = item_valid(k) ? *reinterpret_cast<const double2*>(st + ((it_s[k] & 0xffffu) << 4))
                               : make_double2(0.0, 0.0);
      }
    };
    // largest exponent of each column of a panel into pmq (the exponent
    // field of the larger |x| bit pattern; bit 0 set when any bit is, so
    // that subnormals count) where it exceeds the column's running
    // exponent, one shared-memory atomic per such item (cheaper than
    // reducing the four items of a column in a warp by shuffles first);
    // true if one of this thread's columns exceeds te[k], its nonzero
    // running exponent
    auto scan = [&](const double2 (&v)[kMaxItems], int* pmq, const int (&te)[kMaxItems]) -> bool {
      bool g = false;
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        if (!item_valid(k)) continue;  // an empty slot
        // the larger magnitude's bit pattern; its exponent exceeds te[k]
        // exactly when the pattern reaches (te[k] + 1) << 20.  A panel's
        // maxima are only ever used as max(running exponent, panel
        // maximum), so an item within its column's running exponent changes
        // nothing (with steady exponents, nearly all items).  Subnormals
        // (exponent field 0) never raise a column: its alignment exponent is
        // at least 1 anyway.  Items past the panel's end hold zeros.
        const unsigned m = max(hi32(v[k].x) & 0x7fffffffu, hi32(v[k].y) & 0x7fffffffu);
        if (m >= ((unsigned)te[k] + 1u) << 20) {
          const int e = (int)(m >> 20);
          if (e == 2047) flag = 1;
          atomicMax(&pmq[it_s[k] >> 16], e + EO_GRAM_HEADROOM);
          g |= te[k] != 0;
        }
      }
      return g;
    };

    double2 v[kMaxItems];
    bool grew = false;  // a column of the current panel exceeds its running exponent
    if (npan > 0) {
      stage_values(0, v);
      const int none[kMaxItems] = {};
      (void)scan(v, pmax, none);  // nothing has accumulated yet
    }
    bar_conv<kConvThreads>();
    if (!DIRECT && tid == 0 && 2 < npan) {  // staging buffer 0 is read: panel 2
      fence_proxy_async();
      load_panel(2);
    }

    int undrained = 0, drains = 0, ev = 0, pc = 0;  // ev: drains since the last full one
    for (int p = 0; p < npan; ++p) {
      const int db = p & 1;
      const int pn = pc == 2 ? 0 : pc + 1, pz = pn == 2 ? 0 : pn + 1;  // (p + 1) % 3, (p + 2) % 3
      const int* eprev = Erun + (db ^ 1) * nslots;  // through panel p-1
      const int* pcur = pmax + pc * nslots;         // panel p
      if (tid < nslots) {
        Erun[db * nslots + tid] = max(eprev[tid], pcur[tid]);  // through panel p
        pmax[pz * nslots + tid] = 0;                           // panel p-1's, read for the last time in p-1
      }
      int A[kMaxItems], te[kMaxItems];  // te: running exponent through panel p of the item's column
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        const int c = (int)(it_s[k] >> 16);
        te[k] = max(eprev[c], pcur[c]);
        A[k] = max(te[k], 1);
      }

      // the digit buffer db is free once the MMAs of panel p-2 are done
      if (p >= 2) mbar_wait(fb0 + 8u * db, (unsigned)((p - 2) >> 1) & 1u, &bad);
      // digits of panel p
      unsigned char* dbuf = dig + (size_t)db * pl.dig_bytes;
      const unsigned e1024 = exp1024x2();
      bool off_near = false;  // an item of this warp took the general path
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) {
        const bool valid = item_valid(k) && (!PAD || !(it_d[k] & 0x40000000u));
        // every value of the warp's items normal and within 20 binades of its
        // alignment exponent (nearly always): the words without selects
        const bool near =
            __all_sync(0xffffffffu, !valid || min(abs_hi(v[k].x), abs_hi(v[k].y)) >= near_floor(A[k]));
        off_near |= !near;
        if (valid) {
          unsigned wa[4], wb[4];
          const unsigned signs = ((hi32(v[k].x) >> 31) << 15) | (hi32(v[k].y) & 0x80000000u);
          // operand A or B (warp-uniform; known at compile time in the hot
          // plans): two copies of the stores, so that with a compile-time
          // plan the slab stride is an immediate offset
          unsigned char* dst = dbuf + (it_d[k] & (PAD ? 0x3fffffffu : 0x7fffffffu));
          if (near) {
            xwords_near(v[k].x, 52 - A[k], wa);
            xwords_near(v[k].y, 52 - A[k], wb);
            add_bias_near(wa);
            add_bias_near(wb);
            if (item_b(k))
              store_bal_digits_near<0>(dst, stride_b, pair_lanes(wa, wb), pair_sign(signs, e1024));
            else
              store_bal_digits_near<0>(dst, stride_a, pair_lanes(wa, wb), pair_sign(signs, e1024));
          } else {
            xwords(v[k].x, A[k], wa);
            xwords(v[k].y, A[k], wb);
            add_bias(wa);
            add_bias(wb);
            if (item_b(k))
              store_bal_digits<0>(dst, stride_b, pair_lanes(wa, wb), pair_sign(signs, e1024));
            else
              store_bal_digits<0>(dst, stride_a, pair_lanes(wa, wb), pair_sign(signs, e1024));
          }
        }
      }
      if (off_near && lane == 0) far[db] = p;
      fence_proxy_async();

      // this thread's accumulators (its own TMEM lanes and columns) are drained
      // before it marks panel p ready
      if ((grew || undrained >= pl.drain_panels) && undrained > 0) {
        // a full drain before a fold or a growth; otherwise the groups whose
        // period ends here
        const bool full = grew || drains + 1 == pl.fold_drains;
        int g0 = 0;  // first group due
        if (!full) {
          g0 = 5;
#pragma unroll
          for (int g = 4; g >= 0; --g) {
            const int per = 1 << ((pl.drain_log >> (3 * g)) & 7);
            if (g0 == g + 1 && ((ev + 1) & (per - 1)) == 0) g0 = g;
          }
        }
        if (drainer) {
          // all MMAs so far (the last commit is panel p-1's) are done before TMEM is read
          mbar_wait(fb0 + 8u * ((p - 1) & 1), (unsigned)((p - 1) >> 1) & 1u, &bad);
          tc_fence_after();
          drain(g0);
          if (full) fold();
        }
        ++drains;
        ++ev;
        if (full) {
          drains = 0;
          ev = 0;
        }
        if (grew && drainer) {  // totals onto the new grid: divide by 2^(growth of both columns' exponents)
          const int ysb = pl.shared ? 0 : kxp;
#pragma unroll
          for (int y = 0; y < NYT; ++y) {
            const int cx = xl, cy = ysb + yq + y;
            const int dx = eprev[cx] ? max(eprev[cx], pcur[cx]) - eprev[cx] : 0;
            const int dy = eprev[cy] ? max(eprev[cy], pcur[cy]) - eprev[cy] : 0;
            W[y] = w_shift(W[y], dx + dy);
          }
        }
        tc_fence_before();
        undrained = 0;
      }
      mbar_arrive(rb0 + 8u * db);  // digits of p ready (and TMEM drained if it was due)
      ++undrained;

      // panel p+1: values and column maxima (growth against the exponents through p)
      bool gl = false;
      double2 vn[kMaxItems];
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) vn[k] = make_double2(0.0, 0.0);
      if (p + 1 < npan) {
        stage_values(p + 1, vn);
        gl = scan(vn, pmax + pn * nslots, te);
      }
      grew = bar_conv_or<kConvThreads>(gl);
      if (!DIRECT && tid == 0 && p + 3 < npan) {  // staging buffer (p + 1) & 1 is read: panel p + 3
        fence_proxy_async();
        load_panel(p + 3);
      }
#pragma unroll
      for (int k = 0; k < kMaxItems; ++k) v[k] = vn[k];
      pc = pn;
    }

    if constexpr (DIRECT) asm volatile("cp.async.wait_all;" ::: "memory");  // the last (empty) copies
    // last drain and fold
    if (npan > 0 && drainer) {
      mbar_wait(fb0 + 8u * ((npan - 1) & 1), (unsigned)((npan - 1) >> 1) & 1u, &bad);
      tc_fence_after();
      drain(0);
      fold();
      tc_fence_before();
    }
  }

  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 512);
  }

  // sum the lane blocks (digit phase j) of every output and write the partials
  i128* red = reinterpret_cast<i128*>(dig);  // 128 lanes x KYP entries (the MMAs are done)
  if (warp < kDrainWarps) {
#pragma unroll
    for (int y = 0; y < NYT; ++y) red[L * KYP + yq + y] = W[y];
  }
  __syncthreads();
  const int J = pl.J;
  const int* Efin = Erun + ((npan - 1) & 1) * nslots;  // running exponents through the last panel
  for (int e = tid; e < kxp * KYP; e += kThreads) {
    const int xo = e / KYP, yo = e % KYP;
    const int i = x0 + xo, j = y0 + yo;
    if (i >= kx || j >= ky) continue;
    i128 w = 0;
    for (int b = 0; b < J; ++b) w += red[(b * kxp + xo) * KYP + yo];
    const int cy = pl.shared ? yo : kxp + yo;
    FxPart o;
    o.wl = (long long)(unsigned long long)(u128)w;
    o.wh = (long long)(w >> 64);
    o.s = max(Efin[xo], 1) + max(Efin[cy], 1) - kOffsetDigits;
    o.flag = flag | bad;
    o.pad = 0;
    parts[(size_t)blockIdx.y * ((size_t)kx * ky) + (size_t)j * kx + i] = o;
  }
}

// ------------------------------------------------------------ host side
int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Largest |digit| of slab s: balanced digits are in [-64, 63] except the top
// one, in [-64, 128].
constexpr long long digit_bound(int s) { return s == 0 ? 128 : 64; }

// Largest per-row sum of |D_s D_t| that a column block c in [c0, c1] of any
// lane block j collects: the pairs (s, t) = (J q + j, c - J q) with J q <= c
// and J q + j <= 14.
long long group_bound(int c0, int c1, int J) {
  long long worst = 0;
  for (int c = c0; c <= c1; ++c)
    for (int j = 0; j < J; ++j) {
      long long b = 0;
      for (int q = 0; J * q <= c && J * q + j <= 14; ++q) b += digit_bound(J * q + j) * digit_bound(c - J * q);
      worst = std::max(worst, b);
    }
  return worst;
}

UPlan make_plan(int kx, int ky, bool sym) {
  UPlan p{};
  if (sym && kx <= 16) {
    p.shared = 1;
    p.kxp = 16;
    p.kyp = 16;
  } else {
    p.kxp = std::min(128, std::max(16, pow2_at_least(kx)));
    p.kyp = ky <= 8 ? 8 : 16;
  }
  p.J = kLanes / p.kxp;
  p.nq = 14 / p.J + 1;
  p.ntx = (kx + p.kxp - 1) / p.kxp;
  p.nty = p.shared ? 1 : (ky + p.kyp - 1) / p.kyp;
  p.nslots = p.shared ? p.kxp : p.kxp + p.kyp;
  // rows an accumulator may absorb: the largest sum of digit-pair bounds
  // that one column block collects per row (below 2^24 in total)
  const long long row_bound = group_bound(0, 14, p.J);
  const int rows_cap = (int)((1ll << 24) / row_bound);
  int best = 16;
  for (int P = 16; P <= 128; P *= 2) {
    if (P > rows_cap || (size_t)p.nslots * P / 2 > (size_t)kMaxItems * kConvThreads) break;
    const size_t dig = (size_t)32 * P * (p.shared ? p.kxp : p.kxp + p.kyp);
    const size_t stg = (size_t)p.nslots * P * 8;
    const size_t red = (size_t)kLanes * p.kyp * 16;
    if (std::max(2 * dig, red) + 2 * stg + 20 * (size_t)p.nslots + 1024 > kSmemCap) break;
    best = P;
  }
  p.P = best;
  p.drain_panels = std::max(1, rows_cap / p.P);
  // a drain adds at most drain rows x row_bound to a 32-bit running sum
  const long long per_drain = (long long)p.drain_panels * p.P * row_bound;
  p.fold_drains = (int)std::max(1ll, std::min<long long>(kFoldRows / (p.drain_panels * p.P),
                                                          ((1ll << 31) - 1) / per_drain));
  // Column block c of a lane block collects at most c / J + 1 digit pairs
  // per row, so a group of three blocks stays exact for 2^24 / (its largest
  // per-row bound) rows: it is drained every 2^g-th drain (g <= 3).
  p.drain_log = 0;
  for (int g = 0; g < 5; ++g) {
    const long long dmax = (1ll << 24) / (group_bound(3 * g, std::min(3 * g + 2, 14), p.J) * p.drain_panels * p.P);
    int lg = 0;
    while (lg < 3 && (2ll << lg) <= dmax) ++lg;
    p.drain_log |= lg << (3 * g);
  }
  p.a_bytes = (unsigned)(32 * p.P * p.kxp);
  p.dig_bytes = (unsigned)(32 * p.P * (p.shared ? p.kxp : p.kxp + p.kyp));
  p.stage_bytes = (unsigned)(p.nslots * p.P * 8);
  return p;
}

size_t plan_smem(const UPlan& p) {
  const size_t red = (size_t)kLanes * p.kyp * 16;
  return std::max(2 * (size_t)p.dig_bytes, red) + 2 * (size_t)p.stage_bytes + 5 * sizeof(int) * p.nslots + 1024;
}

int num_chunks(int64_t n, const UPlan& p) {
  const int tiles = p.ntx * p.nty;
  const int64_t by_rows = (n + p.P - 1) / p.P;
  const int64_t want = std::max<int64_t>(1, (152 + tiles - 1) / tiles);  // one CTA per SM
  const int64_t need = (n + (1ll << 22) - 1) >> 22;                     // <= 2^22 rows per chunk
  return (int)std::max<int64_t>(1, std::min(by_rows, std::max(want, need)));
}

// Row chunks under a cap of ctas CTAs (0 = none): never more than num_chunks
// (the scratch is sized for it), never fewer than the 2^22-row bound needs.
int capped_chunks(int64_t n, const UPlan& p, int ctas) {
  const int c = num_chunks(n, p);
  if (ctas <= 0) return c;
  const int64_t need = (n + (1ll << 22) - 1) >> 22;
  const int64_t cap = std::max<int64_t>(1, ctas / (p.ntx * p.nty));
  return (int)std::max<int64_t>(std::max<int64_t>(1, need), std::min<int64_t>(c, cap));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// Tensor map of a column-major n-by-k FP64 matrix: boxes of 16 rows x w columns.
bool make_map(CUtensorMap* m, const double* A, int64_t n, int k, int64_t ld, int w) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)std::max<int64_t>(n, 1), (cuuint64_t)k};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 8u};
  const cuuint32_t box[2] = {16u, (cuuint32_t)w};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(A), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t plan_smem_direct(const UPlan& p) {
  return plan_smem(p) - 2 * (size_t)p.stage_bytes + std::max<size_t>(2 * (size_t)p.stage_bytes, kDirectStageBytes);
}

template <int KYP, bool DIRECT, bool PAD, typename T = double, int KXPC = 0, int PC = 0>
cudaError_t launch_kernel(const UPlan& plan, int chunks, int64_t n, int kx, const T* X, int64_t ldx, int ky,
                          const T* Y, int64_t ldy, int64_t rpc, const CUtensorMap& tmx, const CUtensorMap& tmy,
                          FxPart* parts, const int* gate, cudaStream_t st) {
  const size_t smem = DIRECT ? plan_smem_direct(plan) : plan_smem(plan);
  cudaError_t e = set_dyn_smem(umma_gram_partial_kernel<KYP, DIRECT, PAD, T, KXPC, PC>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(plan.ntx * plan.nty, chunks);
  umma_gram_partial_kernel<KYP, DIRECT, PAD, T, KXPC, PC>
      <<<grid, kThreads, smem, st>>>(n, kx, X, ldx, ky, Y, ldy, plan, rpc, tmx, tmy, parts, gate);
  return cudaGetLastError();
}

// One thread waits for a phase of an mbarrier that nothing completes, bounded
// by limit_ns: the bounded-wait path of the tensor-core kernels, exercised on
// its own (it records the expiry like any other wait that runs out).
__global__ void wait_selftest_kernel(unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  (void)mbar_wait(smem_u32(&bar), 0u, &abort_flag, limit_ns);
}

}  // namespace

cudaError_t umma_wait_selftest(unsigned long long limit_ns, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns);
  return cudaGetLastError();
}

cudaError_t umma_gram_take_wait_record(unsigned* out) { return take_wait_record(out); }

namespace {

// How one product reaches its operands: by TMA (tensor maps) or by the
// converter threads' own copies (direct); neither: the integer limbs.
struct Route {
  UPlan plan;
  bool tma_ok, direct;
  CUtensorMap tmx, tmy;
};
void route(Route& r, int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
           bool sym) {
  r.plan = make_plan(kx, ky, sym);
  r.tmx = CUtensorMap{};
  r.tmy = CUtensorMap{};
  // TMA addresses 16-byte aligned bases and leading dimensions of whole 16-byte units
  r.tma_ok = (uintptr_t)X % 16 == 0 && (uintptr_t)Y % 16 == 0 && ldx % 2 == 0 && ldy % 2 == 0 && n < (1ll << 31) &&
             make_map(&r.tmx, X, n, kx, ldx, r.plan.kxp) && make_map(&r.tmy, Y, n, ky, ldy, r.plan.kyp);
  // EO_DD_GRAM_LOADS=direct uses the copies for TMA-addressable operands too.
  const char* lm = getenv("EO_DD_GRAM_LOADS");
  const bool force_direct = lm && lm[0] == 'd';
  r.direct = (!r.tma_ok || force_direct) && (uintptr_t)X % 8 == 0 && (uintptr_t)Y % 8 == 0 &&
             plan_smem_direct(r.plan) <= kSmemCap;
}

// A symmetric product with more than 16 columns runs as column strips of 16:
// strip c0 .. c1 - 1 is X[:, 0:c1]^T X[:, c0:c1] (the first one the symmetric
// 16-column product), of which the reduction keeps the entries on and above
// the diagonal of G and mirrors them (so G is exactly symmetric).  Each
// value is converted once per strip that reads it, where the one-tile plans
// of X^T Y over all columns convert it once per 16-column Y tile and once
// more as the Y operand.
bool use_strips(int64_t n, int kx, const double* X, int64_t ldx, bool sym) {
  if (!sym || kx <= 16) return false;
  for (int c0 = 0; c0 < kx; c0 += 16) {
    const int c1 = std::min(kx, c0 + 16);
    Route r;
    route(r, n, c1, X, ldx, c1 - c0, X + (size_t)c0 * ldx, ldx, c0 == 0);
    if (!r.tma_ok && !r.direct) return false;
  }
  return true;
}

cudaError_t launch_one(const Route& r, int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y,
                       int64_t ldy, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                       cudaStream_t st, int ctas, bool sym, int jo) {
  const UPlan& plan = r.plan;
  const bool direct = r.direct;
  const CUtensorMap& tmx = r.tmx;
  const CUtensorMap& tmy = r.tmy;
  const int chunks = capped_chunks(n, plan, ctas);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = std::max<int64_t>(plan.P, (rpc + plan.P - 1) / plan.P * plan.P);
  FxPart* parts = static_cast<FxPart*>(scratch);
  const bool pad = plan.ntx * plan.kxp > kx || (!plan.shared && plan.nty * plan.kyp > ky);
  cudaError_t e;
#define EO_UMMA_LAUNCH(K, D, PD) \
  launch_kernel<K, D, PD>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tmx, tmy, parts, gate, st)
  // the two plans of the projection step: V^T Y (64 + 16 columns, 32-row
  // panels) and a symmetric 16-column Gram (128-row panels)
  const bool hot_vty = !direct && !pad && plan.kyp == 16 && !plan.shared && plan.kxp == 64 && plan.P == 32;
  const bool hot_sym = !direct && !pad && plan.kyp == 16 && plan.shared && plan.kxp == 16 && plan.P == 128;
  if (hot_vty)
    e = launch_kernel<16, false, false, double, 64, 32>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tmx, tmy, parts,
                                                        gate, st);
  else if (hot_sym)
    e = launch_kernel<16, false, false, double, 16, 128>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tmx, tmy,
                                                         parts, gate, st);
  else if (plan.kyp == 16)
    e = direct ? (pad ? EO_UMMA_LAUNCH(16, true, true) : EO_UMMA_LAUNCH(16, true, false))
               : (pad ? EO_UMMA_LAUNCH(16, false, true) : EO_UMMA_LAUNCH(16, false, false));
  else
    e = direct ? (pad ? EO_UMMA_LAUNCH(8, true, true) : EO_UMMA_LAUNCH(8, true, false))
               : (pad ? EO_UMMA_LAUNCH(8, false, true) : EO_UMMA_LAUNCH(8, false, false));
#undef EO_UMMA_LAUNCH
  if (e != cudaSuccess) return e;
  return launch_fx_reduce(kx, ky, sym, chunks, parts, G_hi, G_lo, ldg, gate, st, jo);
}

}  // namespace

size_t umma_gram_scratch_bytes(int64_t n, int kx, int ky, bool sym) {
  if (sym) ky = kx;
  size_t b = (size_t)num_chunks(n, make_plan(kx, ky, sym)) * (size_t)kx * ky * sizeof(FxPart);
  if (sym && kx > 16) {  // the column strips (one after another: the largest)
    for (int c0 = 0; c0 < kx; c0 += 16) {
      const int c1 = std::min(kx, c0 + 16);
      b = std::max(b, (size_t)num_chunks(n, make_plan(c1, c1 - c0, c0 == 0)) * (size_t)c1 * (c1 - c0) *
                          sizeof(FxPart));
    }
  }
  return b;
}

int umma_gram_ctas(int64_t n, int kx, int ky, bool sym, int ctas) {
  if (sym) ky = kx;
  const UPlan plan = make_plan(kx, ky, sym);
  int c = plan.ntx * plan.nty * capped_chunks(n, plan, ctas);
  if (sym && kx > 16) {
    for (int c0 = 0; c0 < kx; c0 += 16) {
      const int c1 = std::min(kx, c0 + 16);
      const UPlan ps = make_plan(c1, c1 - c0, c0 == 0);
      c = std::max(c, ps.ntx * ps.nty * capped_chunks(n, ps, ctas));
    }
  }
  return c;
}

int umma_gram_launches(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                       bool sym) {
  (void)ky;
  (void)Y;
  (void)ldy;
  return use_strips(n, kx, X, ldx, sym) ? 2 * ((kx + 15) / 16) : 2;
}

cudaError_t launch_umma_gram(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y, int64_t ldy,
                             bool sym, void* scratch, double* G_hi, double* G_lo, int ldg, const int* gate,
                             cudaStream_t st, int ctas) {
  if (sym) {
    Y = X;
    ldy = ldx;
    ky = kx;
  }
  if (use_strips(n, kx, X, ldx, sym)) {
    for (int c0 = 0; c0 < kx; c0 += 16) {
      const int c1 = std::min(kx, c0 + 16);
      const double* Xs = X + (size_t)c0 * ldx;
      Route r;
      route(r, n, c1, X, ldx, c1 - c0, Xs, ldx, c0 == 0);
      cudaError_t e =
          launch_one(r, n, c1, X, ldx, c1 - c0, Xs, ldx, scratch, G_hi, G_lo, ldg, gate, st, ctas, true, c0);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  Route r;
  route(r, n, kx, X, ldx, ky, Y, ldy, sym);
  // without TMA: the converters copy their own items (when the slots fit), else the integer limbs
  if (!r.tma_ok && !r.direct)
    return launch_fx_gram(n, kx, X, ldx, ky, Y, ldy, sym, scratch, G_hi, G_lo, ldg, gate, st, ctas);
  return launch_one(r, n, kx, X, ldx, ky, Y, ldy, scratch, G_hi, G_lo, ldg, gate, st, ctas, sym, 0);
}

bool umma_gram_f32_supported(const float* X, const float* Y, int kx, int ky, bool sym) {
  if (sym) {
    Y = X;
    ky = kx;
  }
  return (uintptr_t)X % 4 == 0 && (uintptr_t)Y % 4 == 0 && plan_smem_direct(make_plan(kx, ky, sym)) <= kSmemCap;
}

cudaError_t launch_umma_gram_f32(int64_t n, int kx, const float* X, int64_t ldx, int ky, const float* Y,
                                 int64_t ldy, bool sym, void* scratch, double* G_hi, double* G_lo, int ldg,
                                 const int* gate, cudaStream_t st) {
  if (sym) {
    Y = X;
    ldy = ldx;
    ky = kx;
  }
  const UPlan plan = make_plan(kx, ky, sym);
  alignas(64) CUtensorMap tm{};  // unused: FP32 operands are copied by the converter threads
  const int chunks = capped_chunks(n, plan, 0);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = std::max<int64_t>(plan.P, (rpc + plan.P - 1) / plan.P * plan.P);
  FxPart* parts = static_cast<FxPart*>(scratch);
  const bool pad = plan.ntx * plan.kxp > kx || (!plan.shared && plan.nty * plan.kyp > ky);
  cudaError_t e;
  if (plan.kyp == 16)
    e = pad ? launch_kernel<16, true, true, float>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tm, tm, parts, gate, st)
            : launch_kernel<16, true, false, float>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tm, tm, parts, gate,
                                                    st);
  else
    e = pad ? launch_kernel<8, true, true, float>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tm, tm, parts, gate, st)
            : launch_kernel<8, true, false, float>(plan, chunks, n, kx, X, ldx, ky, Y, ldy, rpc, tm, tm, parts, gate,
                                                   st);
  if (e != cudaSuccess) return e;
  return launch_fx_reduce(kx, ky, sym, chunks, parts, G_hi, G_lo, ldg, gate, st);
}

}  // namespace eo
