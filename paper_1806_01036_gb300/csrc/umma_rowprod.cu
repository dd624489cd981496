// umma_rowprod.cu — compensated row products on the tcgen05 tensor cores:
//   projection  Y~ = Y - V C   (arXiv:1806.01036, Sec. 4.2, phase I, with
//                               C = V^T Y a double-double kv-by-k matrix);
//   update      Q  = X Z       (the final multiplication of phase II; Z the
//                               double-double R^{-1} or M^{-1/2}).
// Every output is the exact sum of its products (up to the dropped digit
// pairs), rounded once; the projection subtracts the exact sum from y before
// rounding.
//
// Digits (umma.cuh): a row of the streamed matrix (V or X) is aligned to its
// own largest exponent A_r, a column j of the small matrix (C or Z) to
// B_j = its largest exponent + 1 (room for the low part); both are cut into
// fifteen 7-bit digits.  A tile is 128 rows = the 128 TMEM lanes; the K
// dimension is the kin columns of the row (kin <= 64), the N dimension the
// digit slab t and the output column j (16 columns, padded).  One MMA
// multiplies digit slab s of the tile (M = 128, K = 16) by the slabs
// t = 0 .. 14 - s of the small matrix (N = 16 (15 - s)) and writes at TMEM
// column offset 16 s: column block d of a lane collects the digit diagonal
// d = s + t of its row.  A diagonal sum has at most kin x 15 products of
// magnitude <= 127^2, below 2^24 for kin <= 64, so the FP32 accumulators are
// exact over the whole row: a tile needs no drains, only an epilogue that
// combines its 15 diagonals per output in 128-bit integers,
//   h = sum_d S_d 2^(7 (14 - d)),   sum_i v_i c_ij ~= h 2^(A_r + B_j - 2156),
// and rounds y - h 2^(...) (or h 2^(...)) to FP64 in integer arithmetic.
//
// Pipeline (one CTA per SM, tiles round-robin): the 16 converter warps hold
// a tile's values in registers (8 rows x 4 column groups per warp,
// coalesced along rows), fetched a tile ahead (staged through shared memory
// with cp.async for kin <= 32, loaded into registers after the previous
// tile's digits are stored for kin <= 64), find each row's exponent by
// shuffles, and write the digits in three groups of five slabs into two
// alternating shared-memory buffers; one warp issues the group's MMAs and
// commits them to an mbarrier per buffer; TMEM holds two accumulators, so
// the epilogue of tile i - 1 (tcgen05.ld, exact rounding, stores) runs
// while the tensor cores work on tile i (with two blocks of 16 output
// columns, one accumulator each: see the kernel).  The projection's Y of a tile is
// prefetched into L2 a tile ahead and loaded before its epilogue reads
// TMEM.  Every wait is bounded (the outputs of a CTA whose wait ran out are
// NaN).  Each tile's loads precede its own stores, and no tile is written
// by another CTA, so the update may run in place.
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "fx.cuh"
#include "umma.cuh"

namespace eo {
namespace {

using namespace fx;
using namespace umma;

constexpr int kConvWarps = 16;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kThreads = kConvThreads + 32;  // plus one MMA-issuing warp
constexpr int kRows = 128;                   // rows per tile (MMA M, TMEM lanes)
constexpr int kOut = 16;                     // output columns of the MMA (padded)
// Digit slabs per group (three groups per tile).
template <int W>
constexpr int kGroupSlabs = 5;
template <int W>
constexpr int kGroups = NS / kGroupSlabs<W>;
constexpr int kScaleProd = 2156;             // value of h: h 2^(A_r + B_j - 2156)
constexpr unsigned kAccCols = 256;           // TMEM columns per accumulator (240 used)
constexpr size_t kMinSmem = 120 * 1024;      // keeps one CTA per SM (TMEM: 512 columns)


// With kin <= 32 the digit buffers leave room below the shared-memory floor
// that keeps one CTA per SM: every converter thread then stages its own
// values of the next tile there (one buffer: a tile's values are read before
// the next tile's copies are issued into the same slots) while the current
// tile runs.  kin <= 64 has no room left (and smaller digit groups, to make
// some, cost more than the staging saves): there the next tile's values are
// loaded into registers once this tile's digits are stored (its values and
// digit words are dead then), so the loads are in flight during the
// previous tile's epilogue.
template <int W>
constexpr bool kStageValues = W <= 8;
#ifndef EO_ROW_NEAR
#define EO_ROW_NEAR(W) ((W) >= 8)
#endif

// Diagonal d of a tile sums (d + 1) kin <= (d + 1) 4 W digit products of
// magnitude <= 127^2.  Diagonals d <= kRoundDiag stay below 2^22 units, so
// their integer value comes out of one FP32 add (the bit pattern of
// 1.5 2^23 + S_d is 0x4B400000 + S_d) instead of a float-to-int conversion.
template <int W>
constexpr int kRoundDiag = (int)(4194303 / (4 * W * 127 * 127)) - 1;
static_assert(kRoundDiag<4> >= 14 && kRoundDiag<8> == 7 && kRoundDiag<16> == 3, "diagonal bounds");
// What those patterns add to chain c (diagonals 5c .. 5c + 4, weights 128^(5c + 4 - d)).
template <int W>
__host__ __device__ constexpr long long chain_offset(int c) {
  long long o = 0;
  for (int d = 5 * c; d < 5 * c + 5; ++d) o = o * 128 + (d <= kRoundDiag<W> ? 0x4B400000ll : 0ll);
  return o;
}
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void st_shared_v4(unsigned addr, unsigned a, unsigned b, unsigned c, unsigned d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_shared_v2(unsigned addr, unsigned a, unsigned b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// Three groups of four TMEM columns (this warp's 32 lanes), loaded and waited for in one step.
__device__ __forceinline__ void tmem_ld3x4(unsigned a0, unsigned a1, unsigned a2, unsigned (&v)[3][4]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%12];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%13];\n"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%14];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]),
        "=r"(v[1][3]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3])
      : "r"(a0), "r"(a1), "r"(a2)
      : "memory");
}

// Digit words of slab S for W values of one row (two values per word, low
// half first), stored at dst (W = 16: two 16-byte chunks 128 bytes apart;
// W = 8: one chunk; W = 4: half a chunk).
// near: every value of the warp had its X's low 32 bits zero (within 20
// binades of its row's exponent), so the digits of slabs 11..14 (bits
// 0..27) are zero and are stored as such without being extracted.
template <int S, int W>
__device__ __forceinline__ void store_slab(unsigned dst, const PairLanes (&P)[W / 2], const unsigned (&sg)[W / 2],
                                           bool near) {
  unsigned w[W / 2];
  if (S >= 11 && near) {
#pragma unroll
    for (int m = 0; m < W / 2; ++m) w[m] = 0u;
  } else {
#pragma unroll
    for (int m = 0; m < W / 2; ++m) w[m] = pair_word<S>(P[m], sg[m]);
  }
  if constexpr (W == 16) {
    st_shared_v4(dst, w[0], w[1], w[2], w[3]);
    st_shared_v4(dst + 128u, w[4], w[5], w[6], w[7]);
  } else if constexpr (W == 8) {
    st_shared_v4(dst, w[0], w[1], w[2], w[3]);
  } else {
    st_shared_v2(dst, w[0], w[1]);
  }
}

template <int G, int W, int J = 0>
__device__ __forceinline__ void store_group(unsigned dst, unsigned slab_bytes, const PairLanes (&P)[W / 2],
                                            const unsigned (&sg)[W / 2], bool near) {
  if constexpr (J < kGroupSlabs<W>) {
    store_slab<G * kGroupSlabs<W> + J, W>(dst + J * slab_bytes, P, sg, near);
    store_group<G, W, J + 1>(dst, slab_bytes, P, sg, near);
  }
}

// store_group for a group index known at run time
template <int W>
__device__ __forceinline__ void store_group_rt(int g, unsigned dst, unsigned slab_bytes, const PairLanes (&P)[W / 2],
                                               const unsigned (&sg)[W / 2], bool near) {
  switch (g) {
    case 0: store_group<0, W>(dst, slab_bytes, P, sg, near); break;
    case 1: store_group<1, W>(dst, slab_bytes, P, sg, near); break;
    case 2: store_group<2, W>(dst, slab_bytes, P, sg, near); break;
    case 3: if constexpr (kGroups<W> > 3) store_group<3, W>(dst, slab_bytes, P, sg, near); break;
    default: if constexpr (kGroups<W> > 4) store_group<4, W>(dst, slab_bytes, P, sg, near); break;
  }
}

// x 2^(1127 - A) as a signed 128-bit integer, truncated toward zero.
__device__ __forceinline__ i128 fixed_trunc(double x, int A) {
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
  return (hi >> 31) ? -(i128)X : (i128)X;
}

// The general exact rounding (rare inputs the branch-free forms leave),
// kept out of line so that the kernels' code stays small.
// Outputs of a thread rounded side by side (measured on 4e6 rows: one at a
// time for kin = 64, where two already cost spills at 96 registers; two
// for the narrower products).
template <int W>
constexpr int kRoundPair = W >= 16 ? 1 : 2;
__device__ __noinline__ double round_general(int update, double y, i128 h, int S) {
  return update ? w_to_double(h, S) : sub_round(y, h, S);
}

// KP = 4 W: the K dimension (kin padded to 16, 32 or 64; padded columns
// are converted as zeros).  KO: blocks of 16 output columns (1, or 2 for
// kout up to 32 with kin <= 32).  With one block, TMEM holds two
// accumulators and the epilogue of tile i - 1 overlaps the MMAs of tile i;
// with two, the 480 columns of the two blocks leave one accumulator each:
// the converters store groups 0 and 1 of tile i, read tile i - 1's
// accumulators, release them (tfree) and then store group 2, and the MMAs of
// tile i wait for that release, so the inputs are converted once for all 32
// outputs.
template <int W, int KO = 1>
__global__ void __launch_bounds__(kThreads, 1)
    umma_rowprod_kernel(int update, int64_t n, int kin, const double* A, int64_t lda, int kout,
                        const double* __restrict__ Bh, const double* __restrict__ Bl, int ldb, int tri,
                        const double* Yin, int64_t ldyin, double* Out, int64_t ldo, const int* gate) {
  if (gate && *gate == 0) return;
  constexpr int KP = 4 * W;
  constexpr int KC = KP / 16;             // MMAs (K = 16) per slab
  constexpr unsigned SBO = 16u * KP;      // bytes between 8-row groups of an operand
  constexpr unsigned SLAB_A = 16u * SBO;  // one digit slab of the tile (128 rows)
  constexpr unsigned B_BYTES = 32u * SBO; // 16 slabs x 16 columns (one block of outputs)
  constexpr int NOUT = kOut * KO;
  static_assert(KO == 1 || (KO == 2 && W <= 8), "two output blocks only for kin <= 32");

  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* bdig = smem;                                  // the small matrix's digits
  unsigned char* adig = smem + KO * B_BYTES;                   // two group buffers of 5 slabs
  constexpr int GS = kGroupSlabs<W>, NG = kGroups<W>;
  int* Arow = reinterpret_cast<int*>(adig + 2 * GS * SLAB_A);  // [2][128] row exponents
  int* Rbad = Arow + 2 * kRows;                                // [2][128] non-finite rows
  int* Bexp = Rbad + 2 * kRows;                                // [NOUT] column exponents
  int* Bbad = Bexp + NOUT;                                     // [NOUT] non-finite columns
  double* stg = reinterpret_cast<double*>(Bbad + NOUT);        // [W][512] staged values (kin <= 32)
  __shared__ __align__(8) unsigned long long full_bar[2], ready_bar[2], tfree_bar;
  __shared__ unsigned tmem_base;
  __shared__ int bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (n + kRows - 1) / kRows;

  // ---- set-up: TMEM (two accumulators), barriers, the small matrix's digits
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base), 2 * kAccCols);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&full_bar[b]), 1);
      mbar_init(smem_u32(&ready_bar[b]), kConvThreads);
    }
    mbar_init(smem_u32(&tfree_bar), kConvThreads);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bad = 0;
  }
  if (tid < NOUT) {
    const int j = tid;
    int e = 0, nf = 0;
    if (j < kout) {
      for (int i = 0; i < kin; ++i) {
        if (tri && i > j) continue;
        const int ae = align_exp(Bh[(size_t)j * ldb + i]);
        e = max(e, ae);
        if (ae == 2047 || (Bl && align_exp(Bl[(size_t)j * ldb + i]) == 2047)) nf = 1;
      }
    }
    Bexp[j] = e + 1;  // one binade of headroom: |h + l| may round up past the largest h
    Bbad[j] = nf;
  }
  __syncthreads();
  for (int e = tid; e < NOUT * KP; e += kThreads) {  // block j / 16: B row R = t * 16 + j % 16 (slab t), K index i
    const int j = e / KP, i = e % KP;
    i128 x = 0;
    if (j < kout && i < kin && !(tri && i > j) && !Bbad[j]) {
      const double h = Bh[(size_t)j * ldb + i], l = Bl ? Bl[(size_t)j * ldb + i] : 0.0;
      x = fixed_trunc(h, Bexp[j]) + fixed_trunc(l, Bexp[j]);
    }
    const unsigned sign = x < 0 ? 0x8000u : 0u;
    const u128 U = x < 0 ? (u128)(-x) : (u128)x;  // < 2^104
    for (int t = 0; t < 16; ++t) {
      const unsigned dgt = t < NS ? ((unsigned)(U >> (98 - 7 * t)) & 127u) | sign : 0u;
      const int R = t * kOut + j % kOut;
      *reinterpret_cast<unsigned short*>(bdig + (j / kOut) * B_BYTES + (R >> 3) * SBO + (i >> 3) * 128 +
                                         (R & 7) * 16 + (i & 7) * 2) =
          (unsigned short)dgt;
    }
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned taddr = tmem_base;
  const unsigned fb0 = smem_u32(&full_bar[0]), rb0 = smem_u32(&ready_bar[0]), tfb = smem_u32(&tfree_bar);
  const unsigned adig_s = smem_u32(adig), bdig_s = smem_u32(bdig);

  if (warp == kConvWarps) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int G = 0;  // groups issued
      bool ok = true;
      for (int64_t T = blockIdx.x, i = 0; T < ntiles && ok; T += gridDim.x, ++i) {
        const unsigned acc = taddr + (KO > 1 ? 0u : (unsigned)(i & 1) * kAccCols);
        if constexpr (KO > 1) {
          if (i > 0) {  // tile i - 1's accumulators read by its epilogue
            if (!mbar_wait(tfb, (unsigned)(i - 1) & 1u, &bad)) break;
            tc_fence_after();
          }
        }
#pragma unroll 1
        for (int g = 0; g < NG; ++g, ++G) {
          const int b = G & 1;
          if (!mbar_wait(rb0 + 8u * b, (unsigned)(G >> 1) & 1u, &bad)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const unsigned abuf = adig_s + (unsigned)b * GS * SLAB_A;
          for (int sg = 0; sg < GS; ++sg) {
            const int s = g * GS + sg;
            const unsigned idesc = idesc_f16(kRows, kOut * (NS - s));
#pragma unroll
            for (int h = 0; h < KO; ++h)
#pragma unroll
              for (int kc = 0; kc < KC; ++kc) {
                const unsigned long long ad = sdesc(abuf + (unsigned)sg * SLAB_A + (unsigned)kc * 256u, 128u, SBO);
                const unsigned long long bd = sdesc(bdig_s + (unsigned)h * B_BYTES + (unsigned)kc * 256u, 128u, SBO);
                mma_f16(acc + (unsigned)h * kAccCols + (unsigned)(kOut * s), ad, bd, idesc,
                        (s == 0 && kc == 0) ? 0u : 1u);
              }
          }
          mma_commit(fb0 + 8u * b);
        }
      }
      // the last committed MMAs finish before TMEM and shared memory are released
      if (G > 0) mbar_wait_final(fb0 + 8u * ((G - 1) & 1), (unsigned)((G - 1) >> 1) & 1u, &bad);
    }
    __syncwarp();
  } else {
    // ---------------- converters: loads, row exponents, digits; epilogues
    const int rlo = lane & 7, cg = lane >> 3;
    const int r = warp * 8 + rlo;  // tile row of this thread's values
    const int c0 = cg * W;         // first of its W columns
    // digit offset of (row r, column c0) within a slab
    const unsigned dofs = (unsigned)(r >> 3) * SBO + (unsigned)(c0 >> 3) * 128u + (unsigned)(r & 7) * 16u +
                          (unsigned)(c0 & 7) * 2u;
    // epilogue mapping: TMEM lane quarter warp % 4, outputs 4 (warp / 4) .. + 3
    const int eq = warp & 3, ep = warp >> 2;
    const int L = eq * 32 + lane;
    const unsigned tq = taddr + ((unsigned)(eq * 32) << 16) + (unsigned)(ep * 4);

    // value k of this thread for tile T into its staging slots (zeros beyond the matrix)
    const unsigned stg_s = smem_u32(stg);
    auto prefetch = [&](int64_t T) {
      const int64_t gr = T * kRows + r;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const int col = c0 + k;
        const bool ok = T < ntiles && gr < n && col < kin;
        cp_async8z(stg_s + (unsigned)((k * kConvThreads + tid) * 8), ok ? A + (size_t)col * lda + gr : A,
                   ok ? 8u : 0u);
      }
      cp_async_commit_group();
    };
    if constexpr (kStageValues<W>) prefetch(blockIdx.x);

    // outputs 16 ob + 4 ep .. + 3 (output block ob) of tile T (the index is
    // written out at each use: a variable for it costs a register at the
    // 96-register limit of the kin = 64 kernel, and it spills)
    auto epilogue_block = [&](int64_t T, int64_t i, int ob) {
      if (ob * kOut + ep * 4 >= kout) return;  // all four outputs of this warp are padding (warp-uniform)
      const unsigned tb = tq + (unsigned)(KO > 1 ? ob : (int)(i & 1)) * kAccCols;
      double yv[4];
      {
        const int64_t grow = T * kRows + L;
#pragma unroll
        for (int y = 0; y < 4; ++y)
          yv[y] = (!update && ob * kOut + ep * 4 + y < kout && grow < n)
                      ? Yin[(size_t)(ob * kOut + ep * 4 + y) * ldyin + grow]
                      : 0.0;
      }
      i128 h[4];
      if constexpr (kRoundDiag<W> >= NS - 1) {
        // every diagonal below 2^22 units: q_m = S_2m 128 + S_2m+1 in 32 bits
        // (m = 0..6; the FP32 bit patterns carry the offset 0x4B400000, taken
        // off once per pair), r = q_a 2^14 + q_b in 64 bits, and
        // h = r_0 2^77 + r_1 2^49 + r_2 2^21 + r_3 with r_3 = q_6 2^7 + S_14.
        unsigned qa[4];
        long long ra[4];
#pragma unroll
        for (int d0 = 0; d0 < NS; d0 += 3) {
          unsigned v[3][4];
          tmem_ld3x4(tb + (unsigned)(d0 * kOut), tb + (unsigned)((d0 + 1) * kOut), tb + (unsigned)((d0 + 2) * kOut), v);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const int d = d0 + u, m = d / 2;
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              const unsigned b = __float_as_uint(fmaf(__uint_as_float(v[u][y]), 0x1p48f, 0x1.8p23f));
              if (d == NS - 1) {
                h[y] += (i128)(ra[y] + (long long)(int)(b - 0x4B400000u));
              } else if (d % 2 == 0) {
                qa[y] = b;
              } else {
                const long long q = (long long)(int)((qa[y] << 7) + b - 129u * 0x4B400000u);
                if (m % 2 == 0) ra[y] = q << (m == 6 ? 7 : 14);
                else if (m == 1) h[y] = (i128)(ra[y] + q) << 77;
                else h[y] += (i128)(ra[y] + q) << (m == 3 ? 49 : 21);
              }
            }
          }
        }
      } else {
        // h = p0 2^70 + p1 2^35 + p2 with p_c = sum over the five diagonals
        // d = 5c .. 5c + 4 of S_d 2^(7 (5c + 4 - d)) (|p_c| < 2^53: 64-bit chains)
        long long p[3][4];
#pragma unroll
        for (int d0 = 0; d0 < NS; d0 += 3) {
          unsigned v[3][4];
          tmem_ld3x4(tb + (unsigned)(d0 * kOut), tb + (unsigned)((d0 + 1) * kOut), tb + (unsigned)((d0 + 2) * kOut), v);
#pragma unroll
          for (int u = 0; u < 3; ++u) {
            const int d = d0 + u, c = d / 5;
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              // S_d = accumulator x 2^48; diagonals below 2^22 units come out of
              // the FP32 add of 1.5 2^23 as its bit pattern 0x4B400000 + S_d
              // (the offsets are taken off the chains below)
              const long long sd = d <= kRoundDiag<W>
                                       ? (long long)__float_as_uint(fmaf(__uint_as_float(v[u][y]), 0x1p48f, 0x1.8p23f))
                                       : (long long)__float2int_rn(__uint_as_float(v[u][y]) * 0x1p48f);
              p[c][y] = (d % 5 == 0) ? sd : p[c][y] * 128 + sd;
            }
          }
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
#pragma unroll
          for (int c = 0; c < 3; ++c) p[c][y] -= chain_offset<W>(c);
          h[y] = ((i128)p[0][y] << 70) + ((i128)p[1][y] << 35) + (i128)p[2][y];
        }
      }
      const int64_t grow = T * kRows + L;
      const int Ar = Arow[(i & 1) * kRows + L];
      const bool rbad = Rbad[(i & 1) * kRows + L] != 0;
      // the four roundings without branches (independent, so they
      // interleave); the rare inputs they leave (not ok) take the general
      // rounding out of line
#pragma unroll
      for (int y0 = 0; y0 < 4; y0 += kRoundPair<W>) {
        double o[kRoundPair<W>];
        bool ok[kRoundPair<W>];
        if (update) {
#pragma unroll
          for (int u = 0; u < kRoundPair<W>; ++u)
            o[u] = w_to_double_fast(h[y0 + u], Ar + Bexp[ob * kOut + ep * 4 + y0 + u] - kScaleProd, ok[u]);
        } else {
#pragma unroll
          for (int u = 0; u < kRoundPair<W>; ++u)
            o[u] = sub_round_fast(yv[y0 + u], h[y0 + u], Ar + Bexp[ob * kOut + ep * 4 + y0 + u] - kScaleProd, ok[u]);
        }
#pragma unroll
        for (int u = 0; u < kRoundPair<W>; ++u) {
          const int y = y0 + u, j = ob * kOut + ep * 4 + y;
          if (j < kout && grow < n) {
            if (!ok[u]) o[u] = round_general(update, yv[y], h[y], Ar + Bexp[j] - kScaleProd);
            if (rbad || Bbad[j] || bad) o[u] = __longlong_as_double(0x7ff8000000000000ll);
            Out[(size_t)j * ldo + grow] = o[u];
          }
        }
      }
    };

    // this thread's W values of row r of tile T (zero beyond the matrix)
    auto load_direct = [&](int64_t T, double (&v)[W]) {
      const int64_t gr = T * kRows + r;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        const int col = c0 + k;
        v[k] = (T < ntiles && gr < n && col < kin) ? A[(size_t)col * lda + gr] : 0.0;
      }
    };
    double vn[W];  // without staging: the values of the tile to come
    if constexpr (!kStageValues<W>) load_direct(blockIdx.x, vn);

    int G = 0;
    int64_t Tprev = -1, iprev = 0;
    for (int64_t T = blockIdx.x, i = 0; T < ntiles; T += gridDim.x, ++i) {
      double v[W];
      if constexpr (kStageValues<W>) {
        asm volatile("cp.async.wait_all;" ::: "memory");  // this tile's copies, issued a tile ago
#pragma unroll
        for (int k = 0; k < W; ++k) v[k] = stg[k * kConvThreads + tid];
        prefetch(T + gridDim.x);  // the next tile's values into the same slots, while this one runs
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) v[k] = vn[k];
      }
      // the row's exponent: max of the |x| high words over the four threads
      // of the row (a row of subnormals and zeros has exponent field 0 and
      // is aligned to 1, the subnormals' own exponent)
      unsigned key = 0, low = 0xffffffffu;  // largest and smallest |x| high word
#pragma unroll
      for (int k = 0; k < W; ++k) {
        key = max(key, abs_hi(v[k]));
        low = min(low, abs_hi(v[k]));
      }
      key = max(key, __shfl_xor_sync(0xffffffffu, key, 8));
      key = max(key, __shfl_xor_sync(0xffffffffu, key, 16));
      const int e = (int)(key >> 20);
      const int Ar = max(e, 1);
      if (cg == 0) {
        Arow[(i & 1) * kRows + r] = Ar;
        Rbad[(i & 1) * kRows + r] = e == 2047;
      }
      PairLanes P[W / 2];  // the W values as interleaved pairs
      unsigned sg[W / 2];
      // every value of the warp normal and within 20 binades of its row's
      // exponent (nearly always): the aligned words without selects
      const bool near = EO_ROW_NEAR(W) && __all_sync(0xffffffffu, low >= near_floor(Ar));
#pragma unroll
      for (int m = 0; m < W / 2; ++m) {
        unsigned xa[4], xb[4];
        if (near) {
          xwords_near(v[2 * m], 52 - Ar, xa);
          xwords_near(v[2 * m + 1], 52 - Ar, xb);
        } else {
          xwords(v[2 * m], Ar, xa);
          xwords(v[2 * m + 1], Ar, xb);
        }
        P[m] = pair_lanes(xa, xb);
        sg[m] = ((hi32(v[2 * m]) >> 31) << 15) | (hi32(v[2 * m + 1]) & 0x80000000u);
      }

      // NG groups of GS slabs into the alternating buffers
#pragma unroll
      for (int g = 0; g < NG; ++g, ++G) {
        const int b = G & 1;
        if constexpr (KO > 1) {
          if (g == NG - 1 && Tprev >= 0) {
            // one accumulator per output block: the previous tile's MMAs are
            // done (its last group was waited for before group 1 of this tile
            // was stored), so its epilogue reads them here and releases them
            // to this tile's MMAs
            tc_fence_after();
#pragma unroll 1
            for (int ob = 0; ob < KO; ++ob) epilogue_block(Tprev, iprev, ob);
            tc_fence_before();
            mbar_arrive(tfb);
          }
        }
        if (G >= 2) mbar_wait(fb0 + 8u * b, (unsigned)((G - 2) >> 1) & 1u, &bad);  // MMAs of group G - 2 done
        store_group_rt<W>(g, adig_s + (unsigned)b * GS * SLAB_A + dofs, SLAB_A, P, sg, near);
        fence_proxy_async();
        mbar_arrive(rb0 + 8u * b);
      }
      if constexpr (!kStageValues<W>) load_direct(T + gridDim.x, vn);
      if (!update && tid < 8 * kout) {  // Y of this tile, read by its epilogue a tile from now: into L2
        const int64_t g0 = T * kRows + (tid & 7) * 16;  // 16 rows = one 128-byte line per thread
        if (g0 < n) prefetch_l2(Yin + (size_t)(tid >> 3) * ldyin + g0);
      }
      // the previous tile's MMAs completed (its last group was waited for before
      // this tile's second group was written): its epilogue overlaps this tile's MMAs
      if constexpr (KO == 1) {
        if (Tprev >= 0) {
          tc_fence_after();
          epilogue_block(Tprev, iprev, 0);
          tc_fence_before();
        }
      }
      bar_conv<kConvThreads>();  // row exponents of buffer (i - 1) & 1 are free again
      Tprev = T;
      iprev = i;
    }
    if (Tprev >= 0) {  // the last tile
      mbar_wait(fb0 + 8u * ((G - 1) & 1), (unsigned)((G - 1) >> 1) & 1u, &bad);
      tc_fence_after();
      if constexpr (KO == 1) {
        epilogue_block(Tprev, iprev, 0);
      } else {
#pragma unroll 1
        for (int ob = 0; ob < KO; ++ob) epilogue_block(Tprev, iprev, ob);
      }
      tc_fence_before();
    }
    if constexpr (kStageValues<W>) asm volatile("cp.async.wait_all;" ::: "memory");  // the last (empty) prefetch
  }

  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(taddr, 2 * kAccCols);
  }
}

template <int W, int KO>
size_t smem_bytes() {
  constexpr int KP = 4 * W;
  const size_t sbo = 16u * KP;
  const size_t b = KO * 32 * sbo, a = 2 * kGroupSlabs<W> * 16 * sbo, small = (4 * kRows + 2 * kOut * KO) * sizeof(int);
  const size_t stage = kStageValues<W> ? (size_t)W * kConvThreads * sizeof(double) : 0;
  return std::max(b + a + small + stage, kMinSmem);
}

template <int W, int KO = 1>
cudaError_t launch_w(bool update, int64_t n, int kin, const double* A, int64_t lda, int kout, const double* Bh,
                     const double* Bl, int ldb, bool tri, const double* Yin, int64_t ldyin, double* Out, int64_t ldo,
                     const int* gate, cudaStream_t st, int ctas) {
  const size_t smem = smem_bytes<W, KO>();
  cudaError_t e = set_dyn_smem(umma_rowprod_kernel<W, KO>, smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (n + kRows - 1) / kRows;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, ctas > 0 ? ctas : 152));
  umma_rowprod_kernel<W, KO><<<grid, kThreads, smem, st>>>(update ? 1 : 0, n, kin, A, lda, kout, Bh, Bl, ldb,
                                                                tri ? 1 : 0, Yin, ldyin, Out, ldo, gate);
  return cudaGetLastError();
}

}  // namespace

cudaError_t umma_rowprod_take_wait_record(unsigned* out) { return take_wait_record(out); }

bool umma_rowprod_supported(int kin, int kout) {
  const char* e = getenv("EO_DD_ROW_ENGINE");
  if (e && e[0] == 'i') return false;
  if (kin < 1 || kin > 64 || kout < 1 || kout > 2 * kOut || (kout > kOut && kin > 32)) return false;
  // Small products run faster on the integer limbs: a tile's fixed cost
  // (15 digit slabs, 16 padded outputs) dominates below kin max(kout, 4) =
  // 128 (measured on 4e6 rows: kin = kout = 4 0.38 vs 1.29 ms, kin = 10,
  // kout = 4 0.64 vs 1.30 ms; equal at 16 x 8; kin = 64, kout = 16 7.05 vs
  // 2.35 ms the other way).  EO_DD_ROW_ENGINE=umma keeps the tensor cores.
  if (!(e && e[0] == 'u') && kin * std::max(kout, 4) < 128) return false;
  return true;
}

cudaError_t launch_umma_rowprod(bool update, int64_t n, int kin, const double* A, int64_t lda, int kout,
                                const double* Bh, const double* Bl, int ldb, bool tri, const double* Yin,
                                int64_t ldyin, double* Out, int64_t ldo, const int* gate, cudaStream_t st,
                                int ctas) {
  if (n <= 0) return cudaSuccess;
  if (kout > kOut)  // two blocks of output columns (kin <= 32): the inputs converted once
    return launch_w<8, 2>(update, n, kin, A, lda, kout, Bh, Bl, ldb, tri, Yin, ldyin, Out, ldo, gate, st, ctas);
  if (kin <= 16)
    return launch_w<4>(update, n, kin, A, lda, kout, Bh, Bl, ldb, tri, Yin, ldyin, Out, ldo, gate, st, ctas);
  if (kin <= 32)
    return launch_w<8>(update, n, kin, A, lda, kout, Bh, Bl, ldb, tri, Yin, ldyin, Out, ldo, gate, st, ctas);
  return launch_w<16>(update, n, kin, A, lda, kout, Bh, Bl, ldb, tri, Yin, ldyin, Out, ldo, gate, st, ctas);
}

}  // namespace eo
