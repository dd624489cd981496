// fx.cuh — exact fixed-point accumulation of FP64 products on the integer pipe.
//
// The compensated ("DD") mode of arXiv:1806.01036, Sec. 4.2 needs sums of
// FP64 products accurate to about 2^-104 relative.  GB300 runs FP64 at about
// 2 FMA/clk/SM, but 32x32->64-bit integer multiply-adds (IMAD.WIDE) at about
// 64/clk/SM, so the sums are formed here in integer arithmetic, exactly,
// instead of with FP64 error-free transformations:
//
//  * A group of doubles that is summed over (a column of a row panel, a row
//    of V, a column of Z) shares one alignment exponent A = the largest
//    biased exponent in the group.  Each member x becomes the integer
//      X = floor(|x| * 2^(1126 - A)) < 2^104   (x ~= sign(x) * X * 2^(A - 1126)),
//    which is exact for every member within 51 binades of the largest, and
//    is split into four signed 26-bit limbs L_0..L_3 (L_0 most significant).
//    (A is a biased exponent: |x| < 2^(A - 1022), so X < 2^104.)
//  * A product x*y is sum_{a,b} L_a(x) L_b(y) 2^(26(6-a-b)) * 2^(Ax+Ay-2252).
//    The ten limb products with a + b <= 3 are accumulated per diagonal
//    d = a + b into 64-bit integers (each product < 2^52: exact for up to
//    448 rows per accumulator); the dropped pairs contribute less than
//    6 * 2^-104 of max|x| * max|y| per product.
//  * Diagonal accumulators are combined into a 128-bit integer W in units of
//    2^(Ax+Ay-2148) and rounded to FP64, or to a double-double, with
//    round-to-nearest-even done in integer arithmetic.
//
// Integer sums are exact and associative, so every reduction built on this
// is independent of the order of its partial sums.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace eo {
namespace fx {

FX_HD unsigned hi32(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return (unsigned)(b >> 32);
#endif
}
FX_HD unsigned lo32(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return (unsigned)b;
#endif
}
FX_HD double from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
FX_HD int clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

constexpr int kLimbBits = 26;
constexpr long long kLimbMask = (1ll << kLimbBits) - 1;
constexpr int kRowsPerDrain = 384;  // rows a diagonal accumulator may absorb (< 448)
constexpr int kScaleOffset = 2148;  // value = W * 2^(Ax + Ay - 2148)

typedef __int128 i128;
typedef unsigned __int128 u128;

struct Limbs {
  int v[4];
};

// Biased exponent used for alignment: 1..2046 for finite nonzero values (1 for
// subnormals), 0 for zero, 2047 for Inf/NaN.
FX_HD int align_exp(double x) {
  const unsigned hi = hi32(x);
  const unsigned lo = lo32(x);
  const int be = (hi >> 20) & 0x7ff;
  if (be == 0) return ((hi & 0xfffffu) | lo) ? 1 : 0;
  return be;
}

// Limbs of floor(|x| 2^(1126 - A)) with the sign of x; requires A >= align_exp(x).
// X = m 2^t (t = 51 - (A - be) <= 51) is formed as a 128-bit integer and the
// limbs are cut from it with funnel shifts.
FX_HD Limbs to_limbs(double x, int A) {
  const unsigned hi = hi32(x);
  const unsigned lo = lo32(x);
  int be = (hi >> 20) & 0x7ff;
  unsigned mh = hi & 0xfffffu;
  if (be) mh |= 0x100000u; else be = 1;
  const unsigned long long m = ((unsigned long long)mh << 32) | lo;  // < 2^53
  const int t = 51 - (A - be);
  u128 X;
  if (t >= 0) X = (u128)m << t;
  else if (t > -64) X = (u128)(m >> (-t));
  else X = 0;
  const unsigned long long x0 = (unsigned long long)X, x1 = (unsigned long long)(X >> 64);
  Limbs L;
  L.v[3] = (int)(x0 & kLimbMask);
  L.v[2] = (int)((x0 >> 26) & kLimbMask);
  L.v[1] = (int)(((x0 >> 52) | (x1 << 12)) & kLimbMask);
  L.v[0] = (int)((x1 >> 14) & kLimbMask);
  if (hi >> 31) {
#pragma unroll
    for (int a = 0; a < 4; ++a) L.v[a] = -L.v[a];
  }
  return L;
}

// Limbs of a double-double h + l (|l| <= ulp(h)/2) aligned to A > align_exp(h):
// floor(|h + l| 2^(1126 - A)), computed exactly in 128-bit integers.
FX_HD Limbs to_limbs_dd(double h, double l, int A) {
  auto fixed = [A](double x) -> i128 {  // signed, truncated toward zero
    const unsigned hi = hi32(x);
    const unsigned lo = lo32(x);
    int be = (hi >> 20) & 0x7ff;
    unsigned mh = hi & 0xfffffu;
    if (be) mh |= 0x100000u; else be = 1;
    const unsigned long long m = ((unsigned long long)mh << 32) | lo;
    const int t = 51 - (A - be);
    u128 X;
    if (t >= 0) X = (u128)m << t;       // t <= 51 + (be_l - be_h) <= 51
    else if (t > -64) X = (u128)(m >> (-t));
    else X = 0;
    return (hi >> 31) ? -(i128)X : (i128)X;
  };
  i128 X = fixed(h) + fixed(l);
  const bool neg = X < 0;
  u128 U = neg ? (u128)(-X) : (u128)X;
  Limbs L;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int p = 78 - kLimbBits * a;
    int v = (int)((U >> p) & (u128)kLimbMask);
    L.v[a] = neg ? -v : v;
  }
  return L;
}

// acc += a * b with a 32x32 -> 64-bit signed multiply-add (one IMAD.WIDE).
FX_HD void madw(long long& acc, int a, int b) {
#ifdef __CUDA_ARCH__
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
#else
  acc += (long long)a * b;
#endif
}

// acc[d] += sum_{a+b=d} x_a y_b for d = 0..3 (ten IMAD.WIDE).
FX_HD void mac(long long acc[4], const Limbs& x, const Limbs& y) {
  madw(acc[0], x.v[0], y.v[0]);
  madw(acc[1], x.v[0], y.v[1]);
  madw(acc[1], x.v[1], y.v[0]);
  madw(acc[2], x.v[0], y.v[2]);
  madw(acc[2], x.v[1], y.v[1]);
  madw(acc[2], x.v[2], y.v[0]);
  madw(acc[3], x.v[0], y.v[3]);
  madw(acc[3], x.v[1], y.v[2]);
  madw(acc[3], x.v[2], y.v[1]);
  madw(acc[3], x.v[3], y.v[0]);
}

// mac() on limbs held in int4 (x = L0, y = L1, z = L2, w = L3).
FX_HD void mac4(long long acc[4], const int4& x, const int4& y) {
  madw(acc[0], x.x, y.x);
  madw(acc[1], x.x, y.y);
  madw(acc[1], x.y, y.x);
  madw(acc[2], x.x, y.z);
  madw(acc[2], x.y, y.y);
  madw(acc[2], x.z, y.x);
  madw(acc[3], x.x, y.w);
  madw(acc[3], x.y, y.z);
  madw(acc[3], x.z, y.y);
  madw(acc[3], x.w, y.x);
}

// W in units of 2^(Ax+Ay-2148): acc0 2^52 + acc1 2^26 + acc2 + floor(acc3 2^-26).
FX_HD i128 acc_to_w(const long long acc[4]) {
  return ((i128)acc[0] << 52) + ((i128)acc[1] << 26) + (i128)acc[2] + (i128)(acc[3] >> 26);
}

// Divide the accumulated value by 2^sh (floor), as when the alignment
// exponent of one of its factors grows by sh.  The diagonals carry different
// weights, so the value is combined first and redistributed exactly:
// W' = floor(W 2^-sh) = acc0' 2^52 + acc2' with 0 <= acc2' < 2^52.
FX_HD void acc_shift(long long acc[4], int sh) {
  if (sh <= 0) return;
  i128 w = ((i128)acc[0] << 52) + ((i128)acc[1] << 26) + (i128)acc[2] + (i128)(acc[3] >> 26);
  w = sh >= 127 ? (w < 0 ? (i128)-1 : (i128)0) : (w >> sh);
  acc[0] = (long long)(w >> 52);
  acc[1] = 0;
  acc[2] = (long long)(w & (((i128)1 << 52) - 1));
  acc[3] = 0;
}

FX_HD i128 w_shift(i128 w, int sh) {
  if (sh <= 0) return w;
  return sh >= 127 ? (i128)0 : (w >> sh);
}

FX_HD int clz128(u128 u) {
  const unsigned long long h = (unsigned long long)(u >> 64);
  return h ? clz64(h) : 64 + clz64((unsigned long long)u);
}

// Double with magnitude m * 2^e2 (2^52 <= m < 2^53, or m == 0) and the given sign.
FX_HD double make_double(bool neg, unsigned long long m, int e2) {
  if (m == 0) return neg ? -0.0 : 0.0;
  const int be = e2 + 52 + 1023;
  if (be >= 1 && be <= 2046) {
    const unsigned long long bits =
        ((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1));
    return from_bits(bits);
  }
  if (be > 2046) return from_bits(((unsigned long long)neg << 63) | 0x7ff0000000000000ull);
  const double v = ldexp((double)m, e2);  // subnormal range: rare
  return neg ? -v : v;
}

// Round |u| * 2^S to 53 bits (nearest, ties to even).  Returns the rounded
// mantissa m (2^52 <= m < 2^53) and its exponent e2 (value = m * 2^e2), and the
// rounded value as an integer in units of 2^S when it fits (for remainders).
struct Rounded {
  unsigned long long m;
  int e2;
  u128 as_units;  // m * 2^(e2 - S), exact
  bool fits;
};

FX_HD Rounded round53(u128 u, int S) {
  Rounded r;
  const int p = 127 - clz128(u);
  if (p <= 52) {
    r.m = (unsigned long long)u << (52 - p);
    r.e2 = S + p - 52;
    r.as_units = u;
    r.fits = true;
    return r;
  }
  int sh = p - 52;
  unsigned long long m = (unsigned long long)(u >> sh);
  const u128 rem = u & (((u128)1 << sh) - 1);
  const u128 half = (u128)1 << (sh - 1);
  if (rem > half || (rem == half && (m & 1))) ++m;
  u128 units = (u128)m << sh;  // m may be 2^53 here; the shift keeps it exact
  r.fits = sh + 53 < 127;
  if (m >> 53) {
    m >>= 1;
    ++sh;
  }
  r.m = m;
  r.e2 = S + sh;
  r.as_units = units;
  return r;
}

// Nearest double to w * 2^S (ties to even).  The top 64 bits of |w| and a
// sticky bit for the rest decide the rounding; results outside the normal
// range take the general path.
FX_HD double w_to_double(i128 w, int S) {
  if (w == 0) return 0.0;
  const bool neg = w < 0;
  const u128 u = neg ? (u128)(-w) : (u128)w;
  const unsigned long long uh = (unsigned long long)(u >> 64), ul = (unsigned long long)u;
  int lz;
  unsigned long long t;
  bool sticky;
  if (uh) {
    lz = clz64(uh);
    t = lz ? (uh << lz) | (ul >> (64 - lz)) : uh;
    sticky = (ul << lz) != 0;
  } else {
    lz = 64 + clz64(ul);
    t = ul << (lz - 64);
    sticky = false;
  }
  // t holds bits p .. p - 63 of u, p = 127 - lz its top bit: m = bits p .. p - 52
  unsigned long long m = t >> 11;
  const unsigned long long rb = t & 0x7ffull;
  if (rb > 0x400ull || (rb == 0x400ull && (sticky || (m & 1ull)))) ++m;
  int e2 = S + (127 - lz) - 52;
  if (m >> 53) {
    m >>= 1;
    ++e2;
  }
  const int be = e2 + 52 + 1023;
  if (be < 1 || be > 2046) {
    const Rounded r = round53(u, S);
    return make_double(neg, r.m, r.e2);
  }
  return from_bits(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1)));
}

// Double-double (hi, lo) nearest to w * 2^S: hi = RN(w 2^S), lo = RN(w 2^S - hi).
FX_HD void w_to_dd(i128 w, int S, double& hi, double& lo) {
  if (w == 0) {
    hi = 0.0;
    lo = 0.0;
    return;
  }
  const bool neg = w < 0;
  const u128 u = neg ? (u128)(-w) : (u128)w;
  const Rounded r = round53(u, S);
  hi = make_double(neg, r.m, r.e2);
  const i128 rem = (i128)u - (i128)r.as_units;  // |rem| <= half an ulp of hi, exact
  lo = w_to_double(neg ? -rem : rem, S);
}

// y - w 2^S, rounded to nearest.
FX_HD double sub_round(double y, i128 w, int S) {
  if (w == 0) return y;
  const unsigned hi = hi32(y);
  const unsigned lo = lo32(y);
  int be = (hi >> 20) & 0x7ff;
  unsigned mh = hi & 0xfffffu;
  if (be) mh |= 0x100000u; else be = 1;
  const unsigned long long m = ((unsigned long long)mh << 32) | lo;
  if (m == 0) return -w_to_double(w, S);
  const int ey = be - 1075;  // y = +-m 2^ey
  int d = ey - S;
  int T = S;
  i128 ym;
  if (d > 72) {  // y dominates: coarsen the grid to 2^(ey - 72)
    const int sh = d - 72;
    w = w_shift(w, sh);
    T = S + sh;
    ym = (i128)m << 72;
  } else if (d >= 0) {
    ym = (i128)m << d;
  } else {
    // y has bits below the product's grid: move w onto y's grid when it fits,
    // otherwise (|w| too large to shift) drop y's bits below 2^S
    const u128 aw = w < 0 ? (u128)(-w) : (u128)w;
    if (clz128(aw) > 1 - d) {
      w <<= -d;
      T = S + d;
      ym = (i128)m;
    } else {
      ym = -d >= 64 ? (i128)0 : (i128)(m >> (-d));
    }
  }
  if (hi >> 31) ym = -ym;
  return w_to_double(ym - w, T);
}

// Branch-free forms of w_to_double and sub_round for the common case, so
// that a thread can interleave the roundings of several outputs: the same
// bits as those functions whenever ok is set; ok is cleared when the
// result is not a normal double, and (sub_round) when y is not a normal
// double or has bits below the grid 2^S, and the caller then takes the
// general function.
FX_HD double w_to_double_fast(i128 w, int S, bool& ok) {
  const bool neg = w < 0;
  const u128 u = neg ? (u128)(-w) : (u128)w;
  const unsigned long long uh = (unsigned long long)(u >> 64), ul = (unsigned long long)u;
  const int lz = uh ? clz64(uh) : 64 + clz64(ul);
  const u128 v = u << (lz & 127);  // top bit at 127 (u == 0: result replaced below)
  const unsigned long long t = (unsigned long long)(v >> 64);
  const bool sticky = (unsigned long long)v != 0ull;
  unsigned long long m = t >> 11;
  const unsigned long long rb = t & 0x7ffull;
  m += (unsigned long long)(rb > 0x400ull || (rb == 0x400ull && (sticky || (m & 1ull))));
  const int carry = (int)(m >> 53);
  m >>= carry;
  const int be = S + 1150 - lz + carry;  // e2 + 52 + 1023 with e2 = S + (127 - lz) - 52 + carry
  ok = u == 0 || (be >= 1 && be <= 2046);
  const unsigned long long bits =
      ((unsigned long long)neg << 63) | ((unsigned long long)(be & 0x7ff) << 52) | (m & ((1ull << 52) - 1));
  return u == 0 ? 0.0 : from_bits(bits);
}

FX_HD double sub_round_fast(double y, i128 w, int S, bool& ok) {
  const unsigned hi = hi32(y), lo = lo32(y);
  const int be = (int)((hi >> 20) & 0x7ffu);
  const unsigned long long m = ((unsigned long long)((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  const int d = be - 1075 - S;  // y = +-m 2^(S + d)
  // y dominating by more than 2^72: the product's grid coarsened to
  // 2^(S + d - 72), w truncated onto it (as sub_round does)
  const int sh = d > 72 ? d - 72 : 0;
  const i128 wc = sh >= 127 ? (i128)0 : (w >> sh);
  const u128 ym = (u128)m << (d < 0 ? 0 : (d > 72 ? 72 : d));
  const i128 r = ((hi >> 31) ? -(i128)ym : (i128)ym) - wc;
  bool okr;
  const double o = w_to_double_fast(r, S + sh, okr);
  ok = okr && be >= 1 && be <= 2046 && d >= 0;
  return o;
}

// 256-bit signed accumulator for sums of 128-bit terms.
struct Acc256 {
  u128 lo;
  i128 hi;
  FX_HD void zero() {
    lo = 0;
    hi = 0;
  }
  FX_HD void add(i128 v) {
    const u128 nl = lo + (u128)v;
    hi += (v < 0 ? (i128)-1 : (i128)0) + (nl < lo ? (i128)1 : (i128)0);
    lo = nl;
  }
  FX_HD void add(const Acc256& o) {
    const u128 nl = lo + o.lo;
    hi += o.hi + (nl < lo ? (i128)1 : (i128)0);
    lo = nl;
  }
  // Reduce to a 128-bit value and an extra scale shift (truncating if needed).
  FX_HD i128 narrow(int& extra) const {
    const i128 top = (i128)lo >> 127;  // sign extension of lo as signed
    if (hi == top && (((i128)lo < 0) == (hi < 0))) {
      extra = 0;
      return (i128)lo;
    }
    // find how many bits the 256-bit value needs and shift right to fit in 126
    const bool neg = hi < 0;
    u128 mh = (u128)hi, ml = lo;
    if (neg) {  // magnitude of the two's complement 256-bit value
      ml = ~ml + 1;
      mh = ~mh + (ml == 0 ? 1 : 0);
    }
    const int bits = 128 + (128 - clz128(mh));
    const int sh = bits - 126;
    const u128 mag = (ml >> sh) | (mh << (128 - sh));
    extra = sh;
    return neg ? -(i128)mag : (i128)mag;
  }
};

}  // namespace fx
}  // namespace eo
