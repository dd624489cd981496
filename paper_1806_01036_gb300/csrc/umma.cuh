// umma.cuh — building blocks of the tcgen05 digit kernels (umma_gram.cu,
// umma_rowprod.cu): inline PTX for mbarriers, TMA, tensor-memory allocation,
// loads and stores, shared-memory matrix descriptors and tcgen05.mma, and the
// 7-bit digits of an FP64 value aligned to a group exponent.
//
// Digits: a value x aligned to the exponent A of its group (A >= the biased
// exponent of every member) is the integer X = floor(|x| 2^(1127 - A)) < 2^105
// = sum_{s=0}^{14} D_s 2^(98 - 7s).  The row kernels (umma_rowprod.cu) use
// plain digits D_s in [0, 127], each the FP16 subnormal +-D_s 2^-24 whose bit
// pattern is the digit with the value's sign, so products of two digits are
// exact and FP32 sums of fewer than 2^24 units of 2^-48 are exact.  The Gram
// kernel (umma_gram.cu) uses balanced digits (below), FP16 integers of at
// most 64 in magnitude (128 for the top digit), whose products are smaller
// and let its accumulators run longer between drains.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "fx.cuh"

namespace eo {
namespace umma {

using namespace fx;

constexpr int NS = 15;  // digits per value
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound of every mbarrier wait

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// One bounded wait: the thread sleeps until the phase completes or up to
// kSuspendNs have passed (no busy polling).
constexpr unsigned kSuspendNs = 1000000u;
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "n"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Set to 1 by a bounded wait that ran out; the host reads and clears it
// (eo_device_status).  Every translation unit that includes this file has
// its own copy, read through that unit's take_wait_record.
static __device__ unsigned g_wait_expired = 0u;

// Wait for the phase of the given parity to complete.  Gives up (false) once
// *abort is set or after limit_ns, and then sets *abort so that every other
// wait of the CTA gives up at once; a wait that ran out records it in
// g_wait_expired.
static __device__ __noinline__ bool mbar_wait_slow(unsigned bar, unsigned parity, volatile int* abort,
                                                   unsigned long long limit_ns) {
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    const bool late = gtimer() - t0 > limit_ns;
    if (*abort || late) {
      if (late) atomicExch(&g_wait_expired, 1u);
      *abort = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, volatile int* abort,
                                          unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;  // the common case: no call
  return mbar_wait_slow(bar, parity, abort, limit_ns);
}
// The same, but only the time limit ends it (waits for MMAs already issued).
static __device__ __noinline__ bool mbar_wait_final(unsigned bar, unsigned parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer() - t0 > kWaitNs) {
      atomicExch(&g_wait_expired, 1u);
      *abort = 1;
      return false;
    }
  }
  return true;
}

// Host side: copy this unit's record to *out (synchronous) and clear it.
static inline cudaError_t take_wait_record(unsigned* out) {
  cudaError_t e = cudaMemcpyFromSymbol(out, g_wait_expired, sizeof(unsigned), 0, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  const unsigned zero = 0u;
  return *out ? cudaMemcpyToSymbol(g_wait_expired, &zero, sizeof(unsigned), 0, cudaMemcpyHostToDevice) : e;
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Barrier 1 among the NT threads of the converter warps only.
template <int NT>
__device__ __forceinline__ void bar_conv() {
  asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}
template <int NT>
__device__ __forceinline__ bool bar_conv_or(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "n"(NT)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(unsigned dst, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout;
// lbo = bytes between core matrices adjacent in K, sbo = in M/N.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP16 A and B (K-major), FP32 D.
__host__ __device__ constexpr unsigned idesc_f16(int M, int N) {
  return (1u << 4) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                        unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// Three column groups of NY consecutive TMEM columns (this warp's 32 lanes),
// loaded and waited for in one step.
template <int NY>
__device__ __forceinline__ void tmem_ld3(unsigned a0, unsigned a1, unsigned a2, unsigned (&v)[3][NY]) {
  if constexpr (NY == 4) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%13];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%14];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]),
          "=r"(v[1][3]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3])
        : "r"(a0), "r"(a1), "r"(a2)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%6];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2,%3}, [%7];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[2][0]), "=r"(v[2][1])
        : "r"(a0), "r"(a1), "r"(a2)
        : "memory");
  }
}

// Six groups: three of the accumulators and three of the running sums.
template <int NY>
__device__ __forceinline__ void tmem_ld3x2(unsigned a0, unsigned a1, unsigned a2, unsigned b0, unsigned b1,
                                           unsigned b2, unsigned (&v)[3][NY], unsigned (&w)[3][NY]) {
  if constexpr (NY == 4) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%25];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%26];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%27];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16,%17,%18,%19}, [%28];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%20,%21,%22,%23}, [%29];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]),
          "=r"(v[1][3]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3]), "=r"(w[0][0]), "=r"(w[0][1]),
          "=r"(w[0][2]), "=r"(w[0][3]), "=r"(w[1][0]), "=r"(w[1][1]), "=r"(w[1][2]), "=r"(w[1][3]), "=r"(w[2][0]),
          "=r"(w[2][1]), "=r"(w[2][2]), "=r"(w[2][3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(b0), "r"(b1), "r"(b2)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2,%3}, [%13];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%14];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6,%7}, [%15];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8,%9}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10,%11}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(w[0][0]),
          "=r"(w[0][1]), "=r"(w[1][0]), "=r"(w[1][1]), "=r"(w[2][0]), "=r"(w[2][1])
        : "r"(a0), "r"(a1), "r"(a2), "r"(b0), "r"(b1), "r"(b2)
        : "memory");
  }
}
// The same loads without the wait; tmem_wait_ld_regs completes them (it names
// the destination registers so that no use can move above the wait).
template <int NY>
__device__ __forceinline__ void tmem_ld3x2_nowait(unsigned a0, unsigned a1, unsigned a2, unsigned b0, unsigned b1,
                                                  unsigned b2, unsigned (&v)[3][NY], unsigned (&w)[3][NY]) {
  if constexpr (NY == 4) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%24];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%25];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%26];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%27];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16,%17,%18,%19}, [%28];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%20,%21,%22,%23}, [%29];\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[0][2]), "=r"(v[0][3]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[1][2]),
          "=r"(v[1][3]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(v[2][2]), "=r"(v[2][3]), "=r"(w[0][0]), "=r"(w[0][1]),
          "=r"(w[0][2]), "=r"(w[0][3]), "=r"(w[1][0]), "=r"(w[1][1]), "=r"(w[1][2]), "=r"(w[1][3]), "=r"(w[2][0]),
          "=r"(w[2][1]), "=r"(w[2][2]), "=r"(w[2][3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(b0), "r"(b1), "r"(b2)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2,%3}, [%13];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%14];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6,%7}, [%15];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8,%9}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10,%11}, [%17];\n"
        : "=r"(v[0][0]), "=r"(v[0][1]), "=r"(v[1][0]), "=r"(v[1][1]), "=r"(v[2][0]), "=r"(v[2][1]), "=r"(w[0][0]),
          "=r"(w[0][1]), "=r"(w[1][0]), "=r"(w[1][1]), "=r"(w[2][0]), "=r"(w[2][1])
        : "r"(a0), "r"(a1), "r"(a2), "r"(b0), "r"(b1), "r"(b2)
        : "memory");
  }
}
template <int NY>
__device__ __forceinline__ void tmem_wait_ld_regs(unsigned (&v)[3][NY], unsigned (&w)[3][NY]) {
  if constexpr (NY == 4) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[0][2]), "+r"(v[0][3]), "+r"(v[1][0]), "+r"(v[1][1]),
                   "+r"(v[1][2]), "+r"(v[1][3]), "+r"(v[2][0]), "+r"(v[2][1]), "+r"(v[2][2]), "+r"(v[2][3]),
                   "+r"(w[0][0]), "+r"(w[0][1]), "+r"(w[0][2]), "+r"(w[0][3]), "+r"(w[1][0]), "+r"(w[1][1]),
                   "+r"(w[1][2]), "+r"(w[1][3]), "+r"(w[2][0]), "+r"(w[2][1]), "+r"(w[2][2]), "+r"(w[2][3])
                 :
                 : "memory");
  } else {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0][0]), "+r"(v[0][1]), "+r"(v[1][0]), "+r"(v[1][1]), "+r"(v[2][0]), "+r"(v[2][1]),
                   "+r"(w[0][0]), "+r"(w[0][1]), "+r"(w[1][0]), "+r"(w[1][1]), "+r"(w[2][0]), "+r"(w[2][1])
                 :
                 : "memory");
  }
}
template <int NY>
__device__ __forceinline__ void tmem_st3(unsigned a0, unsigned a1, unsigned a2, const unsigned (&v)[3][NY]) {
  if constexpr (NY == 4) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%3,%4,%5,%6};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%1], {%7,%8,%9,%10};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%2], {%11,%12,%13,%14};\n" ::"r"(a0),
        "r"(a1), "r"(a2), "r"(v[0][0]), "r"(v[0][1]), "r"(v[0][2]), "r"(v[0][3]), "r"(v[1][0]), "r"(v[1][1]),
        "r"(v[1][2]), "r"(v[1][3]), "r"(v[2][0]), "r"(v[2][1]), "r"(v[2][2]), "r"(v[2][3])
        : "memory");
  } else {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%3,%4};\n"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%1], {%5,%6};\n"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%2], {%7,%8};\n" ::"r"(a0),
        "r"(a1), "r"(a2), "r"(v[0][0]), "r"(v[0][1]), "r"(v[1][0]), "r"(v[1][1]), "r"(v[2][0]), "r"(v[2][1])
        : "memory");
  }
}
// Zeros into three column blocks of NY columns (one zero register for all).
template <int NY>
__device__ __forceinline__ void tmem_zero3(unsigned a0, unsigned a1, unsigned a2) {
  const unsigned z = 0u;
  if constexpr (NY == 4) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%3,%3,%3,%3};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%1], {%3,%3,%3,%3};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%2], {%3,%3,%3,%3};\n" ::"r"(a0),
        "r"(a1), "r"(a2), "r"(z)
        : "memory");
  } else {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%3,%3};\n"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%1], {%3,%3};\n"
        "tcgen05.st.sync.aligned.32x32b.x2.b32 [%2], {%3,%3};\n" ::"r"(a0),
        "r"(a1), "r"(a2), "r"(z)
        : "memory");
  }
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// 2-D TMA tile load (box of the tensor map at coordinates (x, y) = (row, column)).
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------ digits
// X = floor(|x| 2^(1127 - A)) < 2^105 as four 32-bit words (w[0] least
// significant); A >= align_exp(x).  X = m 2^t with m the 53-bit significand.
__device__ __forceinline__ void xwords(double x, int A, unsigned (&w)[4]) {
  const unsigned hi = hi32(x), lo = lo32(x);
  const int e = (hi >> 20) & 0x7ff;
  const unsigned mh = (hi & 0xfffffu) | (e ? 0x100000u : 0u);
  const int t = 52 - A + max(e, 1);
  if (t >= 0) {
    const int bo = t & 31;
    const unsigned s0 = lo << bo, s1 = __funnelshift_l(lo, mh, bo), s2 = __funnelshift_l(mh, 0u, bo);
    const bool up = t >= 32;
    w[0] = up ? 0u : s0;
    w[1] = up ? s0 : s1;
    w[2] = up ? s1 : s2;
    w[3] = up ? s2 : 0u;
  } else {  // more than 52 binades below the column's largest value
    const int r = -t;
    const unsigned long long m = ((unsigned long long)mh << 32) | lo;
    const unsigned long long v = r < 64 ? m >> r : 0ull;
    w[0] = (unsigned)v;
    w[1] = (unsigned)(v >> 32);
    w[2] = 0u;
    w[3] = 0u;
  }
}

// X for a normal value within 20 binades of A (its exponent e >= A - 20,
// so t = 52 - A + e is in [32, 52]): the significand shifted by t - 32
// lands in words 1..3 and word 0 is zero.  cA = 52 - A.  The shift amount
// is taken from the low five bits of (hi >> 20) + cA: the sign bit above
// the exponent field adds a multiple of 32, and the funnel shifts use the
// amount modulo 32.
__device__ __forceinline__ void xwords_near(double x, int cA, unsigned (&w)[4]) {
  const unsigned hi = hi32(x), lo = lo32(x);
  const unsigned bo = (hi >> 20) + (unsigned)cA;
  const unsigned mh = (hi & 0xfffffu) | 0x100000u;
  w[0] = 0u;
  w[1] = __funnelshift_l(0u, lo, bo);
  w[2] = __funnelshift_l(lo, mh, bo);
  w[3] = __funnelshift_l(mh, 0u, bo);
}
// Smallest |x| high word that xwords_near accepts for alignment exponent A:
// exponent at least max(A - 20, 1) (zeros and subnormals take xwords).
__device__ __forceinline__ unsigned near_floor(int A) { return (unsigned)max(A - 20, 1) << 20; }
__device__ __forceinline__ unsigned abs_hi(double x) { return hi32(x) & 0x7fffffffu; }

// 8-byte asynchronous copy global -> shared; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async8z(unsigned dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
// 4-byte asynchronous copy global -> shared; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async4z(unsigned dst, const void* src, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// A pair of values (a, b) interleaved in 16-bit lanes: Z[k] holds bits
// 16k .. 16k + 15 of a in its low half and of b in its high half (k = 0..6),
// Z8[k] the same for bits 16k + 8 .. 16k + 23 (k = 0..5).  Every 7-bit digit
// field of both values then lies inside one lane of one word.
struct PairLanes {
  unsigned Z[7], Z8[6];
};
__device__ __forceinline__ PairLanes pair_lanes(const unsigned (&a)[4], const unsigned (&b)[4]) {
  PairLanes p;
#pragma unroll
  for (int k = 0; k < 7; ++k) p.Z[k] = __byte_perm(a[k >> 1], b[k >> 1], (k & 1) ? 0x7632 : 0x5410);
#pragma unroll
  for (int k = 0; k < 6; ++k) p.Z8[k] = __byte_perm(p.Z[k], p.Z[k + 1], 0x6341);
  return p;
}
// Digit word of slab S for the pair: (D_S(a) | sign a) | ((D_S(b) | sign b) << 16),
// both halves FP16 subnormals +-D 2^-24 (signs: bit 15 and bit 31).
template <int S>
__device__ __forceinline__ unsigned pair_word(const PairLanes& p, unsigned signs) {
  constexpr int q = 98 - 7 * S, k = q >> 4, o = q & 15;
  constexpr bool low = o <= 9;
  constexpr int sh = low ? o : o - 8;
  const unsigned z = low ? p.Z[k] : p.Z8[k];
  // the shift as a high-half multiplication (the FMA pipe), then one
  // three-input logic operation (z & 0x007f007f) | signs (the ALU)
  unsigned zs = z, w;
  if constexpr (sh > 0) asm("mul.hi.u32 %0, %1, %2;" : "=r"(zs) : "r"(z), "n"(1u << (32 - sh)));
  asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(w) : "r"(zs), "n"(0x007f007fu), "r"(signs));
  return w;
}
// The 15 digit words of two consecutive rows (low half: row r, high half:
// row r + 1) into their slabs, slab s at dst + s * stride.
template <int S>
__device__ __forceinline__ void store_digits(unsigned char* dst, unsigned stride, const PairLanes& p,
                                             unsigned signs) {
  if constexpr (S < NS) {
    *reinterpret_cast<unsigned*>(dst + S * stride) = pair_word<S>(p, signs);
    store_digits<S + 1>(dst, stride, p, signs);
  }
}

// Balanced digits.  With B = sum_s 64 * 2^(98 - 7s) (64 in every digit
// place), X' = X + B has 7-bit fields f_s in [0, 127] for s >= 1 and a top
// field f_0 = X' >> 98 in [0, 192] (X < 2^105), and
//   X = sum_s (f_s - 64) 2^(98 - 7s),   D_s = f_s - 64,
// so D_s is in [-64, 63] for s >= 1 and in [-64, 128] for s = 0: products
// of two digits are at most 2^12 (2^13 with D_0, 2^14 for D_0^2) instead of
// 127^2 for unsigned 7-bit digits.  On the tensor cores a digit is the FP16
// integer sign(x) D_s: the field is placed in the significand of the FP16
// 1024 (bit pattern 0x6400 | f, the value 1024 + f), and one f16x2 FMA
// forms sign * (1024 + f) - sign * 1088 = sign (f - 64) exactly (integers
// below 2048 are exact in FP16).
constexpr unsigned kBias0 = 0x08102040u, kBias1 = 0x40810204u, kBias2 = 0x04081020u, kBias3 = 0x102u;
__device__ __forceinline__ void add_bias(unsigned (&w)[4]) {
  asm("add.cc.u32 %0, %0, %4;\n\t"
      "addc.cc.u32 %1, %1, %5;\n\t"
      "addc.cc.u32 %2, %2, %6;\n\t"
      "addc.u32 %3, %3, %7;"
      : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3])
      : "n"(kBias0), "n"(kBias1), "n"(kBias2), "n"(kBias3));
}
// add_bias for X with its low word zero (a value within 20 binades of A):
// the low word becomes the bias's own and carries nothing.
__device__ __forceinline__ void add_bias_near(unsigned (&w)[4]) {
  w[0] = kBias0;
  asm("add.cc.u32 %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, %4;\n\t"
      "addc.u32 %2, %2, %5;"
      : "+r"(w[1]), "+r"(w[2]), "+r"(w[3])
      : "n"(kBias1), "n"(kBias2), "n"(kBias3));
}
// The FP16 exponent field of 1024 in both halves, as a register (so that
// the digit's mask and this constant fit one three-input logic operation).
__device__ __forceinline__ unsigned exp1024x2() {
  unsigned r;
  asm volatile("mov.b32 %0, 0x64006400;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned hfma2(unsigned a, unsigned b, unsigned c) {
  unsigned d;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// Signs of a pair (bit 15: value a, bit 31: value b) -> the f16x2 factors
// (+-1, +-1) and addends (-+1088, -+1088) of the digit FMA.
struct PairSign {
  unsigned mul, add, e1024;
};
__device__ __forceinline__ PairSign pair_sign(unsigned signs, unsigned e1024) {
  return PairSign{0x3C003C00u | signs, 0xE440E440u ^ signs, e1024};
}
// Balanced digit word of slab S for the pair (lanes of X'): low half value a,
// high half value b, both FP16 integers sign * D_S.
template <int S>
__device__ __forceinline__ unsigned bal_word(const PairLanes& p, PairSign sg) {
  constexpr int q = 98 - 7 * S, k = q >> 4, o = q & 15;
  constexpr unsigned m = S == 0 ? 0x00ff00ffu : 0x007f007fu;  // the top field has 8 bits
  constexpr bool low = o <= (S == 0 ? 8 : 9);
  constexpr int sh = low ? o : o - 8;
  const unsigned z = low ? p.Z[k] : p.Z8[k];
  // the shift as a high-half multiplication (the FMA pipe), then one
  // three-input logic operation (z & m) | e1024 (the ALU)
  unsigned zs = z, f;
  if constexpr (sh > 0) asm("mul.hi.u32 %0, %1, %2;" : "=r"(zs) : "r"(z), "n"(1u << (32 - sh)));
  asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(f) : "r"(zs), "n"(m), "r"(sg.e1024));
  return hfma2(f, sg.mul, sg.add);
}
template <int S>
__device__ __forceinline__ void store_bal_digits(unsigned char* dst, unsigned stride, const PairLanes& p,
                                                 PairSign sg) {
  if constexpr (S < NS) {
    *reinterpret_cast<unsigned*>(dst + S * stride) = bal_word<S>(p, sg);
    store_bal_digits<S + 1>(dst, stride, p, sg);
  }
}
// The same for a pair whose X have their low 32 bits zero (add_bias_near):
// the fields of slabs 11..14 (bits 0..27) are then the bias's, so those
// digits are zero.
template <int S>
__device__ __forceinline__ void store_bal_digits_near(unsigned char* dst, unsigned stride, const PairLanes& p,
                                                      PairSign sg) {
  if constexpr (S < NS) {
    *reinterpret_cast<unsigned*>(dst + S * stride) = S >= 11 ? 0u : bal_word<S>(p, sg);
    store_bal_digits_near<S + 1>(dst, stride, p, sg);
  }
}

}  // namespace umma
}  // namespace eo
