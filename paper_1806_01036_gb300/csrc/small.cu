// small.cu — the k-by-k steps of phase II, one CTA each
// (arXiv:1806.01036, Sec. 4.2: the k-by-k work costs little next to the
// n-row passes, in extended precision too).
//
//   chol_small:  M = R^T R (R upper with positive diagonal) by the
//                square-root-free elimination M = L D L^T, carrying
//                L^{-1} along, so R = D^{1/2} L^T and Z = R^{-1} =
//                L^{-T} D^{-1/2}; T <- R T (R of all passes), and the gates
//                of what follows.
//   svqb_small:  M = U Lambda U^T by cyclic Jacobi in the parallel
//                (round-robin) ordering, Z = U Lambda^{+1/2} U^T = M^{-1/2}
//                (Frobenius-nearest to I among Z with Z^T M Z = I, by the
//                Procrustes argument of the same section), T <- T Z.
//                Rotated form (one pass): the Jacobi runs on D M D with
//                D = diag(M)^{-1/2} and Z = D U Lambda^{+1/2}, columns in
//                ascending eigenvalue order, each eigenvector's largest
//                entry positive (the SVQB of Stathopoulos and Wu, 2002).
// In EO_DD the arithmetic is DD throughout (divisions, reciprocals and
// square roots by Newton-Raphson); otherwise it is FP64.
#include <algorithm>

#include "common.cuh"

namespace eo {
namespace {

constexpr int kThreads = 256;
// Jacobi rotates a pair while |a_pq| > eps sqrt(|a_pp a_qq|).  The rotations
// of a sweep leave off-diagonal entries at the rounding level of the
// arithmetic (2^-106 in DD, 2^-53 in FP64), so eps sits a few bits above it:
// at the rounding level itself a sweep would never end without rotations.
constexpr double kJacobiEpsDD = 0x1p-100;
constexpr double kJacobiEpsFP64 = 0x1p-48;

template <int MODE>
struct Ar {
  static __device__ __forceinline__ dd add(dd a, dd b) { return dd{__dadd_rn(a.hi, b.hi), 0.0}; }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd{__dsub_rn(a.hi, b.hi), 0.0}; }
  static __device__ __forceinline__ dd mul(dd a, dd b) { return dd{__dmul_rn(a.hi, b.hi), 0.0}; }
  static __device__ __forceinline__ dd div(dd a, dd b) { return dd{__ddiv_rn(a.hi, b.hi), 0.0}; }
  static __device__ __forceinline__ dd sqrt(dd a) { return dd{__dsqrt_rn(a.hi), 0.0}; }
  static __device__ __forceinline__ dd fma(dd a, dd b, dd c) { return dd{__fma_rn(a.hi, b.hi, c.hi), 0.0}; }
  static __device__ __forceinline__ dd recip(dd a) { return dd{__drcp_rn(a.hi), 0.0}; }
  static __device__ __forceinline__ dd dot2(dd a, dd x, dd b, dd y) { return add(mul(a, x), mul(b, y)); }
  static __device__ __forceinline__ dd rsqrt(dd a) { return dd{__ddiv_rn(1.0, __dsqrt_rn(a.hi)), 0.0}; }
};

template <>
struct Ar<MODE_DD> {
  static __device__ __forceinline__ dd add(dd a, dd b) { return dd_add(a, b); }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_sub(a, b); }
  static __device__ __forceinline__ dd mul(dd a, dd b) { return dd_mul(a, b); }
  static __device__ __forceinline__ dd div(dd a, dd b) { return dd_div(a, b); }
  static __device__ __forceinline__ dd sqrt(dd a) { return dd_sqrt(a); }
  static __device__ __forceinline__ dd fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }
  // 1/a for a > 0: y0 = RN(1/a.hi), whose residual 1 - a.hi y0 is exact in
  // one FMA; with e = 1 - a y0 (|e| <= 2^-52), 1/a = y0 (1 + e + e^2 + ...)
  // and y0 (e + e^2) is the low part (relative error about 2^-105).
  static __device__ __forceinline__ dd recip(dd a) {
    const double y0 = __drcp_rn(a.hi);
    double e = __fma_rn(-a.hi, y0, 1.0);
    e = __fma_rn(-a.lo, y0, e);
    return fast_two_sum(y0, y0 * __fma_rn(e, e, e));
  }
  // a x + b y: the two leading products exactly, their sum exactly, the
  // cross terms by FMAs into the low part, one renormalization.  The error
  // is about 2^-104 (|a x| + |b y|), not relative to the result: enough for
  // a plane rotation, whose rounding errors count against the norm of what
  // it rotates (and it costs about 22 FP64 operations, against 34 for two
  // products and an accurate sum).
  static __device__ __forceinline__ dd dot2(dd a, dd x, dd b, dd y) {
    const dd p = two_prod(a.hi, x.hi), q = two_prod(b.hi, y.hi);
    const dd h = two_sum(p.hi, q.hi);
    double lo = __dadd_rn(p.lo, q.lo);
    lo = __fma_rn(a.hi, x.lo, lo);
    lo = __fma_rn(a.lo, x.hi, lo);
    lo = __fma_rn(b.hi, y.lo, lo);
    lo = __fma_rn(b.lo, y.hi, lo);
    return two_sum(h.hi, __dadd_rn(h.lo, lo));
  }
  // 1/sqrt(a) for a > 0: y0 = RN(1/RN(sqrt(a.hi))); r = 1 - a y0^2 to about
  // 2^-105 (y0^2 and a.hi y0^2 split exactly, 1 - hi exact as hi is near 1);
  // 1/sqrt(a) = y0 (1 - r)^(-1/2) = y0 (1 + r/2 + 3 r^2/8 + ...), |r| < 2^-50.
  static __device__ __forceinline__ dd rsqrt(dd a) {
    const double y0 = __drcp_rn(__dsqrt_rn(a.hi));
    const dd q = two_prod(y0, y0), p = two_prod(a.hi, q.hi);
    double r = __dsub_rn(__dsub_rn(1.0, p.hi), p.lo);
    r = __fma_rn(-a.hi, q.lo, r);
    r = __fma_rn(-a.lo, q.hi, r);
    return fast_two_sum(y0, y0 * __fma_rn(0.375 * r, r, 0.5 * r));
  }
};

__device__ __forceinline__ double dabs(double x) { return x < 0 ? -x : x; }

__global__ void status_init_kernel(DevStatus* s, int k) {
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s->gate[i] = i == 0;
  if (threadIdx.x == 0) {
    s->info = 0;
    s->rank = k;
    s->iters = 0;
    s->sweeps = 0;
  }
}

__device__ void finish_gates(const SmallGates& g, int run_update, int want_next) {
  *g.upd = run_update;
  if (g.next) *g.next = want_next;
}

// ------------------------------------------------------------ Cholesky

template <int MODE>
__device__ __forceinline__ void chol_small_body(int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                                                double* Rh_u, double* Rl_u, int ldr, DevStatus* st, SmallGates g,
                                                int pass, int passes, double thr, int* info_user) {
  using A_ = Ar<MODE>;
  if (*g.run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* A = reinterpret_cast<dd*>(smem_raw);  // A(i,j) = A[j*k+i]; R overwrites the upper triangle
  dd* Z = A + k * k;
  dd* Tb = Z + k * k;  // W = L^{-1}
  __shared__ int flag;
  const int tid = threadIdx.x;
  if (tid == 0) flag = 0;
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    const int a = min(i, j), b = max(i, j);
    dd v = dd{Mh[(size_t)b * ldm + a], Ml ? Ml[(size_t)b * ldm + a] : 0.0};
    if (MODE != MODE_DD) v.lo = 0.0;
    if (!dd_finite(v)) atomicExch(&flag, -1);
    A[t] = v;
  }
  __syncthreads();
  // Square-root-free (L D L^T) elimination on the upper triangle: at step j
  // the pivot d_j = A(j,j) and the row A(j, j+1..) are those of the
  // standard algorithm before scaling, the Schur complement takes
  // A(a,b) -= A(j,a) A(j,b) / d_j, and W = L^{-1} (L(l,j) = A(j,l) / d_j)
  // takes W(l,:) -= L(l,j) W(j,:).  The products do not depend on the pivot,
  // so they run while one thread forms 1/d_j: the dependent chain of a step
  // is one reciprocal and one multiply-subtract.  Afterwards
  // R = D^{1/2} L^T and Z = R^{-1} = L^{-T} D^{-1/2} (W: Tb, W(l,c) = Tb[c k + l];
  // the products: Z, as scratch).
  __shared__ dd piv_inv;
  for (int t = tid; t < k * k; t += kThreads) Tb[t] = dd{(t % k) == (t / k) ? 1.0 : 0.0, 0.0};
  __syncthreads();
  if (flag == 0) {
    for (int j = 0; j < k; ++j) {
      const int m = k - j - 1, np = m * (m + 1) / 2, nq = m * (j + 1);
      if (tid == kThreads - 1) {
        const dd d = A[j * k + j];
        if (!(d.hi > 0.0)) flag = j + 1;
        else piv_inv = A_::recip(d);
      }
      for (int t = tid; t < np + nq; t += kThreads) {
        if (t < np) {  // (a, b) = j + 1 + (u, v), u <= v, t = v (v + 1) / 2 + u
          int v = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
          if ((v + 1) * (v + 2) / 2 <= t) ++v;
          if (v * (v + 1) / 2 > t) --v;
          const int a = j + 1 + t - v * (v + 1) / 2, b = j + 1 + v;
          Z[t] = A_::mul(A[a * k + j], A[b * k + j]);
        } else {  // W row l = j + 1 + q % m, column c = q / m <= j
          const int q = t - np, l = j + 1 + q % m, c = q / m;
          Z[t] = A_::mul(A[l * k + j], Tb[c * k + j]);
        }
      }
      __syncthreads();
      if (flag) break;
      const dd w = piv_inv;
      for (int t = tid; t < np + nq; t += kThreads) {
        if (t < np) {
          int v = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
          if ((v + 1) * (v + 2) / 2 <= t) ++v;
          if (v * (v + 1) / 2 > t) --v;
          const int a = j + 1 + t - v * (v + 1) / 2, b = j + 1 + v;
          A[b * k + a] = A_::sub(A[b * k + a], A_::mul(Z[t], w));
        } else {
          const int q = t - np, l = j + 1 + q % m, c = q / m;
          Tb[c * k + l] = A_::sub(Tb[c * k + l], A_::mul(Z[t], w));
        }
      }
      __syncthreads();
    }
  }
  if (flag != 0) {
    if (tid == 0) {
      st->info = flag;
      finish_gates(g, 0, 0);
      if (info_user) *info_user = flag;
    }
    return;
  }
  // s_j = sqrt(d_j) and 1 / s_j (kept in the diagonal of Z for the moment)
  for (int j = tid; j < k; j += kThreads) {
    const dd r = A_::sqrt(A[j * k + j]);
    A[j * k + j] = r;
    Z[j * k + j] = A_::recip(r);
  }
  __syncthreads();
  // R(j, l) = A(j, l) / s_j (l > j); Z(i, j) = W(j, i) / s_j (i < j)
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    if (i < j) {
      A[j * k + i] = A_::mul(A[j * k + i], Z[i * k + i]);
      Z[t] = A_::mul(Tb[i * k + j], Z[j * k + j]);
    } else if (i > j) {
      Z[t] = dd{0.0, 0.0};
    }
  }
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    ws->Zh[j * KMAX + i] = Z[t].hi;
    ws->Zl[j * KMAX + i] = Z[t].lo;
  }
  __syncthreads();
  // T <- R T (upper triangular product); T = R on the first pass.
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    dd v = dd{0.0, 0.0};
    if (i <= j) {
      if (pass == 0) {
        v = A[j * k + i];
      } else {
        for (int l = i; l <= j; ++l)
          v = A_::fma(A[l * k + i], dd{ws->Th[j * KMAX + l], ws->Tl[j * KMAX + l]}, v);
      }
    }
    Z[t] = v;  // Z's copy is already in global memory
  }
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    ws->Th[j * KMAX + i] = Z[t].hi;
    ws->Tl[j * KMAX + i] = Z[t].lo;
    if (Rh_u) Rh_u[(size_t)j * ldr + i] = Z[t].hi;
    if (Rl_u) Rl_u[(size_t)j * ldr + i] = Z[t].lo;
  }
  if (tid == 0) {
    double dmax = 0.0, dmin = 1e308;
    for (int i = 0; i < k; ++i) {
      dmax = fmax(dmax, A[i * k + i].hi);
      dmin = fmin(dmin, A[i * k + i].hi);
    }
    int next = 0;
    if (pass == 0) next = passes == 2 ? 1 : (passes == 0 ? (dmax > thr * dmin) : 0);
    finish_gates(g, 1, next);
    if (info_user) *info_user = st->info;
  }
}

// ----------------------------------------- pivoted, partial Cholesky

// One CTA.  A, R and the inverse of R11 in shared memory (double-double in
// EO_DD, FP64 otherwise); see launch_pivchol_small.
template <int MODE>
__global__ void __launch_bounds__(kThreads)
    pivchol_small_kernel(int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws, double* Rh_u,
                         double* Rl_u, int ldr, double tol, DevStatus* st, SmallGates g, int pass, int passes,
                         double thr, int* info_user, int* rank_user, int* perm_user) {
  using A_ = Ar<MODE>;
  if (*g.run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* A = reinterpret_cast<dd*>(smem_raw);  // A(i,j) = A[j*k+i], the trailing matrix
  dd* R = A + k * k;                        // R(i,j) = R[j*k+i]
  dd* Zs = R + k * k;                       // R11^{-1}
  __shared__ int flag, piv, stop, perm_s[KMAX];
  __shared__ dd rinv;
  const int tid = threadIdx.x;
  const int lim = pass == 0 ? k : st->rank;  // columns that may be factored
  if (tid == 0) {
    flag = 0;
    stop = lim;
  }
  for (int i = tid; i < k; i += kThreads) perm_s[i] = pass == 0 ? i : st->perm[i];
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    const int a = min(i, j), b = max(i, j);
    dd v = dd{Mh[(size_t)b * ldm + a], Ml ? Ml[(size_t)b * ldm + a] : 0.0};
    if (MODE != MODE_DD) v.lo = 0.0;
    if (!dd_finite(v)) atomicExch(&flag, -1);
    A[t] = v;
    R[t] = dd{0.0, 0.0};
    Zs[t] = dd{0.0, 0.0};
  }
  __syncthreads();
  double dmax = 0.0;
  for (int i = 0; i < k; ++i) dmax = fmax(dmax, A[i * k + i].hi);
  const double cut = tol * dmax;
  int r = 0;
  if (flag == 0) {
    for (int j = 0; j < lim; ++j) {
      if (tid == 0) {
        int p = j;
        if (pass == 0)  // the largest remaining diagonal entry, lowest index on ties
          for (int i = j + 1; i < k; ++i) {
            const dd a = A[i * k + i], b = A[p * k + p];
            if (a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo)) p = i;
          }
        const dd d = A[p * k + p];
        if (pass == 0 ? !(d.hi > 0.0 && d.hi > cut) : !(d.hi > 0.0)) {
          stop = j;
          if (pass != 0) flag = j + 1;  // the second pass breaks down
        } else {
          piv = p;
        }
      }
      __syncthreads();
      if (stop == j) break;
      const int p = piv;
      if (p != j) {  // symmetric swap of rows and columns j and p; the rows of R built so far
        for (int i = tid; i < k; i += kThreads) {
          const dd t = A[j * k + i];
          A[j * k + i] = A[p * k + i];
          A[p * k + i] = t;
        }
        __syncthreads();
        for (int i = tid; i < k; i += kThreads) {
          const dd t = A[i * k + j];
          A[i * k + j] = A[i * k + p];
          A[i * k + p] = t;
          if (i < j) {
            const dd u = R[j * k + i];
            R[j * k + i] = R[p * k + i];
            R[p * k + i] = u;
          }
        }
        if (tid == 0) {
          const int t = perm_s[j];
          perm_s[j] = perm_s[p];
          perm_s[p] = t;
        }
        __syncthreads();
      }
      if (tid == 0) {
        const dd rjj = A_::sqrt(A[j * k + j]);
        R[j * k + j] = rjj;
        rinv = A_::recip(rjj);
      }
      __syncthreads();
      for (int l = j + 1 + tid; l < lim; l += kThreads) R[l * k + j] = A_::mul(A[l * k + j], rinv);
      __syncthreads();
      const int m = lim - j - 1;
      for (int t = tid; t < m * m; t += kThreads) {
        const int a = j + 1 + t % m, b = j + 1 + t / m;
        A[b * k + a] = A_::sub(A[b * k + a], A_::mul(R[a * k + j], R[b * k + j]));
      }
      __syncthreads();
      r = j + 1;
    }
  }
  if (flag != 0) {  // NaN / Inf, or a breakdown of the second pass: X stays as it is
    if (tid == 0) {
      st->info = flag;
      if (flag < 0) st->rank = -1;
      finish_gates(g, 0, 0);
      if (info_user) *info_user = flag;
      if (rank_user) *rank_user = st->rank;
    }
    return;
  }
  // R11^{-1}: column c by one thread, back substitution
  for (int c = tid; c < r; c += kThreads) {
    Zs[c * k + c] = A_::recip(R[c * k + c]);
    for (int i = c - 1; i >= 0; --i) {
      dd s2 = dd{0.0, 0.0};
      for (int l = i + 1; l <= c; ++l) s2 = A_::fma(R[l * k + i], Zs[c * k + l], s2);
      Zs[c * k + i] = A_::mul(dd_neg(s2), Zs[i * k + i]);
    }
  }
  __syncthreads();
  // Z: the pivots' rows of R11^{-1} (pass 0), R2^{-1} itself (pass 1); zero beyond the rank
  for (int t = tid; t < KMAX * k; t += kThreads) {
    const int i = t % KMAX, c = t / KMAX;
    if (i < k) {
      ws->Zh[c * KMAX + i] = 0.0;
      ws->Zl[c * KMAX + i] = 0.0;
    }
  }
  __syncthreads();
  for (int t = tid; t < r * r; t += kThreads) {
    const int i = t % r, c = t / r;
    const int row = pass == 0 ? perm_s[i] : i;
    ws->Zh[c * KMAX + row] = Zs[c * k + i].hi;
    ws->Zl[c * KMAX + row] = Zs[c * k + i].lo;
  }
  // R of the whole: R (pass 0) or R2 R_old (pass 1), rows beyond the rank zero
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    dd v = dd{0.0, 0.0};
    if (i < r) {
      if (pass == 0) {
        v = R[j * k + i];
      } else {
        for (int l = i; l < r; ++l) v = A_::fma(R[l * k + i], dd{ws->Th[j * KMAX + l], ws->Tl[j * KMAX + l]}, v);
      }
    }
    Zs[t] = v;
  }
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    ws->Th[j * KMAX + i] = Zs[t].hi;
    ws->Tl[j * KMAX + i] = Zs[t].lo;
    if (Rh_u) Rh_u[(size_t)j * ldr + i] = Zs[t].hi;
    if (Rl_u) Rl_u[(size_t)j * ldr + i] = Zs[t].lo;
  }
  if (pass == 0)
    for (int i = tid; i < k; i += kThreads) {
      st->perm[i] = perm_s[i];
      if (perm_user) perm_user[i] = perm_s[i];
    }
  if (tid == 0) {
    if (pass == 0) st->rank = r;
    int next = 0;
    if (pass == 0 && r > 0)
      next = passes == 2 ? 1 : (passes == 0 ? (R[0].hi > thr * R[(r - 1) * k + (r - 1)].hi) : 0);
    finish_gates(g, 1, next);
    if (info_user) *info_user = st->info;
    if (rank_user) *rank_user = st->rank;
  }
}

// --------------------------------------------------------------- SVQB

template <int MODE>
__device__ __forceinline__ void svqb_small_body(int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                                                double* Zh_u, double* Zl_u, int ldz, double tol, DevStatus* st,
                                                SmallGates g, int pass, int passes, double thr, double eps,
                                                int* rank_user, bool rotated) {
  using A_ = Ar<MODE>;
  if (*g.run == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* A = reinterpret_cast<dd*>(smem_raw);  // k*k (upper triangle read during the sweeps)
  dd* A2 = A + k * k;                        // k*k: the next A
  dd* U = A2 + k * k;                        // k*k
  dd* cs = U + k * k;                        // 2 * (k/2 + 1): c, s per pair
  dd* dv = cs + 2 * (k / 2 + 1);             // k: D = diag(M)^{-1/2} (rotated form)
  int* pr = reinterpret_cast<int*>(dv + k);  // 2 * (k/2 + 1): p, q per pair
  int* perm = pr + 2 * (k / 2 + 1);          // k: eigenpair of column j (rotated form)
  __shared__ int flag, rot_count;
  const int tid = threadIdx.x;
  const int kk = k + (k & 1);  // even number of players; index k is a dummy
  const int npairs = kk / 2;
  if (tid == 0) flag = 0;
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    const int a = min(i, j), b = max(i, j);
    dd v = dd{Mh[(size_t)b * ldm + a], Ml ? Ml[(size_t)b * ldm + a] : 0.0};
    if (MODE != MODE_DD) v.lo = 0.0;
    if (!dd_finite(v)) atomicExch(&flag, -1);
    A[t] = v;
    U[t] = dd{i == j ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  if (flag != 0) {
    if (tid == 0) {
      st->rank = -1;
      finish_gates(g, 0, 0);
      if (rank_user) *rank_user = -1;
    }
    return;
  }
  if (rotated) {  // the Jacobi runs on D M D (unit diagonal; a zero diagonal gives d_i = 0)
    for (int i = tid; i < k; i += kThreads) {
      const dd m = A[i * k + i];
      dv[i] = m.hi > 0.0 ? A_::div(dd{1.0, 0.0}, A_::sqrt(m)) : dd{0.0, 0.0};
      perm[i] = i;
    }
    __syncthreads();
    for (int t = tid; t < k * k; t += kThreads) A[t] = A_::mul(A_::mul(dv[t % k], A[t]), dv[t / k]);
    __syncthreads();
  }
  // Sweeps of the parallel (round-robin) ordering.  Per step: (1) each pair's
  // rotation: the angle in FP64 from the hi parts (t = tan(phi)), then
  // c = 1 / sqrt(1 + t^2) and s = t c in the mode's arithmetic, so that the
  // rotation is orthogonal to that precision while it zeroes a_pq only to
  // FP64 accuracy (the remainder is left in A and removed by later sweeps);
  // (2) A' = J^T A J by 2x2 blocks of pairs on the upper triangle, into the
  // second buffer, and U <- U J in place.
  auto upper = [&](const dd* B, int r, int c) { return B[max(r, c) * k + min(r, c)]; };
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) rot_count = 0;
    __syncthreads();
    for (int step = 0; step < kk - 1; ++step) {
      // round-robin pairing: player 0 fixed, the others rotate by `step`
      for (int p = tid; p < npairs; p += kThreads) {
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (kk - 1); };
        int a = player(p), b = player(kk - 1 - p);
        int lo = min(a, b), hi = max(a, b);
        dd c = dd{1.0, 0.0}, sn = dd{0.0, 0.0};
        if (hi < k) {
          const dd apq = A[hi * k + lo];
          const dd app = A[lo * k + lo], aqq = A[hi * k + hi];
          const double scale = sqrt(dabs(app.hi) * dabs(aqq.hi));
          if (dabs(apq.hi) > eps * scale && apq.hi != 0.0) {
            const double th = A_::sub(aqq, app).hi / (2.0 * apq.hi);
            const double t = dabs(th) > 1e150 ? 0.5 / th : copysign(1.0 / (dabs(th) + sqrt(fma(th, th, 1.0))), th);
            c = A_::rsqrt(A_::add(dd{1.0, 0.0}, A_::mul(dd{t, 0.0}, dd{t, 0.0})));
            sn = A_::mul(c, dd{t, 0.0});
            atomicAdd(&rot_count, 1);
          }
        }
        cs[2 * p] = c;
        cs[2 * p + 1] = sn;
        pr[2 * p] = lo;
        pr[2 * p + 1] = hi;
      }
      __syncthreads();
      // A2 = J^T A J, block (P, Q) of rows {lo_P, hi_P} and columns {lo_Q, hi_Q}, P <= Q
      for (int t = tid; t < npairs * (npairs + 1) / 2; t += kThreads) {
        int Q = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while ((Q + 1) * (Q + 2) / 2 <= t) ++Q;
        while (Q * (Q + 1) / 2 > t) --Q;
        const int P = t - Q * (Q + 1) / 2;
        const int r0 = pr[2 * P], r1 = pr[2 * P + 1], c0 = pr[2 * Q], c1 = pr[2 * Q + 1];
        const dd cP = cs[2 * P], sP = cs[2 * P + 1], cQ = cs[2 * Q], sQ = cs[2 * Q + 1];
        const bool v1 = r1 < k, w1 = c1 < k;  // r0, c0 < k always (the dummy index is the larger)
        dd b00 = upper(A, r0, c0), b01 = w1 ? upper(A, r0, c1) : dd{0.0, 0.0};
        dd b10 = v1 ? upper(A, r1, c0) : dd{0.0, 0.0}, b11 = v1 && w1 ? upper(A, r1, c1) : dd{0.0, 0.0};
        if (!(sQ.hi == 0.0 && sQ.lo == 0.0)) {  // B J_Q
          const dd mQ = dd_neg(sQ);
          const dd t00 = A_::dot2(b00, cQ, b01, mQ), t01 = A_::dot2(b00, sQ, b01, cQ);
          const dd t10 = A_::dot2(b10, cQ, b11, mQ), t11 = A_::dot2(b10, sQ, b11, cQ);
          b00 = t00; b01 = t01; b10 = t10; b11 = t11;
        }
        if (!(sP.hi == 0.0 && sP.lo == 0.0)) {  // J_P^T (B J_Q)
          const dd mP = dd_neg(sP);
          const dd t00 = A_::dot2(cP, b00, mP, b10), t10 = A_::dot2(sP, b00, cP, b10);
          const dd t01 = A_::dot2(cP, b01, mP, b11), t11 = A_::dot2(sP, b01, cP, b11);
          b00 = t00; b01 = t01; b10 = t10; b11 = t11;
        }
        auto put = [&](int r, int c, dd v) { A2[max(r, c) * k + min(r, c)] = v; };
        put(r0, c0, b00);
        if (w1) put(r0, c1, b01);
        if (P == Q) {
          if (v1) put(r1, c1, b11);  // (r1, c0) is the mirror of (r0, c1)
        } else {
          if (v1) put(r1, c0, b10);
          if (v1 && w1) put(r1, c1, b11);
        }
      }
      // U <- U J, columns lo_Q, hi_Q of row m
      for (int t = tid; t < npairs * k; t += kThreads) {
        const int q = t % npairs, m = t / npairs;
        const int a = pr[2 * q], b = pr[2 * q + 1];
        const dd c = cs[2 * q], sn = cs[2 * q + 1];
        if (b >= k || (sn.hi == 0.0 && sn.lo == 0.0)) continue;
        const dd x = U[a * k + m], y = U[b * k + m];
        U[a * k + m] = A_::dot2(c, x, dd_neg(sn), y);
        U[b * k + m] = A_::dot2(sn, x, c, y);
      }
      __syncthreads();
      dd* sw = A;
      A = A2;
      A2 = sw;
    }
    if (rot_count == 0) {
      if (tid == 0) st->sweeps = sweep + 1;
      break;
    }
    __syncthreads();
    if (sweep == 39 && tid == 0) st->sweeps = 40;
  }
  // the upper triangle holds the result: mirror it (the diagonal is eigenvalues)
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    if (i > j) A[t] = A[i * k + j];
  }
  __syncthreads();
  if (rotated) {
    // Column a of U: its largest-magnitude entry (lowest row on ties) made
    // positive; its place in the ascending order of the eigenvalues (ties by
    // index) gives the column of Z it lands in.  Normalized double-doubles
    // compare exactly as (hi, lo) pairs.
    auto lt = [](dd x, dd y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); };
    auto mag = [](dd x) { return x.hi < 0.0 ? dd_neg(x) : x; };
    for (int a = tid; a < k; a += kThreads) {
      dd* u = U + a * k;
      int mb = 0;
      for (int m = 1; m < k; ++m)
        if (lt(mag(u[mb]), mag(u[m]))) mb = m;
      if (u[mb].hi < 0.0)
        for (int m = 0; m < k; ++m) u[m] = dd_neg(u[m]);
      const dd la = A[a * k + a];
      int pos = 0;
      for (int b = 0; b < k; ++b) {
        const dd lb = A[b * k + b];
        pos += lt(lb, la) || (!lt(la, lb) && b < a);
      }
      perm[pos] = a;  // pos < k; with a NaN eigenvalue two columns may collide, the rest keep the identity
    }
    __syncthreads();
  }
  // w_l = lambda_l^{-1/2} for kept eigenvalues; Z = U diag(w) U^T into A's storage.
  __shared__ double lmax_s, lmin_s;
  __shared__ int rank_s;
  dd* w = cs;  // reuse: k entries needed, cs has 2*(k/2+1) >= k
  if (tid == 0) {
    double lmax = 0.0;
    for (int i = 0; i < k; ++i) lmax = fmax(lmax, A[i * k + i].hi);
    int rank = 0;
    double lmin = lmax;
    for (int i = 0; i < k; ++i) {
      const dd l = A[i * k + i];
      if (lmax > 0.0 && l.hi > tol * lmax) {
        w[i] = A_::div(dd{1.0, 0.0}, A_::sqrt(l));
        ++rank;
        lmin = fmin(lmin, l.hi);
      } else {
        w[i] = dd{0.0, 0.0};
      }
    }
    lmax_s = lmax;
    lmin_s = lmin;
    rank_s = rank;
  }
  __syncthreads();
  if (rotated) {  // Z(:, j) = D u_a w_a with a = perm[j]
    for (int t = tid; t < k * k; t += kThreads) {
      const int i = t % k, a = perm[t / k];
      A[t] = A_::mul(A_::mul(dv[i], U[a * k + i]), w[a]);
    }
    __syncthreads();
  } else {  // one triangle, mirrored, so that Z is exactly symmetric
    for (int t = tid; t < k * k; t += kThreads) {
      const int i = t % k, j = t / k;
      if (i > j) continue;
      dd v = dd{0.0, 0.0};
      for (int l = 0; l < k; ++l) v = A_::fma(A_::mul(U[l * k + i], w[l]), U[l * k + j], v);
      A[t] = v;
    }
    __syncthreads();
    for (int t = tid; t < k * k; t += kThreads) {
      const int i = t % k, j = t / k;
      if (i > j) A[t] = A[i * k + j];
    }
    __syncthreads();
  }
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    ws->Zh[j * KMAX + i] = A[t].hi;
    ws->Zl[j * KMAX + i] = A[t].lo;
  }
  __syncthreads();
  // T <- T Z (full product); T = Z on the first pass.  U's storage is free now.
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    dd v = dd{0.0, 0.0};
    if (pass == 0) {
      v = A[t];
    } else {
      for (int l = 0; l < k; ++l) v = A_::fma(dd{ws->Th[l * KMAX + i], ws->Tl[l * KMAX + i]}, A[j * k + l], v);
    }
    U[t] = v;
  }
  __syncthreads();
  for (int t = tid; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    ws->Th[j * KMAX + i] = U[t].hi;
    ws->Tl[j * KMAX + i] = U[t].lo;
    if (Zh_u) Zh_u[(size_t)j * ldz + i] = U[t].hi;
    if (Zl_u) Zl_u[(size_t)j * ldz + i] = U[t].lo;
  }
  if (tid == 0) {
    st->rank = rank_s;
    int next = 0;
    if (pass == 0) next = passes == 2 ? 1 : (passes == 0 ? (lmax_s > thr * thr * lmin_s) : 0);
    finish_gates(g, 1, next);
    if (rank_user) *rank_user = rank_s;
  }
}

// ----------------------------------------------------- kernel wrappers

template <int MODE>
__global__ void __launch_bounds__(kThreads) chol_small_kernel(int k, const double* Mh, const double* Ml, int ldm,
                                                              SmallWs* ws, double* Rh_u, double* Rl_u, int ldr,
                                                              DevStatus* st, SmallGates g, int pass, int passes,
                                                              double thr, int* info_user) {
  chol_small_body<MODE>(k, Mh, Ml, ldm, ws, Rh_u, Rl_u, ldr, st, g, pass, passes, thr, info_user);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) svqb_small_kernel(int k, const double* Mh, const double* Ml, int ldm,
                                                              SmallWs* ws, double* Zh_u, double* Zl_u, int ldz,
                                                              double tol, DevStatus* st, SmallGates g, int pass,
                                                              int passes, double thr, double eps, int* rank_user,
                                                              bool rotated) {
  svqb_small_body<MODE>(k, Mh, Ml, ldm, ws, Zh_u, Zl_u, ldz, tol, st, g, pass, passes, thr, eps, rank_user, rotated);
}

// One CTA per job: the factorization of pass `pass` of many independent
// blocks, each from its own workspace's Gram matrix and gates.
__device__ __forceinline__ SmallGates job_gates(const SmallJob& j, int pass, int npass) {
  return SmallGates{&j.st->gate[2 * pass], &j.st->gate[2 * pass + 1],
                    pass + 1 < npass ? &j.st->gate[2 * pass + 2] : nullptr};
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) chol_small_batched_kernel(const SmallJob* jobs, int pass, int passes,
                                                                      double thr) {
  const SmallJob j = jobs[blockIdx.x];
  const int npass = passes == 1 ? 1 : 2;
  chol_small_body<MODE>(j.k, j.ws->Mh, j.ws->Ml, KMAX, j.ws, j.Oh, j.Ol, j.ldo, j.st, job_gates(j, pass, npass), pass,
                        passes, thr, j.out);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) svqb_small_batched_kernel(const SmallJob* jobs, int pass, int passes,
                                                                      double thr, double eps) {
  const SmallJob j = jobs[blockIdx.x];
  const int npass = passes == 1 ? 1 : 2;
  svqb_small_body<MODE>(j.k, j.ws->Mh, j.ws->Ml, KMAX, j.ws, j.Oh, j.Ol, j.ldo, j.tol, j.st,
                        job_gates(j, pass, npass), pass, passes, thr, eps, j.out, false);
}

__global__ void status_init_batched_kernel(const SmallJob* jobs, int njobs) {
  for (int b = blockIdx.x; b < njobs; b += gridDim.x) {
    DevStatus* s = jobs[b].st;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s->gate[i] = i == 0;
    if (threadIdx.x == 0) {
      s->info = 0;
      s->rank = jobs[b].k;
      s->iters = 0;
      s->sweeps = 0;
    }
  }
}

// ------------------------------------------------------ convergence test

__global__ void __launch_bounds__(kThreads) converge_kernel(const int* run, const double* Ch, const double* Cl, int ldc,
                                                            int kv, int k, const double* Mh, const double* Ml,
                                                            int ldm, double eps, DevStatus* st, int iter,
                                                            int max_iter, int* iters_user, int* rank_user) {
  if (*run == 0) return;
  // Frobenius norms of C and of M - I (each bounds the 2-norm from above),
  // as sums of squares in a fixed reduction order
  __shared__ double red[2][kThreads];
  double sc = 0.0, sm = 0.0;
  for (int t = threadIdx.x; t < kv * k; t += kThreads) {
    const int i = t % kv, j = t / kv;
    const double c = Ch[(size_t)j * ldc + i] + (Cl ? Cl[(size_t)j * ldc + i] : 0.0);
    sc += c * c;
  }
  for (int t = threadIdx.x; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    // (M_hi - delta) + M_lo: the subtraction of 1 is exact near 1
    const double e = (Mh[(size_t)j * ldm + i] - (i == j ? 1.0 : 0.0)) + (Ml ? Ml[(size_t)j * ldm + i] : 0.0);
    sm += e * e;
  }
  red[0][threadIdx.x] = sc;
  red[1][threadIdx.x] = sm;
  __syncthreads();
  for (int w = kThreads / 2; w >= 1; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double fc = sqrt(red[0][0]), fm = sqrt(red[1][0]);
    const bool conv = fc <= eps && fm <= eps;  // false for NaN
    st->gate[kItSvqb + iter] = conv ? 0 : 1;
    if (iter + 1 < max_iter) st->gate[kItRun + iter + 1] = conv ? 0 : 1;
    if (conv) st->iters = iter;  // updates applied before convergence was seen
    else if (iter + 1 == max_iter) st->iters = -max_iter;
    if (iters_user && (conv || iter + 1 == max_iter)) *iters_user = st->iters;
    if (rank_user && conv) *rank_user = st->rank;  // k when no SVQB was needed
  }
}

}  // namespace

cudaError_t launch_converge(const int* run, const double* Ch, const double* Cl, int ldc, int kv, int k,
                            const double* Mh, const double* Ml, int ldm, double eps, DevStatus* s, int iter,
                            int max_iter, int* iters_user, int* rank_user, cudaStream_t st) {
  converge_kernel<<<1, kThreads, 0, st>>>(run, Ch, Cl, ldc, kv, k, Mh, Ml, ldm, eps, s, iter, max_iter, iters_user,
                                          rank_user);
  return cudaGetLastError();
}

__global__ void symmetrize_kernel(int k, double* Mh, double* Ml, int ld, const int* gate) {
  if (gate && *gate == 0) return;
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    const int i = t % k, j = t / k;
    if (i >= j) continue;  // one thread per pair i < j
    const size_t u = (size_t)j * ld + i, l = (size_t)i * ld + j;
    dd s = dd_add(dd{Mh[u], Ml ? Ml[u] : 0.0}, dd{Mh[l], Ml ? Ml[l] : 0.0});
    s.hi *= 0.5;  // halving is exact
    s.lo *= 0.5;
    Mh[u] = Mh[l] = s.hi;
    if (Ml) Ml[u] = Ml[l] = s.lo;
  }
}

cudaError_t launch_symmetrize(int k, double* Mh, double* Ml, int ld, const int* gate, cudaStream_t st) {
  symmetrize_kernel<<<1, 256, 0, st>>>(k, Mh, Ml, ld, gate);
  return cudaGetLastError();
}

cudaError_t launch_status_init(DevStatus* s, int k, cudaStream_t st) {
  status_init_kernel<<<1, 32, 0, st>>>(s, k);
  return cudaGetLastError();
}

size_t chol_smem(int k) { return 3 * (size_t)k * k * sizeof(dd); }

cudaError_t launch_pivchol_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                                 double* R_hi, double* R_lo, int ldr, double tol, DevStatus* s, SmallGates g,
                                 int pass, int passes, int* info_user, int* rank_user, int* perm_user,
                                 cudaStream_t st) {
  const size_t smem = chol_smem(k);
  cudaError_t e;
  if (mode == MODE_DD) {
    e = set_dyn_smem(pivchol_small_kernel<MODE_DD>, smem);
    if (e != cudaSuccess) return e;
    pivchol_small_kernel<MODE_DD><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, R_hi, R_lo, ldr, tol, s, g, pass,
                                                              passes, 1e7, info_user, rank_user, perm_user);
  } else {
    e = set_dyn_smem(pivchol_small_kernel<MODE_FP64>, smem);
    if (e != cudaSuccess) return e;
    pivchol_small_kernel<MODE_FP64><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, R_hi, R_lo, ldr, tol, s, g,
                                                                pass, passes, 1e4, info_user, rank_user, perm_user);
  }
  return cudaGetLastError();
}
size_t svqb_smem(int k) {
  return 3 * (size_t)k * k * sizeof(dd) + (2 * (size_t)(k / 2 + 1) + k) * sizeof(dd) +
         (2 * (size_t)(k / 2 + 1) + k) * sizeof(int);
}

cudaError_t launch_chol_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                              double* R_hi, double* R_lo, int ldr, DevStatus* s, SmallGates g, int pass, int passes,
                              int* info_user, cudaStream_t st) {
  const size_t smem = chol_smem(k);
  cudaError_t e;
  if (mode == MODE_DD) {
    e = set_dyn_smem(chol_small_kernel<MODE_DD>, smem);
    if (e != cudaSuccess) return e;
    chol_small_kernel<MODE_DD><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, R_hi, R_lo, ldr, s, g, pass, passes,
                                                         1e7, info_user);
  } else {
    e = set_dyn_smem(chol_small_kernel<MODE_FP64>, smem);
    if (e != cudaSuccess) return e;
    chol_small_kernel<MODE_FP64><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, R_hi, R_lo, ldr, s, g, pass, passes,
                                                           1e4, info_user);
  }
  return cudaGetLastError();
}

cudaError_t launch_svqb_small(Mode mode, int k, const double* Mh, const double* Ml, int ldm, SmallWs* ws,
                              double* Z_hi, double* Z_lo, int ldz, double tol, DevStatus* s, SmallGates g, int pass,
                              int passes, int* rank_user, cudaStream_t st, bool rotated) {
  const size_t smem = svqb_smem(k);
  if (rotated) passes = 1;
  cudaError_t e;
  if (mode == MODE_DD) {
    if (tol < 0) tol = k * 0x1p-104;
    e = set_dyn_smem(svqb_small_kernel<MODE_DD>, smem);
    if (e != cudaSuccess) return e;
    svqb_small_kernel<MODE_DD><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, Z_hi, Z_lo, ldz, tol, s, g, pass,
                                                         passes, 1e7, kJacobiEpsDD, rank_user, rotated);
  } else {
    if (tol < 0) tol = k * 0x1p-52;
    e = set_dyn_smem(svqb_small_kernel<MODE_FP64>, smem);
    if (e != cudaSuccess) return e;
    svqb_small_kernel<MODE_FP64><<<1, kThreads, smem, st>>>(k, Mh, Ml, ldm, ws, Z_hi, Z_lo, ldz, tol, s, g, pass,
                                                           passes, 1e4, kJacobiEpsFP64, rank_user, rotated);
  }
  return cudaGetLastError();
}

double svqb_default_tol(Mode mode, int k) { return mode == MODE_DD ? k * 0x1p-104 : k * 0x1p-52; }

cudaError_t launch_status_init_batched(const SmallJob* jobs, int njobs, cudaStream_t st) {
  status_init_batched_kernel<<<std::min(njobs, 1024), 64, 0, st>>>(jobs, njobs);
  return cudaGetLastError();
}

cudaError_t launch_small_batched(bool chol, Mode mode, int njobs, int kmax, const SmallJob* jobs, int pass,
                                 int passes, cudaStream_t st) {
  const bool ddm = mode == MODE_DD;
  cudaError_t e;
  if (chol) {
    const size_t smem = chol_smem(kmax);
    auto kern = ddm ? chol_small_batched_kernel<MODE_DD> : chol_small_batched_kernel<MODE_FP64>;
    e = set_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<njobs, kThreads, smem, st>>>(jobs, pass, passes, ddm ? 1e7 : 1e4);
  } else {
    // A DD Jacobi eigensolve of 16 or more columns keeps one SM's FP64 pipe
    // busy on its own (a k = 32 one takes 7-11 ms alone): when several share
    // an SM they all slow down and the launch ends with the last of them.
    // Asking for more than half of an SM's shared memory keeps one such CTA
    // per SM (the jobs are ordered widest first, so the first wave spreads
    // the widest over the SMs).
    size_t smem = svqb_smem(kmax);
    if (kmax >= 16) smem = std::max<size_t>(smem, 116 * 1024);
    auto kern = ddm ? svqb_small_batched_kernel<MODE_DD> : svqb_small_batched_kernel<MODE_FP64>;
    e = set_dyn_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<njobs, kThreads, smem, st>>>(jobs, pass, passes, ddm ? 1e7 : 1e4, ddm ? kJacobiEpsDD : kJacobiEpsFP64);
  }
  return cudaGetLastError();
}

}  // namespace eo
