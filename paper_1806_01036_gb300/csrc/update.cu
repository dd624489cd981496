// update.cu — the final multiplication Y = Y~ Z of phase II
// (arXiv:1806.01036, Sec. 4.2: the multiplication by Z that ends phase II; CholQR uses
// the upper-triangular Z = R^{-1}, SVQB the full symmetric Z).
//
// Each thread owns whole rows: it loads the k entries of its row, then forms
// q_j = sum_i x_i Z_ij (i <= j for triangular Z) with DD accumulation of the
// exact products x_i * (Z_hi + Z_lo)_ij in EO_DD (one rounding per entry), or
// FP64 fma accumulation otherwise.  All loads of a row precede its stores, so
// the update is done in place.  Z lives in shared memory.
#include <algorithm>

#include "common.cuh"

namespace eo {
namespace {

constexpr int kThreads = 128;

template <int MODE, typename T, int KM>
__global__ void __launch_bounds__(kThreads) update_kernel(int64_t n, int k, T* X, int64_t ldx,
                                                          const double* __restrict__ Zh, const double* __restrict__ Zl,
                                                          int tri, const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* Zs = reinterpret_cast<dd*>(smem_raw);  // k-by-k, leading dimension k
  for (int t = threadIdx.x; t < k * k; t += kThreads) {
    const int i = t % k, j = t / k;
    Zs[j * k + i] = dd{Zh[(size_t)j * KMAX + i], Zl[(size_t)j * KMAX + i]};
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x; r < n; r += stride) {
    double x[KM];  // the whole row stays in registers, so q_j may overwrite x_j at once
#pragma unroll
    for (int i = 0; i < KM; ++i) x[i] = i < k ? (double)X[(size_t)i * ldx + r] : 0.0;
#pragma unroll 1
    for (int j = 0; j < k; ++j) {
      const int iend = tri ? j + 1 : k;
      double q;
      if (MODE == MODE_DD) {
        dd s = dd{0.0, 0.0};
#pragma unroll
        for (int i = 0; i < KM; ++i)
          if (i < iend) dd_fma_acc_dd(s, Zs[j * k + i], x[i]);
        q = __dadd_rn(s.hi, s.lo);
      } else {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < KM; ++i)
          if (i < iend) s = __fma_rn(x[i], Zs[j * k + i].hi, s);
        q = s;
      }
      X[(size_t)j * ldx + r] = (T)q;
    }
  }
}

template <int MODE, typename T>
cudaError_t launch_k(int64_t n, int k, void* X, int64_t ldx, const double* Zh, const double* Zl, bool tri,
                     const int* gate, cudaStream_t st) {
  T* x = static_cast<T*>(X);
  int64_t blocks64 = (n + kThreads - 1) / kThreads;
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks64, 152 * 16));
  const int t = tri ? 1 : 0;
  const size_t smem = (size_t)k * k * sizeof(dd);
  cudaError_t e = cudaSuccess;
  if (k <= 8) {
    update_kernel<MODE, T, 8><<<blocks, kThreads, smem, st>>>(n, k, x, ldx, Zh, Zl, t, gate);
  } else if (k <= 16) {
    update_kernel<MODE, T, 16><<<blocks, kThreads, smem, st>>>(n, k, x, ldx, Zh, Zl, t, gate);
  } else if (k <= 32) {
    update_kernel<MODE, T, 32><<<blocks, kThreads, smem, st>>>(n, k, x, ldx, Zh, Zl, t, gate);
  } else {
    e = set_dyn_smem(update_kernel<MODE, T, 64>, smem);
    if (e != cudaSuccess) return e;
    update_kernel<MODE, T, 64><<<blocks, kThreads, smem, st>>>(n, k, x, ldx, Zh, Zl, t, gate);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_update(Mode mode, int64_t n, int k, void* X, int64_t ldx, const double* Zh, const double* Zl,
                          bool tri, const int* gate, cudaStream_t st) {
  switch (mode) {
    case MODE_DD: return launch_k<MODE_DD, double>(n, k, X, ldx, Zh, Zl, tri, gate, st);
    case MODE_F32: return launch_k<MODE_F32, float>(n, k, X, ldx, Zh, Zl, tri, gate, st);
    default: return launch_k<MODE_FP64, double>(n, k, X, ldx, Zh, Zl, tri, gate, st);
  }
}

}  // namespace eo
