// project.cu — phase I projection Y~ = Y - V C fused with the phase-II Gram
// matrix M = Y~^T Y~ (arXiv:1806.01036, Sec. 4.2: the plain projection
// Y~ = (I - W W^T) X of phase I, and "kernel fusion (combining several basic
// operations to further reduce memory accesses)").
//
// C = V^T Y is computed beforehand by the Gram kernels.  This kernel reads V
// and Y once, writes Y~ once, and accumulates M from the rounded Y~ it wrote:
//   phase 1 (per panel of P rows): thread (row, column group) forms
//     y~_j = y_j - sum_i v_i C_ij, accumulated in DD (EO_DD) or FP64 and
//     rounded once, stores it to Yout and to a shared-memory panel;
//   phase 2: the CTA's threads own TSxTS tiles of M and accumulate the
//     panel's rows (Dot2 in EO_DD) into register accumulators that persist
//     across panels;
//   end: tiles are summed over the threads sharing them in a fixed order and
//   stored as the CTA's partial; the Gram reducer of gram.cu-style (below)
//   produces M.
#include <algorithm>

#include "common.cuh"

namespace eo {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 16;  // output columns per thread in phase 1
constexpr int TS = 4;       // M tile size in phase 2

__device__ __forceinline__ dd shfl_xor_dd(dd v, int m) {
  return dd{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

template <int MODE>
__device__ __forceinline__ dd addm(dd a, dd b) {
  if (MODE == MODE_DD) return dd_add(a, b);
  return dd{__dadd_rn(a.hi, b.hi), 0.0};
}

// Shared memory: C (kv*k dd) followed by the panel (P*k doubles).
template <int MODE>
__global__ void __launch_bounds__(kThreads) project_fused_kernel(int64_t n, int kv, const double* __restrict__ V,
                                                                 int64_t ldv, int k, const double* Y,
                                                                 int64_t ldy, double* Yout, int64_t ldyo,
                                                                 const double* __restrict__ C_hi,
                                                                 const double* __restrict__ C_lo, int ldc, int P,
                                                                 int want_m, dd* __restrict__ parts,
                                                                 const int* gate) {
  if (gate && *gate == 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* Cs = reinterpret_cast<dd*>(smem_raw);
  double* panel = reinterpret_cast<double*>(Cs + (size_t)kv * k);
  __shared__ dd red[kThreads];

  for (int t = threadIdx.x; t < kv * k; t += kThreads) {
    int i = t % kv, j = t / kv;
    Cs[t] = dd{C_hi[(size_t)j * ldc + i], C_lo ? C_lo[(size_t)j * ldc + i] : 0.0};
  }
  __syncthreads();

  const int ngroups = (k + kGroup - 1) / kGroup;
  const int nt = (k + TS - 1) / TS;
  const int ntiles = nt * (nt + 1) / 2;
  const int lanes_per_tile = kThreads / ntiles;  // >= 1 for k <= 64
  const int my_tile = threadIdx.x % ntiles;
  const int my_lane = threadIdx.x / ntiles;
  const bool gram_active = want_m && my_lane < lanes_per_tile;
  int ti = 0, tj = 0;
  {
    int t = my_tile, row = 0;
    while (t >= nt - row) {
      t -= nt - row;
      ++row;
    }
    ti = row;
    tj = row + t;
  }

  dd acc[TS][TS];
#pragma unroll
  for (int a = 0; a < TS; ++a)
#pragma unroll
    for (int b = 0; b < TS; ++b) acc[a][b] = dd{0.0, 0.0};

  const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpc;
  const int64_t r1 = min(n, r0 + rpc);

  for (int64_t pr = r0; pr < r1; pr += P) {
    const int rows = (int)min((int64_t)P, r1 - pr);
    // phase 1: projection of the panel
    for (int w = threadIdx.x; w < P * ngroups; w += kThreads) {
      const int lr = w % P, g = w / P;
      if (lr >= rows) continue;
      const int64_t r = pr + lr;
      const int jb = g * kGroup, je = min(k, jb + kGroup);
      dd s[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q) s[q] = dd{0.0, 0.0};
      for (int i = 0; i < kv; ++i) {
        const double v = __ldg(V + (size_t)i * ldv + r);
#pragma unroll
        for (int q = 0; q < kGroup; ++q) {
          if (jb + q < je) {
            const dd c = Cs[(size_t)(jb + q) * kv + i];
            if (MODE == MODE_DD)
              dd_fma_acc_dd(s[q], c, v);
            else
              s[q].hi = __fma_rn(v, c.hi, s[q].hi);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        if (jb + q < je) {
          const int j = jb + q;
          const double y = Y[(size_t)j * ldy + r];  // Y may alias Yout: plain load
          double out;
          if (MODE == MODE_DD) {
            dd t = two_sum(y, -s[q].hi);
            t.lo = __dsub_rn(t.lo, s[q].lo);
            out = __dadd_rn(t.hi, t.lo);
          } else {
            out = __dsub_rn(y, s[q].hi);
          }
          Yout[(size_t)j * ldyo + r] = out;
          panel[(size_t)j * P + lr] = out;
        }
      }
    }
    __syncthreads();
    // phase 2: Gram tiles over the panel
    if (gram_active) {
      for (int lr = my_lane; lr < rows; lr += lanes_per_tile) {
        double xv[TS], yv[TS];
#pragma unroll
        for (int a = 0; a < TS; ++a) {
          const int i = min(ti * TS + a, k - 1), j = min(tj * TS + a, k - 1);
          xv[a] = panel[(size_t)i * P + lr];
          yv[a] = panel[(size_t)j * P + lr];
        }
#pragma unroll
        for (int a = 0; a < TS; ++a)
#pragma unroll
          for (int b = 0; b < TS; ++b) {
            if (MODE == MODE_DD)
              dd_fma_acc(acc[a][b], xv[a], yv[b]);
            else
              acc[a][b].hi = __fma_rn(xv[a], yv[b], acc[a][b].hi);
          }
      }
    }
    __syncthreads();
  }
  if (!want_m) return;

  // Sum the tile accumulators over the lanes that share a tile, lane 0 first.
  const int E = k * k;
#pragma unroll
  for (int a = 0; a < TS; ++a)
#pragma unroll
    for (int b = 0; b < TS; ++b) {
      red[threadIdx.x] = (MODE == MODE_DD) ? dd_norm(acc[a][b]) : acc[a][b];
      __syncthreads();
      if (my_lane == 0) {
        dd v = red[threadIdx.x];
        for (int l = 1; l < lanes_per_tile; ++l) v = addm<MODE>(v, red[l * ntiles + my_tile]);
        const int i = ti * TS + a, j = tj * TS + b;
        if (i < k && j < k) parts[(size_t)blockIdx.x * E + (size_t)j * k + i] = v;
      }
      __syncthreads();
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) sym_reduce_kernel(int k, int nparts, const dd* __restrict__ parts,
                                                              double* G_hi, double* G_lo, int ldg, const int* gate) {
  if (gate && *gate == 0) return;
  const int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int E = k * k;
  if (warp >= E) return;
  const int i = warp % k, j = warp / k;
  if (i > j) return;
  dd v = dd{0.0, 0.0};
  for (int p = lane; p < nparts; p += 32) v = addm<MODE>(v, parts[(size_t)p * E + warp]);
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v = addm<MODE>(v, shfl_xor_dd(v, m));
  if (lane == 0) {
    if (MODE == MODE_DD) v = fast_two_sum(v.hi, v.lo);
    G_hi[(size_t)j * ldg + i] = v.hi;
    G_hi[(size_t)i * ldg + j] = v.hi;
    if (G_lo) {
      G_lo[(size_t)j * ldg + i] = v.lo;
      G_lo[(size_t)i * ldg + j] = v.lo;
    }
  }
}

int panel_rows(int k) {
  const int ngroups = (k + kGroup - 1) / kGroup;
  return std::max(32, kThreads / ngroups);
}

int project_parts(int64_t n, int k) {
  const int P = panel_rows(k);
  int64_t by_rows = (n + P - 1) / P;
  return (int)std::max<int64_t>(1, std::min<int64_t>(by_rows, 152 * 2));
}

}  // namespace

size_t project_scratch_bytes(int64_t n, int kv, int k) {
  (void)kv;
  return (size_t)project_parts(n, k) * (size_t)k * k * sizeof(dd);
}

cudaError_t launch_project_fused(Mode mode, int64_t n, int kv, const double* V, int64_t ldv, int k, const double* Y,
                                 int64_t ldy, double* Yout, int64_t ldyo, const double* C_hi, const double* C_lo,
                                 int ldc, void* scratch, double* M_hi, double* M_lo, int ldm, const int* gate,
                                 cudaStream_t st) {
  const int P = panel_rows(k);
  const int np = project_parts(n, k);
  const size_t smem = (size_t)kv * k * sizeof(dd) + (size_t)P * k * sizeof(double);
  dd* parts = static_cast<dd*>(scratch);
  const int want_m = M_hi != nullptr;
  cudaError_t e;
  if (mode == MODE_DD) {
    e = set_dyn_smem(project_fused_kernel<MODE_DD>, smem);
    if (e != cudaSuccess) return e;
    project_fused_kernel<MODE_DD><<<np, kThreads, smem, st>>>(n, kv, V, ldv, k, Y, ldy, Yout, ldyo, C_hi, C_lo, ldc, P,
                                                              want_m, parts, gate);
    if (want_m) sym_reduce_kernel<MODE_DD><<<(k * k * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(k, np, parts, M_hi, M_lo, ldm, gate);
  } else {
    e = set_dyn_smem(project_fused_kernel<MODE_FP64>, smem);
    if (e != cudaSuccess) return e;
    project_fused_kernel<MODE_FP64><<<np, kThreads, smem, st>>>(n, kv, V, ldv, k, Y, ldy, Yout, ldyo, C_hi, C_lo, ldc,
                                                                P, want_m, parts, gate);
    if (want_m) sym_reduce_kernel<MODE_FP64><<<(k * k * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(k, np, parts, M_hi, M_lo, ldm, gate);
  }
  return cudaGetLastError();
}

}  // namespace eo
