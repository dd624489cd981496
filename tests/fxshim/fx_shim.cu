// Host-side shim over the library's fixed-point arithmetic (fx.cuh), so that
// the CPU tests can check the exact same integer code the GPU kernels run
// against exact rational arithmetic.  Test infrastructure only.
#include <cstdint>

#include "fx.cuh"

using namespace eo::fx;

extern "C" {

int fxs_align_exp(double x) { return align_exp(x); }

void fxs_to_limbs(double x, int A, int* out) {
  Limbs L = to_limbs(x, A);
  for (int a = 0; a < 4; ++a) out[a] = L.v[a];
}

void fxs_to_limbs_dd(double h, double l, int A, int* out) {
  Limbs L = to_limbs_dd(h, l, A);
  for (int a = 0; a < 4; ++a) out[a] = L.v[a];
}

// sum_i x_i y_i the way the kernels do it: every x aligned to Ax, every y to
// Ay, limb products accumulated per diagonal, combined into W, rounded once to
// a double-double.  n <= kRowsPerDrain.
void fxs_dot(int n, const double* x, const double* y, int Ax, int Ay, double* hi, double* lo) {
  long long acc[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) mac(acc, to_limbs(x[i], Ax), to_limbs(y[i], Ay));
  w_to_dd(acc_to_w(acc), Ax + Ay - kScaleOffset, *hi, *lo);
}

// The dot product of fxs_dot, but the alignment of y grows from Ay0 to Ay1
// after the first n0 terms (the accumulator is rescaled, as in the Gram kernel).
void fxs_dot_rescaled(int n, int n0, const double* x, const double* y, int Ax, int Ay0, int Ay1, double* hi,
                      double* lo) {
  long long acc[4] = {0, 0, 0, 0};
  for (int i = 0; i < n0; ++i) mac(acc, to_limbs(x[i], Ax), to_limbs(y[i], Ay0));
  acc_shift(acc, Ay1 - Ay0);
  for (int i = n0; i < n; ++i) mac(acc, to_limbs(x[i], Ax), to_limbs(y[i], Ay1));
  w_to_dd(acc_to_w(acc), Ax + Ay1 - kScaleOffset, *hi, *lo);
}

static i128 mk(long long lo, long long hi) { return (i128)(((u128)(unsigned long long)hi << 64) | (unsigned long long)lo); }

void fxs_w_to_dd(long long wlo, long long whi, int S, double* hi, double* lo) { w_to_dd(mk(wlo, whi), S, *hi, *lo); }

double fxs_w_to_double(long long wlo, long long whi, int S) { return w_to_double(mk(wlo, whi), S); }

double fxs_sub_round(double y, long long wlo, long long whi, int S) { return sub_round(y, mk(wlo, whi), S); }

double fxs_w_to_double_fast(long long wlo, long long whi, int S, int* ok) {
  bool o = false;
  const double r = w_to_double_fast(mk(wlo, whi), S, o);
  *ok = o;
  return r;
}

double fxs_sub_round_fast(double y, long long wlo, long long whi, int S, int* ok) {
  bool o = false;
  const double r = sub_round_fast(y, mk(wlo, whi), S, o);
  *ok = o;
  return r;
}

// Sum of m 128-bit terms in the 256-bit accumulator, narrowed back to 128 bits
// (w_out, extra shift).
void fxs_acc256(int m, const long long* lo, const long long* hi, long long* wlo, long long* whi, int* extra) {
  Acc256 a;
  a.zero();
  for (int i = 0; i < m; ++i) a.add(mk(lo[i], hi[i]));
  int e = 0;
  i128 w = a.narrow(e);
  *wlo = (long long)(unsigned long long)(u128)w;
  *whi = (long long)(w >> 64);
  *extra = e;
}

int fxs_scale_offset(void) { return kScaleOffset; }
}
