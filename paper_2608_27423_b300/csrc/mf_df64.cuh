// Double-float arithmetic: a value is hi + lo with two floats, |lo| <= ulp(hi)/2,
// about 48 significand bits.  Built from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA form of Dekker's product
// (TwoProd: the rounding error of a*b is fma(a, b, -a*b)).  Used for
// FP64-accurate operator applies on the FP32 pipes of B300, whose FP64 rate is
// 1/62 of its FP32 rate.  Addition is the accurate variant (both parts summed
// with TwoSum), so cancellation costs no more than ~2^-48 of the result.
#pragma once
#include <cuda_runtime.h>

namespace mf {

// keep the CUDA fma overloads (float, double) visible next to the df one below
using ::fma;

struct df {
  float hi, lo;
  df() = default;   // trivial: usable in __constant__ tables; df() value-initialises to zero
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit df(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit df(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df(s, e);
}
__device__ __forceinline__ df df_quick_two_sum(float a, float b) {   // requires |a| >= |b|
  const float s = a + b;
  const float e = b - (s - a);
  return df(s, e);
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  return df(p, e);
}
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  const df t = df_two_sum(a.lo, b.lo);
  const df u = df_quick_two_sum(s.hi, s.lo + t.hi);
  return df_quick_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const df p = df_two_prod(a.hi, b.hi);
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return df_quick_two_sum(p.hi, e);
}
// a*b + c: exact product of the high parts (TwoProd), cross terms folded into
// its error, one TwoSum of the high parts, low parts added in float.  Error
// about 2^-48 of max(|a b|, |c|), i.e. ~30x FP64's 2^-53 under cancellation.
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = a.hi * b.hi;
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe));
  const df s = df_two_sum(p, c.hi);
  return df_quick_two_sum(s.hi, s.lo + (pe + c.lo));
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df& operator-=(df& a, df b) { a = a - b; return a; }
__device__ __forceinline__ df& operator*=(df& a, df b) { a = a * b; return a; }

// I/O types of the apply: double vectors in memory, df in registers
template <typename T> struct IO { using type = T; };
template <> struct IO<df> { using type = double; };
template <typename T> __device__ __forceinline__ T from_io(typename IO<T>::type x) { return (T)x; }
template <> __device__ __forceinline__ df from_io<df>(double x) { return df(x); }
template <typename T> __device__ __forceinline__ typename IO<T>::type to_io(T x) { return x; }
template <> __device__ __forceinline__ double to_io<df>(df x) { return x.to_double(); }

// split a double array into df pairs (hi, lo)
__global__ void k_split_df(const double* __restrict__ a, df* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = df(a[i]);
}

}  // namespace mf
