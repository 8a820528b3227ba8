// Double-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 significant bits). Built from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA-based exact product
// (TwoProd); addition and multiplication follow the "sloppy" double-word
// algorithms analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017).
// Used for the element kernels of the mixed-precision form: FP32 units run
// 62x more operations per clock than FP64 ones on this part, and one
// double-float multiply-add costs about 18 FP32 operations.
#pragma once

#include <cuda_runtime.h>

namespace dgdf {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ dfl(int v) : hi(float(v)), lo(0.f) {}
  __host__ __device__ __forceinline__ explicit dfl(double v) {
    hi = float(v);
    lo = float(v - double(hi));
  }
  __host__ __device__ __forceinline__ explicit operator double() const { return double(hi) + double(lo); }
};

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__host__ __device__ __forceinline__ dfl operator+(dfl x, dfl y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e += x.lo + y.lo;
  float h, l;
  fast_two_sum(s, e, h, l);
  return dfl(h, l);
}

__host__ __device__ __forceinline__ dfl operator-(dfl x) { return dfl(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }

__host__ __device__ __forceinline__ dfl operator*(dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return dfl(h, l);
}

// Multiplication by 1/2 is exact on both words.
__host__ __device__ __forceinline__ dfl half(dfl x) { return dfl(0.5f * x.hi, 0.5f * x.lo); }

__host__ __device__ __forceinline__ double to_double(dfl x) { return double(x.hi) + double(x.lo); }
__host__ __device__ __forceinline__ double to_double(float2 x) { return double(x.x) + double(x.y); }
__host__ __device__ __forceinline__ dfl to_dfl(float2 x) { return dfl(x.x, x.y); }
__host__ __device__ __forceinline__ float2 to_float2(dfl x) { return make_float2(x.hi, x.lo); }

// Compensated accumulator for sums of double-float products (the Dot2 scheme of
// Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005), applied to double-float
// operands): s carries the running FP32 sum of the leading products, c the sum of
// every rounding error, each captured exactly by TwoProd / TwoSum. One
// multiply-add costs 12 FP32 operations; the pair is normalised once, by val().
struct dacc {
  float s, c;
};

__host__ __device__ __forceinline__ dacc dacc_zero() { return dacc{0.f, 0.f}; }
__host__ __device__ __forceinline__ dacc dacc_of(dfl x) { return dacc{x.hi, x.lo}; }

// a += x * y (the lo * lo product is below the double-float rounding and dropped)
__host__ __device__ __forceinline__ void mad(dacc& a, dfl x, dfl y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, t;
  two_sum(a.s, p, s, t);
  a.s = s;
  a.c += t + e;
}

// a += x * z for a double-float x and an FP32 z
__host__ __device__ __forceinline__ void mad(dacc& a, dfl x, float z) {
  const float p = x.hi * z;
  float e = fmaf(x.hi, z, -p);
  e = fmaf(x.lo, z, e);
  float s, t;
  two_sum(a.s, p, s, t);
  a.s = s;
  a.c += t + e;
}

__host__ __device__ __forceinline__ dfl val(dacc a) {
  float h, l;
  two_sum(a.s, a.c, h, l);
  return dfl(h, l);
}

__host__ __device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) { return x = x + y; }
__host__ __device__ __forceinline__ dfl& operator-=(dfl& x, dfl y) { return x = x - y; }
__host__ __device__ __forceinline__ dfl& operator*=(dfl& x, dfl y) { return x = x * y; }
__host__ __device__ __forceinline__ bool operator>=(dfl x, dfl y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo >= y.lo);
}

}  // namespace dgdf
