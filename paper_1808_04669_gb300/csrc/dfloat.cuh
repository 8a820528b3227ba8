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

// ---- two double-float values side by side: their leading words in one float2 and their
// trailing words in another, so that the packed FP32x2 instructions of sm_100+ act on both
// at once (same FP32 throughput as scalar instructions, half the issue slots).
struct dfl2 {
  float2 hi, lo;
};
// paired compensated accumulators (two independent dacc)
struct dacc2 {
  float2 s, c;
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ dacc2 dacc2_zero() { return dacc2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// a += x * y for both halves (Dot2 step, as mad() on dacc, in packed form)
__device__ __forceinline__ void mad2(dacc2& a, const dfl2& x, const dfl2& y) {
  const float2 p = f2mul(x.hi, y.hi);
  float2 e = f2fma(x.hi, y.hi, make_float2(-p.x, -p.y));
  e = f2fma(x.hi, y.lo, e);
  e = f2fma(x.lo, y.hi, e);
  const float2 s = f2add(a.s, p);
  const float2 bb = f2sub(s, a.s);
  const float2 t = f2add(f2sub(a.s, f2sub(s, bb)), f2sub(p, bb));
  a.s = s;
  a.c = f2add(a.c, f2add(t, e));
}

// the same value y for both halves
__device__ __forceinline__ dfl2 splat(dfl y) {
  return dfl2{make_float2(y.hi, y.hi), make_float2(y.lo, y.lo)};
}

// the two accumulated values
__device__ __forceinline__ dfl val_x(const dacc2& a) { return val(dacc{a.s.x, a.c.x}); }
__device__ __forceinline__ dfl val_y(const dacc2& a) { return val(dacc{a.s.y, a.c.y}); }
// their sum (a sum split over even and odd terms)
__device__ __forceinline__ dfl val_sum(const dacc2& a) {
  float s, t;
  two_sum(a.s.x, a.s.y, s, t);
  return val(dacc{s, (a.c.x + a.c.y) + t});
}

__host__ __device__ __forceinline__ dfl& operator+=(dfl& x, dfl y) { return x = x + y; }
__host__ __device__ __forceinline__ dfl& operator-=(dfl& x, dfl y) { return x = x - y; }
__host__ __device__ __forceinline__ dfl& operator*=(dfl& x, dfl y) { return x = x * y; }
__host__ __device__ __forceinline__ bool operator>=(dfl x, dfl y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo >= y.lo);
}

}  // namespace dgdf
