// Device helpers shared by the kernels: sizes per degree, coefficient loads,
// warp/block reductions (fixed order, so results are bitwise reproducible) and
// a grid barrier with a bounded wait.
#pragma once

#include <cuda_runtime.h>

namespace dgdf {

template <int K>
struct Dims {
  static constexpr int NS = (K + 1) * (K + 2) / 2;   // scalar P^k per triangle
  static constexpr int ND = 2 * NS;                  // broken vector DOFs per triangle
  static constexpr int NW = K * (K + 1) / 2;         // P^{k-1} per triangle
  static constexpr int NL = K + 1;                   // P^k per facet
  static constexpr int NQ = K == 1 ? 3 : (K == 2 ? 7 : 16);   // symmetric volume rule, exact to degree 3k-1
  static constexpr int NQF = (3 * K + 2) / 2;        // ceil((3k+1)/2) Gauss-Legendre points per facet
};

template <int N, typename R>
__device__ __forceinline__ void load_coef(const double* __restrict__ p, R (&c)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) c[i] = R(p[i]);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum; every thread of the block must call it; the result is valid in all threads.
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T part[32];
  __syncthreads();
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  T r = (l < nw) ? part[l] : T(0);
  r = warp_sum(r);
  return r;
}

template <typename T>
__device__ __forceinline__ T block_max(T v) {
  __shared__ T part[32];
  __syncthreads();
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) part[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  T r = (l < nw) ? part[l] : T(0);
  r = warp_max(r);
  return r;
}

}  // namespace dgdf
