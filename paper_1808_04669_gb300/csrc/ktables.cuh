// Reference tables of the element kernels (volume and facet quadrature values of
// the Dubiner basis and its reference gradients), staged in shared memory.
#pragma once

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"

namespace dgdf {

// Reference tables staged in shared memory in precision R.
template <int K, typename R>
struct SmemTables {
  using D = Dims<K>;
  R vw[D::NQ];
  R vphi[D::NQ][D::NS];
  R vdphi[D::NQ][D::NS][2];
  R fw[D::NQF];
  R fphi[3][D::NQF][D::NS];
  R fdphi[3][D::NQF][D::NS][2];
};

template <int K, typename R>
__device__ __forceinline__ void load_tables(const DevMesh& m, SmemTables<K, R>& T) {
  using D = Dims<K>;
  for (int i = threadIdx.x; i < D::NQ; i += blockDim.x) T.vw[i] = R(m.vw[i]);
  for (int i = threadIdx.x; i < D::NQ * D::NS; i += blockDim.x) (&T.vphi[0][0])[i] = R(m.vphi[i]);
  for (int i = threadIdx.x; i < D::NQ * D::NS * 2; i += blockDim.x) (&T.vdphi[0][0][0])[i] = R(m.vdphi[i]);
  for (int i = threadIdx.x; i < D::NQF; i += blockDim.x) T.fw[i] = R(m.fw[i]);
  for (int i = threadIdx.x; i < 3 * D::NQF * D::NS; i += blockDim.x) (&T.fphi[0][0][0])[i] = R(m.fphi[i]);
  for (int i = threadIdx.x; i < 3 * D::NQF * D::NS * 2; i += blockDim.x) (&T.fdphi[0][0][0][0])[i] = R(m.fdphi[i]);
}

// Number of float2 words of the double-float tables (the host builds m.tab_df in
// exactly this field order).
template <int K>
struct TablesDf {
  using D = Dims<K>;
  static constexpr int words = D::NQ + D::NQ * D::NS * 3 + D::NQF + 3 * D::NQF * D::NS * 3;
};

// Double-float tables copied from their precomputed (hi, lo) image, no conversions.
template <int K>
__device__ __forceinline__ void load_tables_df(const DevMesh& m, SmemTables<K, dfl>& T) {
  static_assert(sizeof(SmemTables<K, dfl>) == sizeof(float2) * TablesDf<K>::words, "table layout");
  float2* dst = reinterpret_cast<float2*>(&T);
  for (int i = threadIdx.x; i < TablesDf<K>::words; i += blockDim.x) dst[i] = m.tab_df[i];
}

}  // namespace dgdf
