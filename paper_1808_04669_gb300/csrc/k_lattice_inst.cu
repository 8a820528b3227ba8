// One instantiation of the lattice facet solver k_solve_lat<K, MIXED> (k_lattice_kernel.cuh):
// the build compiles this file once per (K, form) with -DDG_LAT_K=<1..3> -DDG_LAT_MIXED=<0|1>,
// so that the six instantiations compile in parallel.
#include "k_lattice_kernel.cuh"

#if !defined(DG_LAT_K) || !defined(DG_LAT_MIXED)
#error "compile with -DDG_LAT_K=<1..3> -DDG_LAT_MIXED=<0|1>"
#endif

#define DG_LAT_CAT2(a, b, c) a##b##_##c
#define DG_LAT_CAT(a, b, c) DG_LAT_CAT2(a, b, c)

namespace dgdf {

const void* DG_LAT_CAT(lattice_kernel_k, DG_LAT_K, DG_LAT_MIXED)() {
  return (const void*)k_solve_lat<DG_LAT_K, DG_LAT_MIXED != 0>;
}

}  // namespace dgdf
