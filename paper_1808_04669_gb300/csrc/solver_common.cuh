// Device helpers shared by the facet-system solvers (k_solver.cu, k_lattice.cu):
// the bounded grid barrier, fixed-order grid reductions and the stencil SpMV.
#pragma once

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"

namespace dgdf {
namespace {

constexpr int kSolverThreads = 256;
constexpr unsigned long long kBarrierSpinLimit = 1ull << 26;

// Grid barrier with a bounded wait. All blocks are co-resident (cooperative
// launch). One atomic per block: block 0 adds 2^31 - (nblocks - 1), the others
// add 1, so the word's top bit flips exactly when the last block arrives and
// the low bits return to zero; a block waits for the top bit to differ from the
// value its own add returned. The word must be zero at launch. Returns false
// if the wait ran out, after setting kFlagBarrierTimeout; once that flag is set
// (by any block) every later barrier of the launch returns false at once, and a
// waiting block stops waiting, so the whole grid leaves within one wait limit.
// Test hooks (DevStats): spin_limit replaces the default limit; skip_block
// names a block that leaves without arriving, so that the others' wait runs out.
__device__ bool grid_sync(GridBar* bar, DevStats* st) {
  __shared__ int ok;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* vflags = &st->flags;
    const unsigned long long limit = st->spin_limit ? st->spin_limit : kBarrierSpinLimit;
    int good = 1;
    if ((*vflags & kFlagBarrierTimeout) || int(blockIdx.x) == st->skip_block - 1) {
      good = 0;
    } else {
      const unsigned int nb = gridDim.x;
      const unsigned int inc = (blockIdx.x == 0) ? (0x80000000u - (nb - 1u)) : 1u;
      const unsigned int old = atomicAdd(&bar->count, inc);
      volatile unsigned int* v = &bar->count;
      unsigned long long spins = 0;
      while (((*v ^ old) & 0x80000000u) == 0u) {
        if (++spins > limit) {
          atomicOr(&st->flags, kFlagBarrierTimeout);
          good = 0;
          break;
        }
        if ((spins & 255u) == 0u && (*vflags & kFlagBarrierTimeout)) {
          good = 0;
          break;
        }
        if (spins > 32) __nanosleep(20);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Writes N block partials to red slots, synchronises the grid, and returns
// the grid sums in every thread (same summation order in every block).
template <int N>
__device__ bool grid_reduce(const DevMesh& m, int slot0, double (&v)[N], GridBar* bar) {
  double s[N];
#pragma unroll
  for (int i = 0; i < N; ++i) s[i] = block_sum(v[i]);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) m.red[size_t(slot0 + i) * kMaxSolverBlocks + blockIdx.x] = s[i];
  }
  if (!grid_sync(bar, m.stats)) return false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double a = 0.0;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) a += __ldcg(&m.red[size_t(slot0 + i) * kMaxSolverBlocks + b]);
    v[i] = block_sum(a);
  }
  return true;
}

template <int NL, typename R>
__device__ __forceinline__ void stencil_rows(const R* __restrict__ blk, const R (&x)[5][NL], R (&y)[NL]) {
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    R v = R(0);
#pragma unroll
    for (int b = 0; b < 5; ++b)
#pragma unroll
      for (int j = 0; j < NL; ++j) v += __ldg(&blk[(b * NL + i) * NL + j]) * x[b][j];
    y[i] = v;
  }
}

template <int NL, typename R>
__device__ __forceinline__ void block_apply(const R* __restrict__ B, const R (&x)[NL], R (&y)[NL]) {
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    R v = R(0);
#pragma unroll
    for (int j = 0; j < NL; ++j) v += __ldg(&B[i * NL + j]) * x[j];
    y[i] = v;
  }
}

// g_F = sum over both sides of facet f (one on a wall) of the side's condensation output mapped to
// the facet's canonical orientation (odd Legendre modes change sign when a side
// traverses the facet backwards). Mixed form: the sides' double-float values are
// summed in double-float and rounded to FP64 once.
template <int NL>
__device__ __forceinline__ void assemble_g_df(const DevMesh& m, int f, dfl (&gv)[NL]);

template <int NL>
__device__ __forceinline__ void assemble_g(const DevMesh& m, int f, double (&gv)[NL]) {
  if (m.elem_df) {
    dfl acc[NL];
    assemble_g_df<NL>(m, f, acc);
#pragma unroll
    for (int j = 0; j < NL; ++j) gv[j] = to_double(acc[j]);
    return;
  }
#pragma unroll
  for (int j = 0; j < NL; ++j) gv[j] = 0.0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int t = __ldg(&m.facet_tri[size_t(f) * 2 + s]);
    if (t < 0) break;   // a wall has one side
    const int e = __ldg(&m.facet_loc[size_t(f) * 2 + s]);
    const bool flip = __ldg(&m.tri_orient[size_t(t) * 3 + e]) < 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const double v = m.gl[size_t(t) * 3 * NL + e * NL + j];
      gv[j] += (flip && (j & 1)) ? -v : v;
    }
  }
}

// The same in double-float (mixed form), from the double-float condensation outputs.
template <int NL>
__device__ __forceinline__ void assemble_g_df(const DevMesh& m, int f, dfl (&gv)[NL]) {
#pragma unroll
  for (int j = 0; j < NL; ++j) gv[j] = dfl(0);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int t = __ldg(&m.facet_tri[size_t(f) * 2 + s]);
    if (t < 0) break;   // a wall has one side
    const int e = __ldg(&m.facet_loc[size_t(f) * 2 + s]);
    const bool flip = __ldg(&m.tri_orient[size_t(t) * 3 + e]) < 0;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const dfl v = to_dfl(m.gl_df[size_t(t) * 3 * NL + e * NL + j]);
      gv[j] += (flip && (j & 1)) ? -v : v;
    }
  }
}

// g on the boundary facets of Sec. 2.5, eq. (be): zero on outflow facets (their multipliers
// are zero: identity rows of S), and minus the data moments <mu_m, u_in.n> on inflow facets,
// so that the solution takes u.n = u_in.n there (homog: u.n = 0 instead).
template <int NL>
__device__ __forceinline__ void boundary_g(const DevMesh& m, int f, int homog, double (&gv)[NL]) {
  if (!m.facet_kind) return;
  const int kd = __ldg(&m.facet_kind[f]);
  if (kd == kFacetOutflow) {
#pragma unroll
    for (int j = 0; j < NL; ++j) gv[j] = 0.0;
  } else if (kd == kFacetInflow && !homog) {
#pragma unroll
    for (int j = 0; j < NL; ++j) gv[j] -= __ldg(&m.inflow_d[size_t(f) * NL + j]);
  }
}

// lam0 of one facet row (NL FP64 values at lam + o; the history vectors share its layout):
// with a history (SolveArgs::hist1, the same stage of earlier steps), the extrapolation
// c1 hist1 + c2 hist2 + c3 hist3, and the history moves down one slot (hist2 -> hist3 if
// hist3 is set, hist1 -> hist2; the caller then stores the new lam in hist1); without one,
// warm_scale lam (zero for a cold start).
template <int NL>
__device__ __forceinline__ void warm_start_row(double* lam, const SolveArgs& a, size_t o) {
  if (!a.hist1) {
#pragma unroll
    for (int j = 0; j < NL; ++j) lam[o + j] = a.warm_scale == 0.0 ? 0.0 : a.warm_scale * lam[o + j];
    return;
  }
  double* h1 = static_cast<double*>(a.hist1) + o;
  double* h2 = static_cast<double*>(a.hist2) + o;
  double* h3 = a.hist3 ? static_cast<double*>(a.hist3) + o : nullptr;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const double v1 = h1[j];
    const double v2 = (a.c2 != 0.0 || h3) ? h2[j] : 0.0;
    double v = a.c1 * v1;
    if (a.c2 != 0.0) v += a.c2 * v2;
    if (a.c3 != 0.0) v += a.c3 * h3[j];
    if (h3) h3[j] = v2;
    h2[j] = v1;
    lam[o + j] = v;
  }
}

template <int NL>
__device__ __forceinline__ void facet_nbrs(const DevMesh& m, int f, int (&nb)[5]) {
  nb[0] = f;
#pragma unroll
  for (int i = 0; i < 4; ++i) nb[i + 1] = __ldg(&m.facet_nbr[size_t(f) * 4 + i]);
}

// y_F = (S x)_F in FP64
template <int NL>
__device__ __forceinline__ void spmv64(const DevMesh& m, int f, const double* x, double (&y)[NL]) {
  int nb[5];
  facet_nbrs<NL>(m, f, nb);
  double xs[5][NL];
#pragma unroll
  for (int b = 0; b < 5; ++b)
#pragma unroll
    for (int j = 0; j < NL; ++j) xs[b][j] = __ldcg(&x[size_t(nb[b]) * NL + j]);
  stencil_rows<NL, double>(m.st_blk + size_t(__ldg(&m.facet_stencil[f])) * 5 * NL * NL, xs, y);
}

}  // namespace
}  // namespace dgdf
