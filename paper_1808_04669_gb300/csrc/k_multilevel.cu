// Facet-system solve with the multilevel preconditioner (multilevel.hpp): FP64
// PCG on S lam = g (the condensed system of eq. (12), Sec. 2.4), preconditioned
// by one V-cycle per iteration, in one persistent cooperative kernel.
//
// Every phase is a grid-stride loop over the rows of one level followed by a
// bounded grid barrier (solver_common.cuh). A V-cycle with L smoothing levels:
//   down, level l: [A] x = d + c1 d + c2 B (b - A d)  (d = c0 B b, set by the
//                  previous phase: the second Chebyshev step from x = 0)
//                  [B] r = b - A x; an injected transfer writes the next level's b
//                  (and its first Chebyshev step) in the same phase
//                  [C] a CSR transfer: b_next = R r (and its first step)
//   coarsest:      x_c = pinv b_c (added into the last level's mode 0 if it injects)
//   up, level l:   [U] a CSR transfer: x += P x_next
//                  [Q] r = b - A x, d = c0 B r
//                  [R] x += d + c1 d + c2 B (r - A d); an injected transfer adds x
//                  into the finer level's leading modes in the same phase
// so a level costs four or five barriers and the V-cycle is symmetric (the same
// Chebyshev polynomial before and after). The level records live in shared memory.
#include <type_traits>

#include "device.cuh"
#include "device3.cuh"
#include "kcommon.cuh"
#include "multilevel.hpp"
#include "solver_common.cuh"

namespace dgdf {

namespace {

constexpr int kMLThreads = 256;

// Operators of the V-cycle in its precision R: the facet stencil blocks and the coarsest
// pseudo-inverse and vectors.
template <typename R>
struct MLOps;
template <>
struct MLOps<double> {
  __device__ static const double* blocks(const DevMesh& m) { return m.st_blk; }
  __device__ static const MLLevelDev* levels(const DevMesh& m) { return m.ml_lv; }
  __device__ static const double* cpinv(const DevMesh& m) { return m.ml_cpinv; }
  __device__ static double* xc(const DevMesh& m) { return m.ml_xc; }
  __device__ static double* bc(const DevMesh& m) { return m.ml_bc; }
};
template <>
struct MLOps<float> {
  __device__ static const float* blocks(const DevMesh& m) { return m.st_blk_f; }
  __device__ static const MLLevelT<float>* levels(const DevMesh& m) { return m.ml_lv_f; }
  __device__ static const float* cpinv(const DevMesh& m) { return m.ml_cpinv_f; }
  __device__ static float* xc(const DevMesh& m) { return m.ml_xc_f; }
  __device__ static float* bc(const DevMesh& m) { return m.ml_bc_f; }
};

// Rows of a level in groups of G lanes of one warp, G = the largest power of two <= 32 with
// G n <= the grid's threads (one round of the grid covers every row whenever n allows): the
// lanes of a group split a row's sum (dot(i, lane, G), a strided partial sum) and add their
// partials by shuffles, then lane 0 of the group calls f(i, sum). Short coarse levels thus keep
// the grid busy instead of one thread walking a long row load by load. The loop bound and the
// shuffles are the same in every lane of a warp.
template <typename R, typename Dot, typename F>
__device__ __forceinline__ void rows_grouped(int n, Dot&& dot, F&& f) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  int G = 1;
  while (G < 32 && 2 * G * n <= gsz) G *= 2;
  const int lane = threadIdx.x & (G - 1), grp = gtid / G, ngrp = gsz / G;
  for (int i0 = 0; i0 < n; i0 += ngrp) {
    const int i = i0 + grp;
    R s = i < n ? dot(i, lane, G) : R(0);
    for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (i < n && lane == 0) f(i, s);
  }
}

// Strided partial sum of a CSR row: sum over p = rp[i] + lane, + G, ... of v[p] x[ci[p]]
template <typename R>
__device__ __forceinline__ R csr_part(const int32_t* rp, const int32_t* ci, const R* v, const R* x, int i, int lane,
                                      int G) {
  R s = R(0);
  const int p1 = __ldg(&rp[i + 1]);
#pragma unroll 4
  for (int p = __ldg(&rp[i]) + lane; p < p1; p += G) s += __ldg(&v[p]) * __ldcg(&x[__ldg(&ci[p])]);
  return s;
}

// y = (A x)_i for row i of a stencil level L (bs <= NL values)
template <int NL, typename R>
__device__ __forceinline__ void ml_row_apply(const DevMesh& m, const MLLevelT<R>& L, int i, const R* x,
                                             R (&y)[NL]) {
  if (L.st_nbr) {
    // the level's own stencil (all NL modes): slot 0 the row itself, then st_nnb neighbours
    const int nnb = L.st_nnb;
    const R* blk = L.st_blk + size_t(__ldg(&L.st_cls[i])) * (1 + nnb) * NL * NL;
#pragma unroll
    for (int ii = 0; ii < NL; ++ii) y[ii] = R(0);
    for (int b = 0; b <= nnb; ++b) {
      const int g = b == 0 ? i : __ldg(&L.st_nbr[size_t(i) * nnb + b - 1]);
      R xs[NL];
#pragma unroll
      for (int jj = 0; jj < NL; ++jj) xs[jj] = __ldcg(&x[size_t(g) * NL + jj]);
#pragma unroll
      for (int ii = 0; ii < NL; ++ii)
#pragma unroll
        for (int jj = 0; jj < NL; ++jj) y[ii] += __ldg(&blk[(b * NL + ii) * NL + jj]) * xs[jj];
    }
    return;
  }
  const int bs = L.bs;
  const R* blk = MLOps<R>::blocks(m) + size_t(__ldg(&m.facet_stencil[i])) * 5 * NL * NL;
  int nb[5];
  nb[0] = i;
#pragma unroll
  for (int b = 0; b < 4; ++b) nb[b + 1] = __ldg(&m.facet_nbr[size_t(i) * 4 + b]);
#pragma unroll
  for (int ii = 0; ii < NL; ++ii) {
    R v = R(0);
    if (ii < bs) {
#pragma unroll
      for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int jj = 0; jj < NL; ++jj)
          if (jj < bs) v += __ldg(&blk[(b * NL + ii) * NL + jj]) * __ldcg(&x[size_t(nb[b]) * bs + jj]);
    }
    y[ii] = v;
  }
}

// out = B v for row i of level L
template <int NL, typename R>
__device__ __forceinline__ void ml_row_binv(const DevMesh& m, const MLLevelT<R>& L, int i, const R (&v)[NL],
                                            R (&out)[NL]) {
  if (L.stencil) {
    const int bs = L.bs;
    const R* B = L.binv + size_t(__ldg(L.st_cls ? &L.st_cls[i] : &m.facet_stencil[i])) * bs * bs;
#pragma unroll
    for (int ii = 0; ii < NL; ++ii) {
      R s = R(0);
      if (ii < bs) {
#pragma unroll
        for (int jj = 0; jj < NL; ++jj)
          if (jj < bs) s += __ldg(&B[ii * bs + jj]) * v[jj];
      }
      out[ii] = s;
    }
  } else {
    out[0] = __ldg(&L.binv[i]) * v[0];
#pragma unroll
    for (int ii = 1; ii < NL; ++ii) out[ii] = R(0);
  }
}

// First Chebyshev step from zero on row i of level L: d = c0 B b, x = d.
template <int NL, typename R>
__device__ __forceinline__ void ml_row_first_step(const DevMesh& m, const MLLevelT<R>& L, int i) {
  const int bs = L.bs;
  R bv[NL], t[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) bv[j] = j < bs ? __ldcg(&L.b[size_t(i) * bs + j]) : R(0);
  ml_row_binv<NL, R>(m, L, i, bv, t);
#pragma unroll
  for (int j = 0; j < NL; ++j)
    if (j < bs) {
      const R d = L.c0 * t[j];
      L.d[size_t(i) * bs + j] = d;
      L.x[size_t(i) * bs + j] = d;
    }
}

// Level 0's input from the PCG residual r (facet f), then its first Chebyshev step. In FP64 the
// level's b is r itself; in FP32 it is r rounded.
template <int NL, typename R>
__device__ __forceinline__ void ml_start_row(const DevMesh& m, const MLLevelT<R>& L0, int f) {
  if constexpr (!std::is_same<R, double>::value) {
#pragma unroll
    for (int j = 0; j < NL; ++j) L0.b[size_t(f) * NL + j] = R(m.r[size_t(f) * NL + j]);
  }
  ml_row_first_step<NL, R>(m, L0, f);
}

// One V-cycle: on entry lv[0].b holds the input and lv[0].d = lv[0].x = c0 B b (set by the
// caller before a barrier, ml_start_row); on return every thread has written its rows of the
// output z (m.z: lv[0].x itself in FP64, its FP64 image in FP32) and accumulated, over its
// level-0 rows, r.z, r.r and the sum of r's mode 0 into red[0..2], with r the PCG residual
// m.r. The caller's reduction is the closing barrier.
template <int NL, typename R>
__device__ bool ml_vcycle(const DevMesh& m, const MLLevelT<R>* lv, double (&red)[3]) {
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  const int nlev = m.ml_nlev;
  GridBar* bar = m.bar;
  for (int l = 0; l < nlev; ++l) {
    const MLLevelT<R>& L = lv[l];
    const int bs = L.bs;
    // [A] second Chebyshev step from zero
    if (L.stencil) {
      for (int i = gtid; i < L.n; i += gsz) {
        R y[NL], res[NL], t[NL];
        ml_row_apply<NL, R>(m, L, i, L.d, y);
#pragma unroll
        for (int j = 0; j < NL; ++j) res[j] = j < bs ? __ldcg(&L.b[size_t(i) * bs + j]) - y[j] : R(0);
        ml_row_binv<NL, R>(m, L, i, res, t);
#pragma unroll
        for (int j = 0; j < NL; ++j)
          if (j < bs) {
            const R d = __ldcg(&L.d[size_t(i) * bs + j]);
            L.x[size_t(i) * bs + j] = d + L.c1 * d + L.c2 * t[j];
          }
      }
    } else {
      rows_grouped<R>(
          L.n, [&](int i, int lane, int G) { return csr_part<R>(L.a_rp, L.a_ci, L.a_v, L.d, i, lane, G); },
          [&](int i, R y) {
            const R t = __ldg(&L.binv[i]) * (__ldcg(&L.b[i]) - y);
            const R d = __ldcg(&L.d[i]);
            L.x[i] = d + L.c1 * d + L.c2 * t;
          });
    }
    if (!grid_sync(bar, m.stats)) return false;
    // [B] residual, injected restriction
    const bool last = l + 1 == nlev;
    if (L.stencil) {
      for (int i = gtid; i < L.n; i += gsz) {
        R y[NL];
        ml_row_apply<NL, R>(m, L, i, L.x, y);
#pragma unroll
        for (int j = 0; j < NL; ++j)
          if (j < bs) {
            const R r = __ldcg(&L.b[size_t(i) * bs + j]) - y[j];
            L.r[size_t(i) * bs + j] = r;
            if (L.inject && j < L.bs_next) {
              if (last) MLOps<R>::bc(m)[i] = r;   // bs_next = 1 into the coarsest level
              else lv[l + 1].b[size_t(i) * L.bs_next + j] = r;
            }
          }
        if (L.inject && !last) ml_row_first_step<NL, R>(m, lv[l + 1], i);
      }
    } else {
      // CSR levels hold one value per row and transfer through R (phase [C])
      rows_grouped<R>(
          L.n, [&](int i, int lane, int G) { return csr_part<R>(L.a_rp, L.a_ci, L.a_v, L.x, i, lane, G); },
          [&](int i, R y) { L.r[i] = __ldcg(&L.b[i]) - y; });
    }
    if (!grid_sync(bar, m.stats)) return false;
    if (!L.inject) {
      // [C] CSR restriction b_next = R r
      rows_grouped<R>(
          L.n_next, [&](int j, int lane, int G) { return csr_part<R>(L.r_rp, L.r_ci, L.r_v, L.r, j, lane, G); },
          [&](int j, R v) {
            if (last) {
              MLOps<R>::bc(m)[j] = v;
            } else {
              lv[l + 1].b[j] = v;
              ml_row_first_step<NL, R>(m, lv[l + 1], j);
            }
          });
      if (!grid_sync(bar, m.stats)) return false;
    }
  }
  // coarsest level: x_c = pinv b_c
  {
    const int nc = m.ml_nc;
    const MLLevelT<R>& Lz = lv[nlev - 1];
    const R* bc = MLOps<R>::bc(m);
    R* xc = MLOps<R>::xc(m);
    rows_grouped<R>(
        nc,
        [&](int i, int lane, int G) {
          R v = R(0);
          const R* row = MLOps<R>::cpinv(m) + size_t(i) * nc;
          for (int j = lane; j < nc; j += G) v += __ldg(&row[j]) * __ldcg(&bc[j]);
          return v;
        },
        [&](int i, R v) {
          xc[i] = v;
          if (Lz.inject) Lz.x[size_t(i) * Lz.bs] += v;
        });
    if (!grid_sync(bar, m.stats)) return false;
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const MLLevelT<R>& L = lv[l];
    const int bs = L.bs;
    if (!L.inject) {
      // [U] CSR prolongation x += P x_next
      const R* xn = (l + 1 == nlev) ? MLOps<R>::xc(m) : lv[l + 1].x;
      rows_grouped<R>(
          L.n, [&](int i, int lane, int G) { return csr_part<R>(L.p_rp, L.p_ci, L.p_v, xn, i, lane, G); },
          [&](int i, R v) { L.x[i] += v; });
      if (!grid_sync(bar, m.stats)) return false;
    }
    // [Q] r = b - A x, d = c0 B r
    if (L.stencil) {
      for (int i = gtid; i < L.n; i += gsz) {
        R y[NL], res[NL], t[NL];
        ml_row_apply<NL, R>(m, L, i, L.x, y);
#pragma unroll
        for (int j = 0; j < NL; ++j) res[j] = j < bs ? __ldcg(&L.b[size_t(i) * bs + j]) - y[j] : R(0);
        ml_row_binv<NL, R>(m, L, i, res, t);
#pragma unroll
        for (int j = 0; j < NL; ++j)
          if (j < bs) {
            L.r[size_t(i) * bs + j] = res[j];
            L.d[size_t(i) * bs + j] = L.c0 * t[j];
          }
      }
    } else {
      rows_grouped<R>(
          L.n, [&](int i, int lane, int G) { return csr_part<R>(L.a_rp, L.a_ci, L.a_v, L.x, i, lane, G); },
          [&](int i, R y) {
            const R res = __ldcg(&L.b[i]) - y;
            L.r[i] = res;
            L.d[i] = L.c0 * (__ldg(&L.binv[i]) * res);
          });
    }
    if (!grid_sync(bar, m.stats)) return false;
    // [R] x += d + c1 d + c2 B (r - A d); inject into the finer level (same facet rows)
    const MLLevelT<R>* F = l > 0 && lv[l - 1].inject ? &lv[l - 1] : nullptr;
    if (!L.stencil) {
      // a CSR level; below an injecting level its rows are the finer level's rows (faces) and its
      // result goes into their mode 0. Level 0 of an assembled hierarchy is CSR too, with one
      // row per face mode: it writes the output z and accumulates the PCG scalars
      const int modes = L.modes > 1 ? L.modes : 1;
      double part[3] = {0.0, 0.0, 0.0};
      rows_grouped<R>(
          L.n, [&](int i, int lane, int G) { return csr_part<R>(L.a_rp, L.a_ci, L.a_v, L.d, i, lane, G); },
          [&](int i, R y) {
            const R t = __ldg(&L.binv[i]) * (__ldcg(&L.r[i]) - y);
            const R d = __ldcg(&L.d[i]);
            const R x = __ldcg(&L.x[i]) + d + L.c1 * d + L.c2 * t;
            L.x[i] = x;
            if (F) F->x[size_t(i) * F->bs] += x;   // injected into the finer level's mode 0
            if (l == 0) {
              const double z = double(x);
              if constexpr (!std::is_same<R, double>::value) m.z[i] = z;
              const double b = __ldcg(&m.r[i]);
              part[0] += b * z;
              part[1] += b * b;
              if (i % modes == 0) part[2] += b;
            }
          });
      if (l == 0) {
#pragma unroll
        for (int j = 0; j < 3; ++j) red[j] += part[j];
        continue;   // the caller's reduction is the closing barrier
      }
      if (!grid_sync(bar, m.stats)) return false;
      continue;
    }
    for (int i = gtid; i < L.n; i += gsz) {
      R y[NL], res[NL], t[NL];
      ml_row_apply<NL, R>(m, L, i, L.d, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) res[j] = j < bs ? __ldcg(&L.r[size_t(i) * bs + j]) - y[j] : R(0);
      ml_row_binv<NL, R>(m, L, i, res, t);
#pragma unroll
      for (int j = 0; j < NL; ++j)
        if (j < bs) {
          const R d = __ldcg(&L.d[size_t(i) * bs + j]);
          const R x = __ldcg(&L.x[size_t(i) * bs + j]) + d + L.c1 * d + L.c2 * t[j];
          L.x[size_t(i) * bs + j] = x;
          if (F) F->x[size_t(i) * F->bs + j] += x;
          if (l == 0) {
            // the output z and the PCG scalars, against the FP64 residual
            const double z = double(x);
            if constexpr (!std::is_same<R, double>::value) m.z[size_t(i) * bs + j] = z;
            const double b = __ldcg(&m.r[size_t(i) * bs + j]);
            red[0] += b * z;
            red[1] += b * b;
            if (j == 0) red[2] += b;
          }
        }
    }
    if (l > 0 && !grid_sync(bar, m.stats)) return false;
  }
  return true;
}

// One solve: g assembled from the element sides, lam0 from the history or warm_scale * lam
// (warm_start_row), constant multiplier removed from g, then PCG with the V-cycle. Level 0's b and x are the PCG vectors r and z.
template <int K, typename R>
__global__ void __launch_bounds__(kMLThreads) k_solve_ml(DevMesh m, SolveArgs a) {
  constexpr int NL = K + 1;
  __shared__ MLLevelT<R> lv[kMLMaxLevels];
  for (int l = threadIdx.x; l < m.ml_nlev; l += blockDim.x) lv[l] = MLOps<R>::levels(m)[l];
  __syncthreads();
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = m.bar;
  double gg[2] = {0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz) {
    double gv[NL];
    assemble_g<NL>(m, f, gv);
    boundary_g<NL>(m, f, a.homog, gv);
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const size_t o = size_t(f) * NL + j;
      m.g[o] = gv[j];
      gg[0] += gv[j] * gv[j];
    }
    warm_start_row<NL>(m.lam, a, size_t(f) * NL);
    gg[1] += gv[0];
  }
  if (!grid_reduce<2>(m, 4, gg, bar)) return;
  // with outflow facets S is definite: no constant component to remove (inv_nf = 0)
  const double inv_nf = m.has_kernel ? 1.0 / double(nF) : 0.0;
  const double c0 = gg[1] * inv_nf;
  const double gnorm = sqrt(fmax(gg[0] - gg[1] * gg[1] * inv_nf, 0.0));
  const double stop = a.rtol * gnorm;
  int it = 0;
  bool conv = false;
  double rr = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz)
#pragma unroll
      for (int j = 0; j < NL; ++j) m.lam[size_t(f) * NL + j] = 0.0;
    conv = true;
  } else {
    // The V-cycle, unlike S, does not annihilate the constant multiplier (mode 0 = 1 on every
    // facet, the kernel of S), and it amplifies that direction by about 1 / lambda_min(S):
    // rounding that leaves a constant component in r would soon dominate z. So r is kept in the
    // range of S: its mode-0 mean is subtracted before every V-cycle (the sum is carried along
    // the updates: sum r_new = sum r_old - alpha sum q).
    for (int f = gtid; f < nF; f += gsz) m.g[size_t(f) * NL] -= c0;
    if (!grid_sync(bar, m.stats)) return;
    // r = g - S lam, and its mode-0 sum
    double r0s[1] = {0.0};
    for (int f = gtid; f < nF; f += gsz) {
      double y[NL];
      spmv64<NL>(m, f, m.lam, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) m.r[size_t(f) * NL + j] = m.g[size_t(f) * NL + j] - y[j];
      r0s[0] += m.r[size_t(f) * NL];
    }
    if (!grid_reduce<1>(m, 0, r0s, bar)) return;
    // remove the constant component; first Chebyshev step of the V-cycle on r
    for (int f = gtid; f < nF; f += gsz) {
      m.r[size_t(f) * NL] -= r0s[0] * inv_nf;
      ml_start_row<NL, R>(m, lv[0], f);
    }
    if (!grid_sync(bar, m.stats)) return;
    double red[3] = {0.0, 0.0, 0.0};
    if (!ml_vcycle<NL, R>(m, lv, red)) return;
    if (!grid_reduce<3>(m, 1, red, bar)) return;
    double rho = red[0];
    rr = fmax(red[1] - red[2] * red[2] * inv_nf, 0.0);
    double rsum = red[2];   // mode-0 sum of r as the V-cycle saw it
    double beta = 0.0;
    double* pold = m.pa;
    double* pnew = m.pb;
    // rounding floor: once 10 iterations in a row fail to halve the best residual, the solve
    // ends, converged if that residual is below floor_rtol (as in the other solvers)
    double best = rr;
    int stall = 0;
    for (;; ++it) {
      if (!isfinite(rr) || !isfinite(rho)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      if (sqrt(rr) <= stop) {
        conv = true;
        break;
      }
      if (rr < 0.25 * best) {
        best = rr;
        stall = 0;
      } else if (++stall >= 10) {
        conv = sqrt(best) <= a.floor_rtol * gnorm;
        break;
      }
      if (it >= a.maxit) break;
      // p_new = z + beta p_old, q = S p_new; reduce p.q and the mode-0 sum of q
      double pq[2] = {0.0, 0.0};
      for (int f = gtid; f < nF; f += gsz) {
        int nb[5];
        facet_nbrs<NL>(m, f, nb);
        double xs[5][NL];
#pragma unroll
        for (int b = 0; b < 5; ++b)
#pragma unroll
          for (int j = 0; j < NL; ++j) {
            const size_t o = size_t(nb[b]) * NL + j;
            xs[b][j] = (it == 0) ? __ldcg(&m.z[o]) : __ldcg(&m.z[o]) + beta * __ldcg(&pold[o]);
          }
        double y[NL];
        stencil_rows<NL, double>(m.st_blk + size_t(__ldg(&m.facet_stencil[f])) * 5 * NL * NL, xs, y);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          pnew[size_t(f) * NL + j] = xs[0][j];
          m.q[size_t(f) * NL + j] = y[j];
          pq[0] += xs[0][j] * y[j];
        }
        pq[1] += y[0];
      }
      if (!grid_reduce<2>(m, 6, pq, bar)) return;
      if (!(pq[0] > 0.0)) {
        if (!isfinite(pq[0]) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        if (m.ml_hist && blockIdx.x == 0 && threadIdx.x == 0 && it < kMLHist) {
          m.ml_hist[4 * it + 0] = sqrt(rr) / gnorm;
          m.ml_hist[4 * it + 1] = rho;
          m.ml_hist[4 * it + 2] = pq[0];
          m.ml_hist[4 * it + 3] = -1.0;
        }
        break;
      }
      const double alpha = rho / pq[0];
      if (m.ml_hist && blockIdx.x == 0 && threadIdx.x == 0 && it < kMLHist) {
        m.ml_hist[4 * it + 0] = sqrt(rr) / gnorm;
        m.ml_hist[4 * it + 1] = rho;
        m.ml_hist[4 * it + 2] = pq[0];
        m.ml_hist[4 * it + 3] = alpha;
      }
      // lam += alpha p, r -= alpha q minus its constant component, first Chebyshev step on r
      const double cmean = (rsum - alpha * pq[1]) * inv_nf;
      for (int f = gtid; f < nF; f += gsz) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          m.lam[o] += alpha * pnew[o];
          m.r[o] -= alpha * m.q[o] + (j == 0 ? cmean : 0.0);
        }
        ml_start_row<NL, R>(m, lv[0], f);
      }
      if (!grid_sync(bar, m.stats)) return;
      double red2[3] = {0.0, 0.0, 0.0};
      if (!ml_vcycle<NL, R>(m, lv, red2)) return;
      if (!grid_reduce<3>(m, 1, red2, bar)) return;
      beta = red2[0] / rho;
      rho = red2[0];
      rr = fmax(red2[1] - red2[2] * red2[2] * inv_nf, 0.0);
      rsum = red2[2];
      double* t = pold;
      pold = pnew;
      pnew = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats* st = m.stats;
    st->last_iters = it;
    st->total_iters += it;
    st->solves += 1;
    st->last_relres = gnorm > 0.0 ? sqrt(rr) / gnorm : 0.0;
    st->last_sweeps = 1;
    st->total_sweeps += 1;
    if (!conv) atomicOr(&st->flags, kFlagNotConverged);
  }
}

// y = (S x)_f on the face stencil of the three-dimensional path (seven blocks), with
// x = a + beta b (b NULL: x = a)
template <int NL>
__device__ __forceinline__ void spmv3_ml(const DevMesh3& m3, int f, const double* a, const double* b, double beta,
                                         double (&y)[NL]) {
  const double* blk = m3.st_blk + size_t(__ldg(&m3.face_stencil[f])) * 7 * NL * NL;
#pragma unroll
  for (int i = 0; i < NL; ++i) y[i] = 0.0;
#pragma unroll
  for (int s = 0; s < 7; ++s) {
    const int g = s == 0 ? f : __ldg(&m3.face_nbr[size_t(f) * 6 + s - 1]);
    double xs[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const size_t o = size_t(g) * NL + j;
      xs[j] = b ? __ldcg(&a[o]) + beta * __ldcg(&b[o]) : __ldcg(&a[o]);
    }
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int j = 0; j < NL; ++j) y[i] += __ldg(&blk[(s * NL + i) * NL + j]) * xs[j];
  }
}

// Face-system solve of the three-dimensional path with the multilevel preconditioner of an
// assembled hierarchy (multilevel.hpp, build_multilevel_csr): FP64 PCG as in k_solve_ml, with
// the face stencil of m3 (seven blocks) for S and g assembled from both sides' G f (canonical
// face basis: no orientation signs). mv carries the hierarchy and the PCG vectors r and z, the
// reduction slots, the barrier and the counters (the same buffers as m3's).
template <int K, typename R>
__global__ void __launch_bounds__(kMLThreads) k_solve3_ml(DevMesh3 m3, DevMesh mv, SolveArgs a) {
  constexpr int NL = (K + 1) * (K + 2) / 2, L4 = 4 * NL;
  __shared__ MLLevelT<R> lv[kMLMaxLevels];
  for (int l = threadIdx.x; l < mv.ml_nlev; l += blockDim.x) lv[l] = MLOps<R>::levels(mv)[l];
  __syncthreads();
  const int nF = m3.n_face;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = mv.bar;
  double gg[2] = {0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz) {
    const int t0 = m3.face_tet[size_t(f) * 2], t1 = m3.face_tet[size_t(f) * 2 + 1];
    const int e0 = m3.face_loc[size_t(f) * 2], e1 = m3.face_loc[size_t(f) * 2 + 1];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const double v = m3.gl[size_t(t0) * L4 + e0 * NL + j] + m3.gl[size_t(t1) * L4 + e1 * NL + j];
      const size_t o = size_t(f) * NL + j;
      m3.g[o] = v;
      gg[0] += v * v;
      if (j == 0) gg[1] += v;
    }
    warm_start_row<NL>(m3.lam, a, size_t(f) * NL);
  }
  if (!grid_reduce<2>(mv, 4, gg, bar)) return;
  const double inv_nf = 1.0 / double(nF);   // closed mesh: the constant multiplier is the kernel of S
  const double c0 = gg[1] * inv_nf;
  const double gnorm = sqrt(fmax(gg[0] - gg[1] * gg[1] * inv_nf, 0.0));
  const double stop = a.rtol * gnorm;
  int it = 0;
  bool conv = false;
  double rr = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz)
#pragma unroll
      for (int j = 0; j < NL; ++j) m3.lam[size_t(f) * NL + j] = 0.0;
    conv = true;
  } else {
    // r = g - c0 1 - S lam, kept in the range of S (its mode-0 mean removed before every
    // V-cycle, as in k_solve_ml), then the first Chebyshev step on every row of level 0
    for (int f = gtid; f < nF; f += gsz) m3.g[size_t(f) * NL] -= c0;
    if (!grid_sync(bar, mv.stats)) return;
    double r0s[1] = {0.0};
    for (int f = gtid; f < nF; f += gsz) {
      double y[NL];
      spmv3_ml<NL>(m3, f, m3.lam, nullptr, 0.0, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) mv.r[size_t(f) * NL + j] = m3.g[size_t(f) * NL + j] - y[j];
      r0s[0] += mv.r[size_t(f) * NL];
    }
    if (!grid_reduce<1>(mv, 0, r0s, bar)) return;
    for (int f = gtid; f < nF; f += gsz) {
      mv.r[size_t(f) * NL] -= r0s[0] * inv_nf;
      ml_start_row<NL, R>(mv, lv[0], f);
    }
    if (!grid_sync(bar, mv.stats)) return;
    double red[3] = {0.0, 0.0, 0.0};
    if (!ml_vcycle<NL, R>(mv, lv, red)) return;
    if (!grid_reduce<3>(mv, 1, red, bar)) return;
    double rho = red[0];
    rr = fmax(red[1] - red[2] * red[2] * inv_nf, 0.0);
    double rsum = red[2];
    double beta = 0.0;
    double* pold = m3.pa;
    double* pnew = m3.pb;
    double best = rr;
    int stall = 0;
    for (;; ++it) {
      if (!isfinite(rr) || !isfinite(rho)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&mv.stats->flags, kFlagNonFinite);
        break;
      }
      if (sqrt(rr) <= stop) {
        conv = true;
        break;
      }
      if (rr < 0.25 * best) {
        best = rr;
        stall = 0;
      } else if (++stall >= 10) {
        conv = sqrt(best) <= a.floor_rtol * gnorm;
        break;
      }
      if (it >= a.maxit) break;
      // p_new = z + beta p_old, q = S p_new; reduce p.q and the mode-0 sum of q
      double pq[2] = {0.0, 0.0};
      for (int f = gtid; f < nF; f += gsz) {
        double y[NL];
        spmv3_ml<NL>(m3, f, mv.z, it == 0 ? nullptr : pold, beta, y);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          const double p = it == 0 ? __ldcg(&mv.z[o]) : __ldcg(&mv.z[o]) + beta * __ldcg(&pold[o]);
          pnew[o] = p;
          m3.q[o] = y[j];
          pq[0] += p * y[j];
        }
        pq[1] += y[0];
      }
      if (!grid_reduce<2>(mv, 6, pq, bar)) return;
      if (!(pq[0] > 0.0)) {
        if (!isfinite(pq[0]) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&mv.stats->flags, kFlagNonFinite);
        break;
      }
      const double alpha = rho / pq[0];
      const double cmean = (rsum - alpha * pq[1]) * inv_nf;
      for (int f = gtid; f < nF; f += gsz) {
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          m3.lam[o] += alpha * pnew[o];
          mv.r[o] -= alpha * m3.q[o] + (j == 0 ? cmean : 0.0);
        }
        ml_start_row<NL, R>(mv, lv[0], f);
      }
      if (!grid_sync(bar, mv.stats)) return;
      double red2[3] = {0.0, 0.0, 0.0};
      if (!ml_vcycle<NL, R>(mv, lv, red2)) return;
      if (!grid_reduce<3>(mv, 1, red2, bar)) return;
      beta = red2[0] / rho;
      rho = red2[0];
      rr = fmax(red2[1] - red2[2] * red2[2] * inv_nf, 0.0);
      rsum = red2[2];
      double* t = pold;
      pold = pnew;
      pnew = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats* st = mv.stats;
    st->last_iters = it;
    st->total_iters += it;
    st->solves += 1;
    st->last_relres = gnorm > 0.0 ? sqrt(rr) / gnorm : 0.0;
    st->last_sweeps = 1;
    st->total_sweeps += 1;
    if (!conv) atomicOr(&st->flags, kFlagNotConverged);
  }
}

// One V-cycle z = M r on its own (test hook dg_test_multilevel_apply): r and z are facet-major
// [n_facet][k+1] in device memory. Uses the solver's level-0 vectors m.r and m.z.
template <int K, typename R>
__global__ void __launch_bounds__(kMLThreads) k_ml_apply(DevMesh m, const double* rin, double* zout) {
  constexpr int NL = K + 1;
  __shared__ MLLevelT<R> lv[kMLMaxLevels];
  for (int l = threadIdx.x; l < m.ml_nlev; l += blockDim.x) lv[l] = MLOps<R>::levels(m)[l];
  __syncthreads();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  for (int f = gtid; f < m.n_facet; f += gsz) {
#pragma unroll
    for (int j = 0; j < NL; ++j) m.r[size_t(f) * NL + j] = rin[size_t(f) * NL + j];
    ml_start_row<NL, R>(m, lv[0], f);
  }
  if (!grid_sync(m.bar, m.stats)) return;
  double red[3] = {0.0, 0.0, 0.0};
  if (!ml_vcycle<NL, R>(m, lv, red)) return;
  for (int f = gtid; f < m.n_facet; f += gsz)
#pragma unroll
    for (int j = 0; j < NL; ++j) zout[size_t(f) * NL + j] = m.z[size_t(f) * NL + j];
}

const void* ml_kernel(int k, bool fp32) {
  switch (k * 2 + (fp32 ? 1 : 0)) {
    case 2: return (const void*)k_solve_ml<1, double>;
    case 3: return (const void*)k_solve_ml<1, float>;
    case 4: return (const void*)k_solve_ml<2, double>;
    case 5: return (const void*)k_solve_ml<2, float>;
    case 6: return (const void*)k_solve_ml<3, double>;
    case 7: return (const void*)k_solve_ml<3, float>;
    default: return nullptr;
  }
}

}  // namespace

cudaError_t launch_ml_apply(const DevMesh& m, const double* r, double* z, int nblocks, cudaStream_t s) {
  const bool fp32 = m.ml_lv_f != nullptr;
  if ((!m.ml_lv && !fp32) || m.ml_nlev < 1 || m.ml_nlev > kMLMaxLevels) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  const void* fn = nullptr;
  switch (m.k * 2 + (fp32 ? 1 : 0)) {
    case 2: fn = (const void*)k_ml_apply<1, double>; break;
    case 3: fn = (const void*)k_ml_apply<1, float>; break;
    case 4: fn = (const void*)k_ml_apply<2, double>; break;
    case 5: fn = (const void*)k_ml_apply<2, float>; break;
    case 6: fn = (const void*)k_ml_apply<3, double>; break;
    case 7: fn = (const void*)k_ml_apply<3, float>; break;
    default: return cudaErrorInvalidValue;
  }
  DevMesh mm = m;
  void* args[] = {&mm, (void*)&r, (void*)&z};
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kMLThreads), args, 0, s);
}

int solver_ml_blocks(const DevMesh& m) {
  const void* fn = ml_kernel(m.k, m.ml_lv_f != nullptr);
  if (!fn) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMLThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = per_sm * sms;
  if (nb > 2 * sms) nb = 2 * sms;   // fewer blocks make the many grid barriers cheaper
  const int need = (m.n_facet + kMLThreads - 1) / kMLThreads;
  if (nb > need) nb = need;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  return nb < 1 ? 1 : nb;
}

const void* ml3_kernel(int k, bool fp32) {
  switch (k * 2 + (fp32 ? 1 : 0)) {
    case 2: return (const void*)k_solve3_ml<1, double>;
    case 3: return (const void*)k_solve3_ml<1, float>;
    case 4: return (const void*)k_solve3_ml<2, double>;
    case 5: return (const void*)k_solve3_ml<2, float>;
    default: return nullptr;
  }
}

int solver3_ml_blocks(const DevMesh3& m, bool fp32) {
  const void* fn = ml3_kernel(m.k, fp32);
  if (!fn) return 0;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMLThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = per_sm * sms;
  if (nb > 2 * sms) nb = 2 * sms;
  const int need = (m.n_face * ((m.k + 1) * (m.k + 2) / 2) + kMLThreads - 1) / kMLThreads;
  if (nb > need) nb = need;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  return nb < 1 ? 1 : nb;
}

cudaError_t launch_solve3_ml(const DevMesh3& m, const DevMesh& mv, const SolveArgs& a, int nblocks, cudaStream_t s) {
  const bool fp32 = mv.ml_lv_f != nullptr;
  const void* fn = ml3_kernel(m.k, fp32);
  if ((!mv.ml_lv && !fp32) || mv.ml_nlev < 1 || mv.ml_nlev > kMLMaxLevels || !fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(mv.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  DevMesh3 mm = m;
  DevMesh vv = mv;
  SolveArgs aa = a;
  void* args[] = {&mm, &vv, &aa};
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kMLThreads), args, 0, s);
}

cudaError_t launch_solve_ml(const DevMesh& m, const SolveArgs& a, int nblocks, cudaStream_t s) {
  const bool fp32 = m.ml_lv_f != nullptr;
  if ((!m.ml_lv && !fp32) || m.ml_nlev < 1 || m.ml_nlev > kMLMaxLevels) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  const void* fn = ml_kernel(m.k, fp32);
  if (!fn) return cudaErrorInvalidValue;
  DevMesh mm = m;
  SolveArgs aa = a;
  void* args[] = {&mm, &aa};
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kMLThreads), args, 0, s);
}

}  // namespace dgdf
