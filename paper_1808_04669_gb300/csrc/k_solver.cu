// Facet-system solve of the hybrid-mixed scheme (eq. (12) after static
// condensation; SPD up to the constant multiplier, Sec. 2.4): one persistent
// cooperative kernel per solve running preconditioned CG with block-Jacobi
// (one (k+1) x (k+1) block per facet).
//
// Matrix-free stencil: row F of S couples F to the other two facets of each
// adjacent triangle; rows with equal blocks share one stencil class, so on a
// translation-invariant mesh the operator is a handful of small blocks held in
// L1 and the SpMV streams only the vectors and 4 neighbour indices per facet.
//
// FP64 form: CG in FP64. Mixed form: FP64 iterative refinement
// (r = g - S lam in FP64) around an inner CG in FP32 on S d = r.
//
// Each CG iteration has two grid-wide reductions; the direction update
// p = z + beta p is fused into the next SpMV (two p buffers), so every
// iteration costs two grid barriers. Reductions sum block partials in a fixed
// order, so results are bitwise reproducible for a given launch shape.
#include <atomic>

#include "device.cuh"
#include "kcommon.cuh"
#include "solver_common.cuh"

namespace dgdf {

namespace {

// Preconditioned CG on S x = b (precision R) starting from x = 0; b is given
// through the initial residual already stored in rv. Vectors: x, r, z, pa/pb
// (two direction buffers), q. Returns iterations; sets *conv.
template <int NL, typename R>
__device__ int pcg(const DevMesh& m, R* x, R* rv, R* zv, R* pa, R* pb, R* qv, const R* blk_all, const R* binv_all,
                   double stop_abs, int maxit, bool x_zero, GridBar* bar, bool* conv, double* rr_out) {
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  // z = B r, rho = r.z, rr = r.r ; x = 0 if requested. The residual norm used for
  // stopping leaves out the component along the kernel of S (mode 0 = 1 on every
  // facet), which CG cannot reduce and which rounding puts into r (none with outflow
  // facets: S is then definite).
  const double inv_nf = m.has_kernel ? 1.0 / double(nF) : 0.0;
  double red[3] = {0.0, 0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz) {
    R r[NL], z[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) r[j] = rv[size_t(f) * NL + j];
    block_apply<NL, R>(binv_all + size_t(__ldg(&m.facet_stencil[f])) * NL * NL, r, z);
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      zv[size_t(f) * NL + j] = z[j];
      if (x_zero) x[size_t(f) * NL + j] = R(0);
      red[0] += double(r[j]) * double(z[j]);
      red[1] += double(r[j]) * double(r[j]);
    }
    red[2] += double(r[0]);
  }
  if (!grid_reduce<3>(m, 1, red, bar)) return 0;
  double rho = red[0], rr = fmax(red[1] - red[2] * red[2] * inv_nf, 0.0);
  double beta = 0.0;
  R* pold = pa;
  R* pnew = pb;
  int it = 0;
  *conv = false;
  for (; it <= maxit; ++it) {
    if (!isfinite(rr) || !isfinite(rho)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
      break;
    }
    if (sqrt(rr) <= stop_abs) {
      *conv = true;
      break;
    }
    if (it == maxit) break;
    // p_new = z + beta p_old (own rows), q = S p_new (from the neighbours' z, p_old)
    const R rb = R(beta);
    double pq[1] = {0.0};
    for (int f = gtid; f < nF; f += gsz) {
      int nb[5];
      facet_nbrs<NL>(m, f, nb);
      R xs[5][NL];
#pragma unroll
      for (int b = 0; b < 5; ++b)
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(nb[b]) * NL + j;
          xs[b][j] = (it == 0) ? __ldcg(&zv[o]) : __ldcg(&zv[o]) + rb * __ldcg(&pold[o]);
        }
      R y[NL];
      stencil_rows<NL, R>(blk_all + size_t(__ldg(&m.facet_stencil[f])) * 5 * NL * NL, xs, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        pnew[size_t(f) * NL + j] = xs[0][j];
        qv[size_t(f) * NL + j] = y[j];
        pq[0] += double(xs[0][j]) * double(y[j]);
      }
    }
    if (!grid_reduce<1>(m, 0, pq, bar)) return it;
    if (!(pq[0] > 0.0)) {
      if (!isfinite(pq[0]) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
      break;
    }
    const double alpha = rho / pq[0];
    const R ra = R(alpha);
    double red2[3] = {0.0, 0.0, 0.0};
    for (int f = gtid; f < nF; f += gsz) {
      R r[NL], z[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const size_t o = size_t(f) * NL + j;
        x[o] += ra * pnew[o];
        r[j] = rv[o] - ra * qv[o];
        rv[o] = r[j];
      }
      block_apply<NL, R>(binv_all + size_t(__ldg(&m.facet_stencil[f])) * NL * NL, r, z);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        zv[size_t(f) * NL + j] = z[j];
        red2[0] += double(r[j]) * double(z[j]);
        red2[1] += double(r[j]) * double(r[j]);
      }
      red2[2] += double(r[0]);
    }
    if (!grid_reduce<3>(m, 1, red2, bar)) return it + 1;
    beta = red2[0] / rho;
    rho = red2[0];
    rr = fmax(red2[1] - red2[2] * red2[2] * inv_nf, 0.0);
    R* t = pold;
    pold = pnew;
    pnew = t;
  }
  *rr_out = rr;
  return it;
}

// One solve: g = assembled element contributions, lam0 from the history or warm_scale * lam
// (warm_start_row), then FP64 PCG (mixed = 0) or FP64 refinement around FP32 PCG (mixed = 1).
template <int K, int MIXED>
__global__ void __launch_bounds__(kSolverThreads) k_solve(DevMesh m, SolveArgs a) {
  constexpr int NL = K + 1;
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = m.bar;
  // g_F = sum over both sides of the side's contribution mapped to canonical orientation
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
  // project g onto the range of S: remove its component along the constant multiplier
  const double inv_nf = m.has_kernel ? 1.0 / double(nF) : 0.0;
  const double c0 = gg[1] * inv_nf;
  if (c0 != 0.0)
    for (int f = gtid; f < nF; f += gsz) m.g[size_t(f) * NL] -= c0;
  const double gnorm = sqrt(fmax(gg[0] - gg[1] * gg[1] * inv_nf, 0.0));
  const double stop = a.rtol * gnorm;
  int iters = 0, sweeps = 0;
  bool conv = false;
  double relres = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz)
#pragma unroll
      for (int j = 0; j < NL; ++j) m.lam[size_t(f) * NL + j] = 0.0;
    conv = true;
  } else {
    // residual r = g - S lam (lam from the first loop: visible after the barrier)
    for (int sweep = 0;; ++sweep) {
      double rr[2] = {0.0, 0.0};
      for (int f = gtid; f < nF; f += gsz) {
        double y[NL];
        spmv64<NL>(m, f, m.lam, y);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          const double r = m.g[o] - y[j];
          if (MIXED) m.rf[o] = float(r);
          else m.r[o] = r;
          rr[0] += r * r;
          if (j == 0) rr[1] += r;
        }
      }
      if (!MIXED) {
        // FP64 CG directly on S d = r with lam as the iterate (no refinement needed)
        bool c = false;
        double rr_end = 0.0;
        if (!grid_sync(bar, m.stats)) return;
        iters = pcg<NL, double>(m, m.lam, m.r, m.z, m.pa, m.pb, m.q, m.st_blk, m.st_binv, stop, a.maxit, false, bar,
                                &c, &rr_end);
        conv = c;
        relres = sqrt(rr_end) / gnorm;
        sweeps = 1;
        break;
      }
      if (!grid_reduce<2>(m, 6, rr, bar)) return;
      rr[0] = fmax(rr[0] - rr[1] * rr[1] * inv_nf, 0.0);
      const double prev = relres;
      relres = sqrt(rr[0]) / gnorm;
      if (!isfinite(rr[0])) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      if (sqrt(rr[0]) <= stop) {
        conv = true;
        break;
      }
      // The FP64 residual g - S lam has a rounding floor of about eps64 * cond(S); once a
      // sweep no longer halves it, the solve is at that floor.
      if (sweep >= 2 && relres > 0.5 * prev) {
        conv = relres <= a.floor_rtol;
        break;
      }
      if (sweep >= a.max_sweeps || iters >= a.maxit) break;
      // inner FP32 solve of S d = r to inner_rtol relative, d in xf
      bool c = false;
      double rr_end = 0.0;
      const double inner_stop = fmax(a.inner_rtol * sqrt(rr[0]), 0.5 * stop);
      const int budget = min(a.inner_maxit, a.maxit - iters);
      const int it = pcg<NL, float>(m, m.xf, m.rf, m.zf, m.paf, m.pbf, m.qf, m.st_blk_f, m.st_binv_f, inner_stop,
                                    budget, true, bar, &c, &rr_end);
      iters += it;
      ++sweeps;
      // lam += d
      for (int f = gtid; f < nF; f += gsz)
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          m.lam[o] += double(m.xf[o]);
        }
      if (!grid_sync(bar, m.stats)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DevStats* st = m.stats;
    st->last_iters = iters;
    st->total_iters += iters;
    st->solves += 1;
    st->last_relres = relres;
    st->last_sweeps = sweeps;
    st->total_sweeps += sweeps;
    if (!conv) atomicOr(&st->flags, kFlagNotConverged);
  }
}

template <int K, int MIXED>
int max_blocks_for() {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<K, MIXED>, kSolverThreads, 0);
  return per_sm * sms;
}

}  // namespace

int solver_max_blocks(const DevMesh& m, int mixed) {
  int nb = 0;
  switch (m.k * 2 + (mixed ? 1 : 0)) {
    case 2: nb = max_blocks_for<1, 0>(); break;
    case 3: nb = max_blocks_for<1, 1>(); break;
    case 4: nb = max_blocks_for<2, 0>(); break;
    case 5: nb = max_blocks_for<2, 1>(); break;
    case 6: nb = max_blocks_for<3, 0>(); break;
    case 7: nb = max_blocks_for<3, 1>(); break;
    default: nb = 0;
  }
  // at most two co-resident blocks per SM: fewer blocks make the grid barriers and the
  // fixed-order reductions cheaper; each thread then loops over a few facets
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nb > 2 * sms) nb = 2 * sms;
  const int need = (m.n_facet + kSolverThreads - 1) / kSolverThreads;
  if (nb > need) nb = need;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  if (nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_solve(const DevMesh& m, const SolveArgs& a, int nblocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  DevMesh mm = m;
  SolveArgs aa = a;
  void* args[] = {&mm, &aa};
  const void* fn = nullptr;
  switch (m.k * 2 + (a.mixed ? 1 : 0)) {
    case 2: fn = (const void*)k_solve<1, 0>; break;
    case 3: fn = (const void*)k_solve<1, 1>; break;
    case 4: fn = (const void*)k_solve<2, 0>; break;
    case 5: fn = (const void*)k_solve<2, 1>; break;
    case 6: fn = (const void*)k_solve<3, 0>; break;
    case 7: fn = (const void*)k_solve<3, 1>; break;
    default: return cudaErrorInvalidValue;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kSolverThreads), args, 0, s);
}

// ---------------------------------------------------------------------------
// Facet solve without allocation (dg_facet_solve_noalloc in include/dgdf.h).
//
// Same FP64 PCG as k_solve<K, 0>, but the caller passes the facet operator, g
// and lam in memory it owns, and every work vector, the reduction slots, the
// grid barrier and the counters live in the file-scope array below, so the
// call makes no allocation. The array (kNoAllocDofs multiplier DOFs, about
// 12.7 MB) exists on every GPU that loads the library until the process exits;
// all calls share it, so calls that overlap on the GPU race.
namespace {

constexpr long long kNoAllocDofs = 1ll << 18;
constexpr long long kNoAllocDoubles =
    6 * kNoAllocDofs + (long long)kRedSlots * kMaxSolverBlocks + 16;   // g r z pa pb q | red | bar, stats
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

template <int K>
__global__ void __launch_bounds__(kSolverThreads) k_solve_noalloc(DevMesh m, const double* gin, double rtol, int maxit) {
  constexpr int NL = K + 1;
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = m.bar;
  double gg[2] = {0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz)
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const size_t o = size_t(f) * NL + j;
      const double v = gin[o];
      m.g[o] = v;
      gg[0] += v * v;
      if (j == 0) gg[1] += v;
    }
  if (!grid_reduce<2>(m, 4, gg, bar)) return;
  const double c0 = gg[1] / double(nF);
  for (int f = gtid; f < nF; f += gsz) m.g[size_t(f) * NL] -= c0;
  const double gnorm = sqrt(fmax(gg[0] - gg[1] * gg[1] / double(nF), 0.0));
  bool conv = false;
  int iters = 0;
  double relres = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz)
#pragma unroll
      for (int j = 0; j < NL; ++j) m.lam[size_t(f) * NL + j] = 0.0;
    conv = true;
  } else {
    for (int f = gtid; f < nF; f += gsz) {
      double y[NL];
      spmv64<NL>(m, f, m.lam, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) m.r[size_t(f) * NL + j] = m.g[size_t(f) * NL + j] - y[j];
    }
    if (!grid_sync(bar, m.stats)) return;
    double rr_end = 0.0;
    iters = pcg<NL, double>(m, m.lam, m.r, m.z, m.pa, m.pb, m.q, m.st_blk, m.st_binv, rtol * gnorm, maxit, false,
                            bar, &conv, &rr_end);
    relres = sqrt(rr_end) / gnorm;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    m.stats->last_iters = iters;
    m.stats->last_relres = relres;
    if (!conv) atomicOr(&m.stats->flags, kFlagNotConverged);
  }
}

constexpr int kMaxDevices = 64;
// Per-device address of the scratch array. Host threads may look it up concurrently: every
// lookup on a device returns the same address, so the first store wins and later ones agree.
std::atomic<double*> g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once per device.
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return cudaSuccess;
}

}  // namespace

long long noalloc_max_dofs() { return kNoAllocDofs; }

cudaError_t solve_noalloc(int k, int n_facet, const int32_t* facet_nbr, const int32_t* stencil, const double* blocks,
                          const double* binv, const double* g, double* lam, double rtol, int maxit, cudaStream_t s,
                          DevStats* host_stats) {
  double* base = nullptr;
  cudaError_t e = noalloc_scratch(&base);
  if (e != cudaSuccess) return e;
  DevMesh m{};
  m.k = k;
  m.nl = k + 1;
  m.has_kernel = 1;   // the operator is taken singular by the constant multiplier
  m.n_facet = n_facet;
  m.facet_nbr = facet_nbr;
  m.facet_stencil = stencil;
  m.st_blk = blocks;
  m.st_binv = binv;
  m.lam = lam;
  m.g = base;
  m.r = base + kNoAllocDofs;
  m.z = base + 2 * kNoAllocDofs;
  m.pa = base + 3 * kNoAllocDofs;
  m.pb = base + 4 * kNoAllocDofs;
  m.q = base + 5 * kNoAllocDofs;
  m.red = base + 6 * kNoAllocDofs;
  double* tail = m.red + (long long)kRedSlots * kMaxSolverBlocks;
  m.bar = reinterpret_cast<GridBar*>(tail);
  m.stats = reinterpret_cast<DevStats*>(tail + 2);
  // the barrier and the counters must start at zero; the array keeps the last call's contents
  e = cudaMemsetAsync(tail, 0, 16 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  const void* fn = nullptr;
  switch (k) {
    case 1: fn = (const void*)k_solve_noalloc<1>; break;
    case 2: fn = (const void*)k_solve_noalloc<2>; break;
    case 3: fn = (const void*)k_solve_noalloc<3>; break;
    default: return cudaErrorInvalidValue;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSolverThreads, 0)) != cudaSuccess) return e;
  int nb = per_sm * sms;
  if (nb > 2 * sms) nb = 2 * sms;
  const int need = (n_facet + kSolverThreads - 1) / kSolverThreads;
  if (nb > need) nb = need;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  if (nb < 1) nb = 1;
  void* args[] = {&m, (void*)&g, &rtol, &maxit};
  if ((e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kSolverThreads), args, 0, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(host_stats, m.stats, sizeof(DevStats), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace dgdf
