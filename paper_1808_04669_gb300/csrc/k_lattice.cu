// Facet-system solve on translation-invariant split-square meshes (the lattice
// path of the condensed hybrid-mixed system, eq. (12) of Sec. 2.4).
//
// On such a mesh the facet operator S is block circulant over the N x N cell
// grid: a 2-D discrete Fourier transform turns it into one Hermitian block
// S^(kappa) of size C = 3(k+1) per wavenumber, and S^+ r = IDFT(S^(kappa)^-1 DFT(r))
// (pseudo-inverse at kappa = 0, the constant multiplier). This kernel runs PCG
// with FP64 vectors and FP64 SpMV, preconditioned by that Fourier-space inverse
// evaluated in precision R (FP32 in the mixed form, FP64 in the FP64 form):
// the preconditioned operator is the identity up to R's rounding, so a solve
// takes one or two iterations (FP64) or a few (FP32), instead of O(N).
// The transforms run in shared memory (radix-2 FFTs when N is a power of two):
//   rows  : DFT along i of r (facets numbered in lattice order), tiles of rows
//   column: DFT along j, multiply by S^(kappa)^-1, inverse DFT along j
//   rows  : inverse DFT along i, scattered back to facet order (scaled 1/N^2)
// (for N not a power of two a direct O(N^2) DFT per row in shared memory)
// with a grid barrier between the three passes. One persistent cooperative
// kernel per solve, one block per SM.
#include "device.cuh"
#include "kcommon.cuh"
#include "solver_common.cuh"

namespace dgdf {
namespace {

constexpr int kLatThreads = 512;

template <typename R>
struct CxT;
template <>
struct CxT<float> {
  using T = float2;
};
template <>
struct CxT<double> {
  using T = double2;
};

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C2>
__device__ __forceinline__ C2 cadd(C2 a, C2 b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename C2>
__device__ __forceinline__ C2 csub(C2 a, C2 b) {
  return {a.x - b.x, a.y - b.y};
}

__device__ __forceinline__ int brev(int t, int logn) { return logn == 0 ? 0 : int(__brev(unsigned(t)) >> (32 - logn)); }

// Radix-2 decimation in time on `rows` rows of length n = 2^logn in shared memory:
// input in bit-reversed order, output in natural order. tw[t] = exp(-2 pi i t / n).
template <typename C2>
__device__ void fft_dit(C2* buf, int rows, int logn, const C2* tw, bool inverse) {
  const int n = 1 << logn, hn = n >> 1;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1), step = n >> s;
    for (int b = threadIdx.x; b < rows * hn; b += blockDim.x) {
      const int row = b / hn, k = b - row * hn;
      const int grp = k >> (s - 1), pos = k & (half - 1);
      const int i0 = row * n + (grp << s) + pos, i1 = i0 + half;
      C2 w = tw[pos * step];
      if (inverse) w.y = -w.y;
      const C2 u = buf[i0], v = cmul(buf[i1], w);
      buf[i0] = cadd(u, v);
      buf[i1] = csub(u, v);
    }
    __syncthreads();
  }
}

// Radix-2 decimation in frequency: input natural, output bit-reversed.
template <typename C2>
__device__ void fft_dif(C2* buf, int rows, int logn, const C2* tw, bool inverse) {
  const int n = 1 << logn, hn = n >> 1;
  for (int s = logn; s >= 1; --s) {
    const int half = 1 << (s - 1), step = n >> s;
    for (int b = threadIdx.x; b < rows * hn; b += blockDim.x) {
      const int row = b / hn, k = b - row * hn;
      const int grp = k >> (s - 1), pos = k & (half - 1);
      const int i0 = row * n + (grp << s) + pos, i1 = i0 + half;
      C2 w = tw[pos * step];
      if (inverse) w.y = -w.y;
      const C2 u = buf[i0], v = buf[i1];
      buf[i0] = cadd(u, v);
      buf[i1] = cmul(csub(u, v), w);
    }
    __syncthreads();
  }
}

// Direct DFT of `rows` rows of length n (any n): out[r][k] = sum_t in[r][t] w^(t k mod n),
// w[m] = exp(-2 pi i m / n) (conjugated for the inverse). Natural order in and out.
template <typename C2>
__device__ void dft(const C2* in, C2* out, int rows, int n, const C2* tw, bool inverse) {
  for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
    const int row = e / n, k = e - row * n;
    const C2* x = in + row * n;
    C2 acc = {0, 0};
    int idx = 0;
    for (int t = 0; t < n; ++t) {
      C2 w = tw[idx];
      if (inverse) w.y = -w.y;
      acc = cadd(acc, cmul(x[t], w));
      idx += k;
      if (idx >= n) idx -= n;
    }
    out[e] = acc;
  }
  __syncthreads();
}

template <int K, typename R>
struct LatCtx {
  using C2 = typename CxT<R>::T;
  static constexpr int NL = K + 1, C = 3 * NL;
  int N, logn, tr, ntj;
  bool pow2;      // radix-2 FFT (N a power of two) or direct DFT
  C2* tw;         // [N] exp(-2 pi i t / N)
  C2* buf;
  C2* buf2;       // second buffer of the direct DFT
  C2* X;          // [C][N(ki)][N(j)]
  const C2* S;    // [N(ki)][C][C][N(kj)]
};

// Position in the transform buffer of the element with index i: bit-reversed for the
// radix-2 passes (input of the forward one, output of the inverse one), natural for the DFT.
template <int K, typename R>
__device__ __forceinline__ int tpos(const LatCtx<K, R>& L, int i) {
  return L.pow2 ? brev(i, L.logn) : i;
}

// Forward transform of rows loaded at tpos(); returns the buffer with the natural-order result.
template <int K, typename R>
__device__ typename CxT<R>::T* xform_fwd(const LatCtx<K, R>& L, typename CxT<R>::T* a, typename CxT<R>::T* b,
                                         int rows) {
  if (L.pow2) {
    fft_dit(a, rows, L.logn, L.tw, false);
    return a;
  }
  dft(a, b, rows, L.N, L.tw, false);
  return b;
}

// Inverse transform of natural-order rows; index i of the result sits at tpos(i).
template <int K, typename R>
__device__ typename CxT<R>::T* xform_inv(const LatCtx<K, R>& L, typename CxT<R>::T* a, typename CxT<R>::T* b,
                                         int rows) {
  if (L.pow2) {
    fft_dif(a, rows, L.logn, L.tw, true);
    return a;
  }
  dft(a, b, rows, L.N, L.tw, true);
  return b;
}

// Facets are numbered (type, j, i) on a lattice mesh, so a tile of tr rows of one
// facet type with all k+1 modes is one contiguous range of the facet-major vectors:
// DOF index ((type N + j) N + i)(k+1) + m.

// Row pass, forward: read r (optionally first updating r -= alpha q, lam += alpha p),
// DFT along i, store transposed. Accumulates r.r into *rr.
template <int K, typename R>
__device__ void rows_forward(const DevMesh& m, const LatCtx<K, R>& L, bool update, double alpha, const double* p,
                             double* rr) {
  using C2 = typename CxT<R>::T;
  constexpr int NL = K + 1;
  const int N = L.N;
  const int ntiles = 3 * L.ntj;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty = tile / L.ntj, j0 = (tile - ty * L.ntj) * L.tr;
    const int rows = min(L.tr, N - j0);
    const size_t base = (size_t(ty) * N + j0) * N * NL;
    for (int e = threadIdx.x; e < rows * N * NL; e += blockDim.x) {
      const int mm = e % NL, rest = e / NL;
      const int r_ = rest / N, i = rest - r_ * N;
      const size_t o = base + e;
      double rv = __ldcg(&m.r[o]);
      if (update) {
        rv -= alpha * __ldcg(&m.q[o]);
        m.r[o] = rv;
        m.lam[o] += alpha * __ldcg(&p[o]);
      }
      *rr += rv * rv;
      L.buf[(mm * rows + r_) * N + tpos(L, i)] = C2{R(rv), R(0)};
    }
    __syncthreads();
    const C2* res = xform_fwd(L, L.buf, L.buf2, NL * rows);
    for (int e = threadIdx.x; e < rows * N * NL; e += blockDim.x) {
      const int r_ = e % rows, rest = e / rows;
      const int mm = rest / N, ki = rest - mm * N;
      L.X[(size_t(ty * NL + mm) * N + ki) * N + j0 + r_] = res[(mm * rows + r_) * N + ki];
    }
    __syncthreads();
  }
}

// Column pass: DFT along j, multiply by S^(kappa)^-1 (warp c computes component c of 32
// consecutive k_j), inverse DFT along j.
template <int K, typename R>
__device__ void columns(const LatCtx<K, R>& L) {
  using C2 = typename CxT<R>::T;
  constexpr int C = LatCtx<K, R>::C;
  const int N = L.N;
  const int lane = threadIdx.x & 31, wc = threadIdx.x >> 5;
  for (int ki = blockIdx.x; ki < N; ki += gridDim.x) {
    for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
      const int c = e / N, j = e - c * N;
      L.buf[c * N + tpos(L, j)] = __ldcg(&L.X[(size_t(c) * N + ki) * N + j]);
    }
    __syncthreads();
    C2* cur = xform_fwd(L, L.buf, L.buf2, C);
    const C2* S = L.S + size_t(ki) * C * C * N;
    for (int kj0 = 0; kj0 < N; kj0 += 32) {
      const int kj = kj0 + lane;
      const bool act = wc < C && kj < N;
      C2 y = {R(0), R(0)};
      if (act) {
#pragma unroll
        for (int cc = 0; cc < C; ++cc) y = cadd(y, cmul(__ldg(&S[(size_t(wc) * C + cc) * N + kj]), cur[cc * N + kj]));
      }
      __syncthreads();
      if (act) cur[wc * N + kj] = y;
      __syncthreads();
    }
    const C2* res = xform_inv(L, cur, cur == L.buf ? L.buf2 : L.buf, C);
    for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
      const int c = e / N, j = e - c * N;
      L.X[(size_t(c) * N + ki) * N + j] = res[c * N + tpos(L, j)];
    }
    __syncthreads();
  }
}

// Row pass, inverse: inverse DFT along i, z = result / N^2 in facet order.
// Accumulates r.z_new into *rz and, if with_old, r.z_old into *rzo.
template <int K, typename R>
__device__ void rows_inverse(const DevMesh& m, const LatCtx<K, R>& L, bool with_old, double* rz, double* rzo) {
  using C2 = typename CxT<R>::T;
  constexpr int NL = K + 1;
  const int N = L.N;
  const double scale = 1.0 / (double(N) * double(N));
  const int ntiles = 3 * L.ntj;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty = tile / L.ntj, j0 = (tile - ty * L.ntj) * L.tr;
    const int rows = min(L.tr, N - j0);
    const size_t base = (size_t(ty) * N + j0) * N * NL;
    for (int e = threadIdx.x; e < rows * N * NL; e += blockDim.x) {
      const int r_ = e % rows, rest = e / rows;
      const int mm = rest / N, ki = rest - mm * N;
      L.buf[(mm * rows + r_) * N + ki] = __ldcg(&L.X[(size_t(ty * NL + mm) * N + ki) * N + j0 + r_]);
    }
    __syncthreads();
    const C2* res = xform_inv(L, L.buf, L.buf2, NL * rows);
    for (int e = threadIdx.x; e < rows * N * NL; e += blockDim.x) {
      const int mm = e % NL, rest = e / NL;
      const int r_ = rest / N, i = rest - r_ * N;
      const size_t o = base + e;
      const double zv = double(res[(mm * rows + r_) * N + tpos(L, i)].x) * scale;
      const double rv = __ldcg(&m.r[o]);
      if (with_old) *rzo += rv * __ldcg(&m.z[o]);
      *rz += rv * zv;
      m.z[o] = zv;
    }
    __syncthreads();
  }
}

template <int K, typename R>
__global__ void __launch_bounds__(kLatThreads, 1) k_solve_lat(DevMesh m, SolveArgs a) {
  using C2 = typename CxT<R>::T;
  constexpr int NL = K + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LatCtx<K, R> L;
  L.N = m.lat_N;
  L.logn = m.lat_logn;
  L.tr = m.lat_tr;
  L.ntj = (L.N + L.tr - 1) / L.tr;
  L.pow2 = (L.N & (L.N - 1)) == 0;
  L.tw = reinterpret_cast<C2*>(smem_raw);
  L.buf = L.tw + L.N;
  L.buf2 = L.buf + m.lat_bufsz;
  L.X = reinterpret_cast<C2*>(m.lat_x);
  L.S = reinterpret_cast<const C2*>(m.lat_sinv);
  for (int t = threadIdx.x; t < L.N; t += blockDim.x) L.tw[t] = C2{R(m.lat_tw[2 * t]), R(m.lat_tw[2 * t + 1])};
  __syncthreads();
  const int nF = m.n_facet;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  GridBar* bar = m.bar;
  // g from both sides of every facet; warm-started lam
  double gg[2] = {0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz) {
    double gv[NL];
    assemble_g<NL>(m, f, gv);
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const size_t o = size_t(f) * NL + j;
      m.g[o] = gv[j];
      m.lam[o] = a.warm_scale == 0.0 ? 0.0 : a.warm_scale * m.lam[o];
      gg[0] += gv[j] * gv[j];
    }
    gg[1] += gv[0];
  }
  if (!grid_reduce<2>(m, 4, gg, bar)) return;
  const double c0 = gg[1] / double(nF);
  const double gnorm = sqrt(fmax(gg[0] - gg[1] * gg[1] / double(nF), 0.0));
  const double stop = a.rtol * gnorm;
  int it = 0;
  bool conv = false;
  double relres = 0.0;
  if (gnorm == 0.0) {
    for (int f = gtid; f < nF; f += gsz)
#pragma unroll
      for (int j = 0; j < NL; ++j) m.lam[size_t(f) * NL + j] = 0.0;
    conv = true;
  } else {
    // r = g - S lam with the constant component of g removed
    for (int f = gtid; f < nF; f += gsz) {
      double y[NL];
      spmv64<NL>(m, f, m.lam, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const size_t o = size_t(f) * NL + j;
        const double gv = m.g[o] - (j == 0 ? c0 : 0.0);
        m.g[o] = gv;
        m.r[o] = gv - y[j];
      }
    }
    if (!grid_sync(bar, m.stats)) return;
    // z = M r
    double rr[1] = {0.0};
    rows_forward<K, R>(m, L, false, 0.0, nullptr, &rr[0]);
    if (!grid_reduce<1>(m, 6, rr, bar)) return;
    columns<K, R>(L);
    if (!grid_sync(bar, m.stats)) return;
    double rz[2] = {0.0, 0.0};
    rows_inverse<K, R>(m, L, false, &rz[0], &rz[1]);
    if (!grid_reduce<2>(m, 1, rz, bar)) return;
    double rho = rz[0], rrv = rr[0];
    double beta = 0.0;
    double* pold = m.pa;
    double* pnew = m.pb;
    for (;; ++it) {
      relres = sqrt(rrv) / gnorm;
      if (!isfinite(rrv) || !isfinite(rho)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      if (sqrt(rrv) <= stop) {
        conv = true;
        break;
      }
      if (it >= a.maxit) break;
      // p_new = z + beta p_old, q = S p_new
      double pq[1] = {0.0};
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
      }
      if (!grid_reduce<1>(m, 0, pq, bar)) return;
      if (!(pq[0] > 0.0)) {
        if (!isfinite(pq[0]) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      const double alpha = rho / pq[0];
      // r -= alpha q, lam += alpha p, and the forward row pass of z = M r
      rr[0] = 0.0;
      rows_forward<K, R>(m, L, true, alpha, pnew, &rr[0]);
      if (!grid_reduce<1>(m, 6, rr, bar)) return;
      rrv = rr[0];
      if (sqrt(rrv) <= stop || !isfinite(rrv)) {
        ++it;
        relres = sqrt(rrv) / gnorm;
        conv = isfinite(rrv);
        if (!conv && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      columns<K, R>(L);
      if (!grid_sync(bar, m.stats)) return;
      rz[0] = rz[1] = 0.0;
      rows_inverse<K, R>(m, L, true, &rz[0], &rz[1]);
      if (!grid_reduce<2>(m, 1, rz, bar)) return;
      // flexible (Polak-Ribiere) beta: the FP32 preconditioner is symmetric only up to rounding
      beta = (rz[0] - rz[1]) / rho;
      rho = rz[0];
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
    st->last_relres = relres;
    st->last_sweeps = 1;
    st->total_sweeps += 1;
    if (!conv) atomicOr(&st->flags, kFlagNotConverged);
  }
}

template <int K, typename R>
const void* lat_fn() {
  return (const void*)k_solve_lat<K, R>;
}

const void* lattice_kernel(int k, int fp32) {
  switch (k * 2 + (fp32 ? 1 : 0)) {
    case 2: return lat_fn<1, double>();
    case 3: return lat_fn<1, float>();
    case 4: return lat_fn<2, double>();
    case 5: return lat_fn<2, float>();
    case 6: return lat_fn<3, double>();
    case 7: return lat_fn<3, float>();
    default: return nullptr;
  }
}

}  // namespace

int lattice_tile_rows(int k, int N, int fp32) {
  const size_t cx = fp32 ? 8 : 16;
  const size_t budget = 96 * 1024;
  long long tr = (long long)(budget / (size_t(k + 1) * N * cx));
  if (tr > 8) tr = 8;
  if (tr < 1) tr = 1;
  if (tr > N) tr = N;
  return int(tr);
}

size_t lattice_buffer_elems(int k, int N, int fp32) {
  const size_t C = 3 * (k + 1), rows_buf = size_t(k + 1) * lattice_tile_rows(k, N, fp32);
  return (C > rows_buf ? C : rows_buf) * N;
}

size_t lattice_smem_bytes(int k, int N, int fp32) {
  const size_t cx = fp32 ? 8 : 16;
  const bool pow2 = (N & (N - 1)) == 0;
  return (size_t(N) + (pow2 ? 1 : 2) * lattice_buffer_elems(k, N, fp32)) * cx;
}

int lattice_blocks(int k, int N, int fp32) {
  const void* fn = lattice_kernel(k, fp32);
  if (!fn) return 0;
  const size_t smem = lattice_smem_bytes(k, N, fp32);
  int per_sm = 0, dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  // the attribute is per kernel, shared by all meshes: allow the device maximum once,
  // so that meshes of different sizes can use the same instantiation
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int max_dyn = optin - int(fa.sharedSizeBytes);
  if (max_dyn <= 0 || smem > size_t(max_dyn)) return 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLatThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (per_sm < 1) return 0;
  int nb = sms;   // one block per SM
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  return nb;
}

cudaError_t launch_solve_lattice(const DevMesh& m, const SolveArgs& a, int nblocks, int fp32, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  const void* fn = lattice_kernel(m.k, fp32);
  if (!fn) return cudaErrorInvalidValue;
  DevMesh mm = m;
  SolveArgs aa = a;
  void* args[] = {&mm, &aa};
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kLatThreads), args,
                                     lattice_smem_bytes(m.k, m.lat_N, fp32), s);
}

}  // namespace dgdf
