// Kernels of the three-dimensional path (closed tetrahedral meshes, FP64): the stage residual +
// condensation, the recovery, the face-system PCG and the lattice / diagnostics helpers.
// One thread per tetrahedron in the element kernels; the volume tables sit in shared memory,
// the face tables (four local faces x six vertex orderings) are read through the L1 cache.
// Conventions (canonical face coordinates, perm index, face rule): setup3.hpp.
#include <algorithm>

#include "device3.cuh"
#include "kcommon.cuh"
#include "solver_common.cuh"

namespace dgdf {

template <int K>
struct Dims3 {
  static constexpr int NS = (K + 1) * (K + 2) * (K + 3) / 6;
  static constexpr int ND = 3 * NS;
  static constexpr int NL = (K + 1) * (K + 2) / 2;
  static constexpr int NQ1 = (3 * K + 1) / 2;
  static constexpr int NQ = NQ1 * NQ1 * NQ1;
  static constexpr int NQF1 = (3 * K + 2) / 2;
  static constexpr int NQF = NQF1 * NQF1;
};

namespace {

constexpr int kTetThreads = 128;

template <int K>
struct VolTables3 {
  double vw[Dims3<K>::NQ];
  double vphi[Dims3<K>::NQ][Dims3<K>::NS];
  double vdphi[Dims3<K>::NQ][Dims3<K>::NS][3];
};

template <int K>
__device__ void load_vol3(const DevMesh3& m, VolTables3<K>& T) {
  using D = Dims3<K>;
  for (int i = threadIdx.x; i < D::NQ; i += blockDim.x) T.vw[i] = m.vw[i];
  for (int i = threadIdx.x; i < D::NQ * D::NS; i += blockDim.x) (&T.vphi[0][0])[i] = m.vphi[i];
  for (int i = threadIdx.x; i < D::NQ * D::NS * 3; i += blockDim.x) (&T.vdphi[0][0][0])[i] = m.vdphi[i];
}

// acc[i] = L(u)(phi_i) on tetrahedron t: -C_h(u; u, phi_i) - B_h(u, phi_i) (eq. (7), eq. (18)).
// Volume: int (u x u - nu grad u) : grad phi. Faces: the upwind flux with u.n the average of both
// traces, and the SIPG consistency, symmetry and penalty terms, at the shared face points (both
// sides evaluate at the same canonical points, so point q is point q on either side).
template <int K>
__device__ void tet_residual(const DevMesh3& m, const VolTables3<K>& T, int t, const double* __restrict__ ug,
                             const double (&up)[Dims3<K>::ND], double (&acc)[Dims3<K>::ND]) {
  using D = Dims3<K>;
  constexpr int NS = D::NS, ND = D::ND;
  const double nu = m.nu;
  const double* geo = m.geo + size_t(__ldg(&m.tet_class[t])) * kGeo3;
  double Ji[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Ji[i] = geo[G3_JINV + i];
  const double det = geo[G3_DET], s = geo[G3_S];
#pragma unroll
  for (int i = 0; i < ND; ++i) acc[i] = 0.0;
  // ---- volume terms
#pragma unroll 1
  for (int q = 0; q < D::NQ; ++q) {
    double u[3], a[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      u[c] = 0.0;
      a[c][0] = a[c][1] = a[c][2] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const double ph = T.vphi[q][j];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double x = up[c * NS + j];
        u[c] += ph * x;
#pragma unroll
        for (int r = 0; r < 3; ++r) a[c][r] += T.vdphi[q][j][r] * x;
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] *= s;
    const double w = T.vw[q] * det * s;
    double H[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double F[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        // physical gradient du_c/dx_d = s sum_r a_cr Jinv[r][d]
        const double g = s * (a[c][0] * Ji[0 * 3 + d] + a[c][1] * Ji[1 * 3 + d] + a[c][2] * Ji[2 * 3 + d]);
        F[d] = u[c] * u[d] - nu * g;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) H[c][r] = w * (F[0] * Ji[r * 3 + 0] + F[1] * Ji[r * 3 + 1] + F[2] * Ji[r * 3 + 2]);
    }
#pragma unroll
    for (int j = 0; j < NS; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        acc[c * NS + j] += H[c][0] * T.vdphi[q][j][0] + H[c][1] * T.vdphi[q][j][1] + H[c][2] * T.vdphi[q][j][2];
  }
  // ---- face terms
#pragma unroll 1
  for (int e = 0; e < 4; ++e) {
    const int tn = __ldg(&m.tet_nbr[size_t(t) * 4 + e]);
    const int en = __ldg(&m.tet_nbr_loc[size_t(t) * 4 + e]);
    const double* geon = m.geo + size_t(__ldg(&m.tet_class[tn])) * kGeo3;
    const double sn = geon[G3_S];
    const int pe = int(geo[G3_PERM + e]), pn = int(geon[G3_PERM + en]);
    const double n[3] = {geo[G3_NRM + 3 * e], geo[G3_NRM + 3 * e + 1], geo[G3_NRM + 3 * e + 2]};
    const double area = geo[G3_AREA + e];
    const double sig = __ldg(&m.face_sigma[__ldg(&m.tet_face[size_t(t) * 4 + e])]);
    // normal derivative in reference gradients: d_n psi = s sum_r d_r psihat (Jinv n)_r, with our
    // normal n for both sides
    double mo[3], mn[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      mo[r] = Ji[r * 3] * n[0] + Ji[r * 3 + 1] * n[1] + Ji[r * 3 + 2] * n[2];
      mn[r] = geon[G3_JINV + r * 3] * n[0] + geon[G3_JINV + r * 3 + 1] * n[1] + geon[G3_JINV + r * 3 + 2] * n[2];
    }
    double un[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) un[i] = __ldg(&ug[size_t(tn) * ND + i]);
    const double* fo = m.fphi + size_t(e * 6 + pe) * D::NQF * NS;
    const double* fdo = m.fdphi + size_t(e * 6 + pe) * D::NQF * NS * 3;
    const double* fn = m.fphi + size_t(en * 6 + pn) * D::NQF * NS;
    const double* fdn = m.fdphi + size_t(en * 6 + pn) * D::NQF * NS * 3;
#pragma unroll 1
    for (int q = 0; q < D::NQF; ++q) {
      double ui[3] = {0, 0, 0}, di[3] = {0, 0, 0}, uo[3] = {0, 0, 0}, dn[3] = {0, 0, 0};
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const double ph = __ldg(&fo[q * NS + j]);
        const double* g = &fdo[(q * NS + j) * 3];
        const double dno = __ldg(&g[0]) * mo[0] + __ldg(&g[1]) * mo[1] + __ldg(&g[2]) * mo[2];
        const double phn = __ldg(&fn[q * NS + j]);
        const double* gn = &fdn[(q * NS + j) * 3];
        const double dnn = __ldg(&gn[0]) * mn[0] + __ldg(&gn[1]) * mn[1] + __ldg(&gn[2]) * mn[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          ui[c] += ph * up[c * NS + j];
          di[c] += dno * up[c * NS + j];
          uo[c] += phn * un[c * NS + j];
          dn[c] += dnn * un[c * NS + j];
        }
      }
      double vn = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ui[c] *= s;
        di[c] *= s;
        uo[c] *= sn;
        dn[c] *= sn;
        vn += (ui[c] + uo[c]) * n[c];
      }
      vn *= 0.5;
      const double w = __ldg(&m.fw[q]) * 2.0 * area * s;
      double A[3], B[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double wup = vn >= 0.0 ? ui[c] : uo[c];
        const double jc = ui[c] - uo[c];
        A[c] = w * (-vn * wup + nu * 0.5 * (di[c] + dn[c]) - nu * sig * jc);
        B[c] = w * 0.5 * nu * jc;
      }
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const double ph = __ldg(&fo[q * NS + j]);
        const double* g = &fdo[(q * NS + j) * 3];
        const double dno = __ldg(&g[0]) * mo[0] + __ldg(&g[1]) * mo[1] + __ldg(&g[2]) * mo[2];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c * NS + j] += A[c] * ph + B[c] * dno;
      }
    }
  }
}

// Stage kernel (modes as StageMode): f = a u^n + b u' + c L(u') (MODE_STAGE), L(u') alone
// (MODE_RESIDUAL: h = f, the Riesz representer since M = I; MODE_PRESSURE: h = f and gl = G f),
// or f = u' (MODE_PROJECT); then h = P f and gl = G f per class.
template <int K>
__global__ void __launch_bounds__(kTetThreads) k_stage3(DevMesh3 m, StageArgs a) {
  using D = Dims3<K>;
  constexpr int ND = D::ND, L4 = 4 * D::NL;
  __shared__ VolTables3<K> T;
  load_vol3<K>(m, T);
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tet) return;
  double up[ND], f[ND];
#pragma unroll
  for (int i = 0; i < ND; ++i) up[i] = a.up[size_t(t) * ND + i];
  if (a.mode == MODE_PROJECT) {
#pragma unroll
    for (int i = 0; i < ND; ++i) f[i] = up[i];
  } else {
    tet_residual<K>(m, T, t, a.up, up, f);
    if (a.mode == MODE_STAGE) {
#pragma unroll
      for (int i = 0; i < ND; ++i) f[i] = a.a * a.un[size_t(t) * ND + i] + a.b * up[i] + a.c * f[i];
    }
  }
  if (a.mode == MODE_RESIDUAL || a.mode == MODE_PRESSURE) {
#pragma unroll
    for (int i = 0; i < ND; ++i) m.h[size_t(t) * ND + i] = f[i];
    if (a.mode == MODE_RESIDUAL) return;
  }
  const int cls = m.tet_class[t];
  const double* P = m.P + size_t(cls) * ND * ND;
  const double* G = m.G + size_t(cls) * L4 * ND;
  if (a.mode != MODE_PRESSURE)
    for (int i = 0; i < ND; ++i) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < ND; ++j) v += __ldg(&P[i * ND + j]) * f[j];
      m.h[size_t(t) * ND + i] = v;
    }
  for (int i = 0; i < L4; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < ND; ++j) v += __ldg(&G[i * ND + j]) * f[j];
    m.gl[size_t(t) * L4 + i] = v;
  }
}

// Recovery u = P f - G^T lam_T (eq. (12) condensed): h holds P f.
template <int K>
__global__ void __launch_bounds__(kTetThreads) k_recover3(DevMesh3 m, double* out) {
  using D = Dims3<K>;
  constexpr int ND = D::ND, NL = D::NL, L4 = 4 * NL;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tet) return;
  double lam[L4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int f = m.tet_face[size_t(t) * 4 + e];
#pragma unroll
    for (int j = 0; j < NL; ++j) lam[e * NL + j] = m.lam[size_t(f) * NL + j];
  }
  const double* G = m.G + size_t(m.tet_class[t]) * L4 * ND;
  for (int i = 0; i < ND; ++i) {
    double v = m.h[size_t(t) * ND + i];
#pragma unroll
    for (int l = 0; l < L4; ++l) v -= __ldg(&G[l * ND + i]) * lam[l];
    out[size_t(t) * ND + i] = v;
  }
}

// Element pressure of eq. (12) (h = f of MODE_PRESSURE, lam the solve's multipliers):
// w = W (f - C^T lam) = W f - WC lam, in the basis s phi_m (m < nw) of P^(k-1); its values at the
// (k-1)-lattice points go to pe, and each block's sum of the integrals of w to part.
template <int K>
__global__ void __launch_bounds__(kTetThreads) k_pressure3(DevMesh3 m, double* pe, double* part) {
  using D = Dims3<K>;
  constexpr int ND = D::ND, NS = D::NS, NL = D::NL, L4 = 4 * NL, NW = K * (K + 1) * (K + 2) / 6;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double integral = 0.0;
  if (t < m.n_tet) {
    double f[ND], lam[L4], w[NW];
#pragma unroll
    for (int i = 0; i < ND; ++i) f[i] = m.h[size_t(t) * ND + i];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int fc = m.tet_face[size_t(t) * 4 + e];
#pragma unroll
      for (int j = 0; j < NL; ++j) lam[e * NL + j] = m.lam[size_t(fc) * NL + j];
    }
    const int cls = m.tet_class[t];
    const double* W = m.W + size_t(cls) * NW * ND;
    const double* WC = m.WC + size_t(cls) * NW * L4;
#pragma unroll
    for (int a = 0; a < NW; ++a) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < ND; ++j) v += __ldg(&W[a * ND + j]) * f[j];
#pragma unroll
      for (int l = 0; l < L4; ++l) v -= __ldg(&WC[a * L4 + l]) * lam[l];
      w[a] = v;
    }
    const double sc = m.geo[size_t(cls) * kGeo3 + G3_S], det = m.geo[size_t(cls) * kGeo3 + G3_DET];
#pragma unroll
    for (int p = 0; p < NW; ++p) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < NW; ++a) v += __ldg(&m.plat_phi[p * NW + a]) * w[a];
      pe[size_t(t) * NW + p] = sc * v;
    }
    for (int q = 0; q < D::NQ; ++q) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < NW; ++a) v += __ldg(&m.vphi[q * NS + a]) * w[a];
      integral += __ldg(&m.vw[q]) * v;
    }
    integral *= det * sc;
  }
  integral = block_sum(integral);
  if (threadIdx.x == 0) part[blockIdx.x] = integral;
}

// The mean c = (sum of the block integrals) / vol, the same in every block (fixed order); pe -= c,
// and the face pressure pf = (the multiplier basis at the face's k-lattice) lam - c.
__global__ void k_pressure3_finish(DevMesh3 m, double* pe, double* pf, const double* part, int nparts, double vol) {
  double a = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) a += part[b];
  const double c = block_sum(a) / vol;
  const size_t gtid = size_t(blockIdx.x) * blockDim.x + threadIdx.x, gsz = size_t(gridDim.x) * blockDim.x;
  const size_t npe = size_t(m.n_tet) * m.nw;
  for (size_t i = gtid; i < npe; i += gsz) pe[i] -= c;
  if (!pf) return;
  const int nl = m.nl;
  const size_t npf = size_t(m.n_face) * nl;
  for (size_t i = gtid; i < npf; i += gsz) {
    const size_t fc = i / nl;
    const int p = int(i - fc * nl);
    double v = 0.0;
    for (int j = 0; j < nl; ++j) v += __ldg(&m.mu_lat[p * nl + j]) * m.lam[fc * nl + j];
    pf[i] = v - c;
  }
}

// Grid sum of N per-thread partials (fixed order; the result in every thread).
template <int N>
__device__ bool reduce3(const DevMesh3& m, int slot0, double (&v)[N]) {
  double s[N];
#pragma unroll
  for (int i = 0; i < N; ++i) s[i] = block_sum(v[i]);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < N; ++i) m.red[size_t(slot0 + i) * kMaxSolverBlocks + blockIdx.x] = s[i];
  if (!grid_sync(m.bar, m.stats)) return false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double a = 0.0;
    for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) a += __ldcg(&m.red[size_t(slot0 + i) * kMaxSolverBlocks + b]);
    v[i] = block_sum(a);
  }
  return true;
}

// y = (S x)_f: the face's own block and the blocks of the three other faces of each side
template <int NL>
__device__ __forceinline__ void spmv3(const DevMesh3& m, int f, const double* x, double (&y)[NL]) {
  const double* blk = m.st_blk + size_t(__ldg(&m.face_stencil[f])) * 7 * NL * NL;
#pragma unroll
  for (int i = 0; i < NL; ++i) y[i] = 0.0;
#pragma unroll
  for (int b = 0; b < 7; ++b) {
    const int g = b == 0 ? f : __ldg(&m.face_nbr[size_t(f) * 6 + b - 1]);
    double xs[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) xs[j] = __ldcg(&x[size_t(g) * NL + j]);
#pragma unroll
    for (int i = 0; i < NL; ++i)
#pragma unroll
      for (int j = 0; j < NL; ++j) y[i] += __ldg(&blk[(b * NL + i) * NL + j]) * xs[j];
  }
}

template <int NL>
__device__ __forceinline__ void binv3(const DevMesh3& m, int f, const double (&r)[NL], double (&z)[NL]) {
  const double* B = m.st_binv + size_t(__ldg(&m.face_stencil[f])) * NL * NL;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    double v = 0.0;
#pragma unroll
    for (int j = 0; j < NL; ++j) v += __ldg(&B[i * NL + j]) * r[j];
    z[i] = v;
  }
}

// Face-system solve, one persistent cooperative kernel: g = both sides' G f (no orientation
// signs: both sides use the canonical face basis), lam0 from the history or warm_scale lam
// (warm_start_row), the constant multiplier (mode 0 on every face, the kernel of S on a closed
// mesh) removed from g, then FP64 PCG with the block-Jacobi preconditioner. Residual norms
// leave out the mode-0 mean.
template <int K>
__global__ void __launch_bounds__(kSolverThreads) k_solve3(DevMesh3 m, SolveArgs a) {
  constexpr int NL = Dims3<K>::NL, L4 = 4 * NL;
  const int nF = m.n_face;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gsz = gridDim.x * blockDim.x;
  const double inv_nf = 1.0 / double(nF);
  double gg[2] = {0.0, 0.0};
  for (int f = gtid; f < nF; f += gsz) {
    const int t0 = m.face_tet[size_t(f) * 2], t1 = m.face_tet[size_t(f) * 2 + 1];
    const int e0 = m.face_loc[size_t(f) * 2], e1 = m.face_loc[size_t(f) * 2 + 1];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const double v = m.gl[size_t(t0) * L4 + e0 * NL + j] + m.gl[size_t(t1) * L4 + e1 * NL + j];
      const size_t o = size_t(f) * NL + j;
      m.g[o] = v;
      gg[0] += v * v;
      if (j == 0) gg[1] += v;
    }
    warm_start_row<NL>(m.lam, a, size_t(f) * NL);
  }
  if (!reduce3<2>(m, 4, gg)) return;
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
    // r = g - c0 1 - S lam, z = B r
    double red[3] = {0.0, 0.0, 0.0};
    for (int f = gtid; f < nF; f += gsz) {
      double y[NL], r[NL], z[NL];
      spmv3<NL>(m, f, m.lam, y);
#pragma unroll
      for (int j = 0; j < NL; ++j) r[j] = m.g[size_t(f) * NL + j] - (j == 0 ? c0 : 0.0) - y[j];
      binv3<NL>(m, f, r, z);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        m.r[size_t(f) * NL + j] = r[j];
        m.z[size_t(f) * NL + j] = z[j];
        red[0] += r[j] * z[j];
        red[1] += r[j] * r[j];
      }
      red[2] += r[0];
    }
    if (!reduce3<3>(m, 1, red)) return;
    double rho = red[0];
    rr = fmax(red[1] - red[2] * red[2] * inv_nf, 0.0);
    double beta = 0.0;
    double* pold = m.pa;
    double* pnew = m.pb;
    for (;; ++it) {
      if (!isfinite(rr) || !isfinite(rho)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      if (sqrt(rr) <= stop) {
        conv = true;
        break;
      }
      if (it >= a.maxit) break;
      // p_new = z + beta p_old (own rows), q = S p_new (from the neighbours' z and p_old)
      double pq[1] = {0.0};
      for (int f = gtid; f < nF; f += gsz) {
        const double* blk = m.st_blk + size_t(__ldg(&m.face_stencil[f])) * 7 * NL * NL;
        double y[NL], p0[NL];
#pragma unroll
        for (int i = 0; i < NL; ++i) y[i] = 0.0;
#pragma unroll
        for (int b = 0; b < 7; ++b) {
          const int g = b == 0 ? f : __ldg(&m.face_nbr[size_t(f) * 6 + b - 1]);
          double xs[NL];
#pragma unroll
          for (int j = 0; j < NL; ++j) {
            const size_t o = size_t(g) * NL + j;
            xs[j] = it == 0 ? __ldcg(&m.z[o]) : __ldcg(&m.z[o]) + beta * __ldcg(&pold[o]);
            if (b == 0) p0[j] = xs[j];
          }
#pragma unroll
          for (int i = 0; i < NL; ++i)
#pragma unroll
            for (int j = 0; j < NL; ++j) y[i] += __ldg(&blk[(b * NL + i) * NL + j]) * xs[j];
        }
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          pnew[size_t(f) * NL + j] = p0[j];
          m.q[size_t(f) * NL + j] = y[j];
          pq[0] += p0[j] * y[j];
        }
      }
      if (!reduce3<1>(m, 0, pq)) return;
      if (!(pq[0] > 0.0)) {
        if (!isfinite(pq[0]) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&m.stats->flags, kFlagNonFinite);
        break;
      }
      const double alpha = rho / pq[0];
      double red2[3] = {0.0, 0.0, 0.0};
      for (int f = gtid; f < nF; f += gsz) {
        double r[NL], z[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const size_t o = size_t(f) * NL + j;
          m.lam[o] += alpha * pnew[o];
          r[j] = m.r[o] - alpha * m.q[o];
          m.r[o] = r[j];
        }
        binv3<NL>(m, f, r, z);
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          m.z[size_t(f) * NL + j] = z[j];
          red2[0] += r[j] * z[j];
          red2[1] += r[j] * r[j];
        }
        red2[2] += r[0];
      }
      if (!reduce3<3>(m, 1, red2)) return;
      beta = red2[0] / rho;
      rho = red2[0];
      rr = fmax(red2[1] - red2[2] * red2[2] * inv_nf, 0.0);
      double* tmp = pold;
      pold = pnew;
      pnew = tmp;
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

// Lattice values [n_tet][ns][3] -> coefficients [n_tet][3 ns]: coef = sqrt(det) Vhat^-1 vals.
template <int K>
__global__ void k_lattice_to_coef3(DevMesh3 m, const double* vals, double* coef) {
  constexpr int NS = Dims3<K>::NS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tet) return;
  const double sq = 1.0 / m.geo[size_t(m.tet_class[t]) * kGeo3 + G3_S];
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < NS; ++j) {
      double v = 0.0;
      for (int p = 0; p < NS; ++p) v += m.lat_inv[j * NS + p] * vals[(size_t(t) * NS + p) * 3 + c];
      coef[size_t(t) * 3 * NS + c * NS + j] = sq * v;
    }
}

template <int K>
__global__ void k_coef_to_lattice3(DevMesh3 m, const double* coef, double* vals) {
  constexpr int NS = Dims3<K>::NS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tet) return;
  const double s = m.geo[size_t(m.tet_class[t]) * kGeo3 + G3_S];
  for (int p = 0; p < NS; ++p)
    for (int c = 0; c < 3; ++c) {
      double v = 0.0;
      for (int j = 0; j < NS; ++j) v += m.lat_phi[p * NS + j] * coef[size_t(t) * 3 * NS + c * NS + j];
      vals[(size_t(t) * NS + p) * 3 + c] = s * v;
    }
}

// Diagnostics partials per block: energy, enstrophy (|curl u|^2), max |div u| at the volume
// points, max |[u.n]| at the face points (each face seen from both sides).
template <int K>
__global__ void __launch_bounds__(kTetThreads) k_diagnostics3(DevMesh3 m, const double* coef) {
  using D = Dims3<K>;
  constexpr int NS = D::NS, ND = D::ND;
  __shared__ VolTables3<K> T;
  load_vol3<K>(m, T);
  __syncthreads();
  double en = 0.0, ens = 0.0, dmax = 0.0, jmax = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.n_tet; t += gridDim.x * blockDim.x) {
    double c[ND];
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      c[i] = coef[size_t(t) * ND + i];
      en += c[i] * c[i];
    }
    const double* geo = m.geo + size_t(m.tet_class[t]) * kGeo3;
    const double det = geo[G3_DET], s = geo[G3_S];
    for (int q = 0; q < D::NQ; ++q) {
      double g[3][3];
      for (int cc = 0; cc < 3; ++cc) {
        double a[3] = {0, 0, 0};
        for (int j = 0; j < NS; ++j)
          for (int r = 0; r < 3; ++r) a[r] += T.vdphi[q][j][r] * c[cc * NS + j];
        for (int d = 0; d < 3; ++d)
          g[cc][d] = s * (a[0] * geo[G3_JINV + d] + a[1] * geo[G3_JINV + 3 + d] + a[2] * geo[G3_JINV + 6 + d]);
      }
      const double w0 = g[2][1] - g[1][2], w1 = g[0][2] - g[2][0], w2 = g[1][0] - g[0][1];
      ens += T.vw[q] * det * (w0 * w0 + w1 * w1 + w2 * w2);
      dmax = fmax(dmax, fabs(g[0][0] + g[1][1] + g[2][2]));
    }
    for (int e = 0; e < 4; ++e) {
      const int tn = m.tet_nbr[size_t(t) * 4 + e], en2 = m.tet_nbr_loc[size_t(t) * 4 + e];
      const double* geon = m.geo + size_t(m.tet_class[tn]) * kGeo3;
      const int pe = int(geo[G3_PERM + e]), pn = int(geon[G3_PERM + en2]);
      const double* fo = m.fphi + size_t(e * 6 + pe) * D::NQF * NS;
      const double* fn = m.fphi + size_t(en2 * 6 + pn) * D::NQF * NS;
      for (int q = 0; q < D::NQF; ++q) {
        double jn = 0.0;
        for (int cc = 0; cc < 3; ++cc) {
          double a = 0.0, b = 0.0;
          for (int j = 0; j < NS; ++j) {
            a += fo[q * NS + j] * c[cc * NS + j];
            b += fn[q * NS + j] * coef[size_t(tn) * ND + cc * NS + j];
          }
          jn += (s * a - geon[G3_S] * b) * geo[G3_NRM + 3 * e + cc];
        }
        jmax = fmax(jmax, fabs(jn));
      }
    }
  }
  en = block_sum(en);
  ens = block_sum(ens);
  dmax = block_max(dmax);
  jmax = block_max(jmax);
  if (threadIdx.x == 0) {
    m.red[0 * kMaxSolverBlocks + blockIdx.x] = en;
    m.red[1 * kMaxSolverBlocks + blockIdx.x] = ens;
    m.red[2 * kMaxSolverBlocks + blockIdx.x] = dmax;
    m.red[3 * kMaxSolverBlocks + blockIdx.x] = jmax;
  }
}

__global__ void k_diag_finish3(DevMesh3 m, int nparts) {
  if (threadIdx.x >= 32) return;
  double a = 0, b = 0, c = 0, d = 0;
  for (int i = threadIdx.x; i < nparts; i += 32) {
    a += m.red[0 * kMaxSolverBlocks + i];
    b += m.red[1 * kMaxSolverBlocks + i];
    c = fmax(c, m.red[2 * kMaxSolverBlocks + i]);
    d = fmax(d, m.red[3 * kMaxSolverBlocks + i]);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_max(c);
  d = warp_max(d);
  if (threadIdx.x == 0) {
    m.diag[0] = a;
    m.diag[1] = b;
    m.diag[2] = c;
    m.diag[3] = d;
  }
}

int blocks3(int n) { return (n + kTetThreads - 1) / kTetThreads; }

template <int K>
int solve3_blocks_for() {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve3<K>, kSolverThreads, 0);
  return per_sm * sms;
}

}  // namespace

#define DGDF_DISPATCH_K3(k, CALL)                \
  switch (k) {                                   \
    case 1: { constexpr int K = 1; CALL; break; } \
    case 2: { constexpr int K = 2; CALL; break; } \
    default: return cudaErrorInvalidValue;       \
  }

bool tet_tables_match(int k, int nq, int nqf) {
  switch (k) {
    case 1: return nq == Dims3<1>::NQ && nqf == Dims3<1>::NQF;
    case 2: return nq == Dims3<2>::NQ && nqf == Dims3<2>::NQF;
    default: return false;
  }
}

cudaError_t launch_stage3(const DevMesh3& m, const StageArgs& a, cudaStream_t s) {
  DGDF_DISPATCH_K3(m.k, (k_stage3<K><<<blocks3(m.n_tet), kTetThreads, 0, s>>>(m, a)));
  return cudaGetLastError();
}

cudaError_t launch_recover3(const DevMesh3& m, double* out, cudaStream_t s) {
  DGDF_DISPATCH_K3(m.k, (k_recover3<K><<<blocks3(m.n_tet), kTetThreads, 0, s>>>(m, out)));
  return cudaGetLastError();
}

cudaError_t launch_lattice_to_coef3(const DevMesh3& m, const double* vals, double* coef, cudaStream_t s) {
  DGDF_DISPATCH_K3(m.k, (k_lattice_to_coef3<K><<<blocks3(m.n_tet), kTetThreads, 0, s>>>(m, vals, coef)));
  return cudaGetLastError();
}

cudaError_t launch_coef_to_lattice3(const DevMesh3& m, const double* coef, double* vals, cudaStream_t s) {
  DGDF_DISPATCH_K3(m.k, (k_coef_to_lattice3<K><<<blocks3(m.n_tet), kTetThreads, 0, s>>>(m, coef, vals)));
  return cudaGetLastError();
}

cudaError_t launch_diagnostics3(const DevMesh3& m, const double* coef, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int nb = blocks3(m.n_tet);
  if (nb > 2 * sms) nb = 2 * sms;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  DGDF_DISPATCH_K3(m.k, (k_diagnostics3<K><<<nb, kTetThreads, 0, s>>>(m, coef)));
  k_diag_finish3<<<1, 32, 0, s>>>(m, nb);
  return cudaGetLastError();
}

int pressure3_parts(const DevMesh3& m) { return blocks3(m.n_tet); }

cudaError_t launch_pressure3(const DevMesh3& m, double* pe, double* pf, double* part, double vol, cudaStream_t s) {
  const int nb = blocks3(m.n_tet);
  DGDF_DISPATCH_K3(m.k, (k_pressure3<K><<<nb, kTetThreads, 0, s>>>(m, pe, part)));
  const size_t n = std::max(size_t(m.n_tet) * m.nw, size_t(m.n_face) * m.nl);
  const int fb = int(std::min<size_t>((n + 255) / 256, 1024));
  k_pressure3_finish<<<fb, 256, 0, s>>>(m, pe, pf, part, nb, vol);
  return cudaGetLastError();
}

int solver3_blocks(const DevMesh3& m) {
  int nb = 0;
  switch (m.k) {
    case 1: nb = solve3_blocks_for<1>(); break;
    case 2: nb = solve3_blocks_for<2>(); break;
    default: return 0;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nb > 2 * sms) nb = 2 * sms;
  const int need = (m.n_face + kSolverThreads - 1) / kSolverThreads;
  if (nb > need) nb = need;
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  return nb < 1 ? 1 : nb;
}

cudaError_t launch_solve3(const DevMesh3& m, const SolveArgs& a, int nblocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(m.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  DevMesh3 mm = m;
  SolveArgs aa = a;
  void* args[] = {&mm, &aa};
  const void* fn = nullptr;
  switch (m.k) {
    case 1: fn = (const void*)k_solve3<1>; break;
    case 2: fn = (const void*)k_solve3<2>; break;
    default: return cudaErrorInvalidValue;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(kSolverThreads), args, 0, s);
}

}  // namespace dgdf
