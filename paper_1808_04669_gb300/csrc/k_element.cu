// Element kernels: stage residual + condensation (K1-K3), recovery (K5), pressure,
// lattice conversion and diagnostics. One thread per triangle; the reference
// tables sit in shared memory and are read as warp broadcasts.
#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"
#include "ktables.cuh"

namespace dgdf {

// Convective term of eq. (7) on boundary facet e of triangle t when it is an inflow or
// outflow facet (Sec. 2.5): the flux (u.n) u^up with u.n the average of the interior trace and
// the exterior state, which is u_in on an inflow facet (stored at the facet points in the
// canonical direction: our point q is point q there when the triangle runs the facet the
// canonical way, else point NQF-1-q) and the interior trace on an outflow facet. The viscous
// form has no boundary terms (natural conditions on every boundary facet).
template <int K, typename R>
__device__ void boundary_flux(const DevMesh& m, const SmemTables<K, R>& T, int t, int e, const R (&Ji)[4], R s,
                              const R (&up)[Dims<K>::ND], R (&acc)[Dims<K>::ND]) {
  using D = Dims<K>;
  constexpr int NS = D::NS;
  const int f = m.tri_facet[size_t(t) * 3 + e];
  const int kd = m.facet_kind[f];
  if (kd == kFacetWall) return;
  const bool canon = m.tri_orient[size_t(t) * 3 + e] > 0;
  const double* geo = m.geo + size_t(m.tri_class[t]) * kGeo;
  const R n0 = R(geo[G_NRM + 2 * e]), n1 = R(geo[G_NRM + 2 * e + 1]);
  const R len = R(geo[G_FLEN + e]);
#pragma unroll 1
  for (int q = 0; q < D::NQF; ++q) {
    R ui0 = 0, ui1 = 0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const R ph = T.fphi[e][q][j];
      ui0 += ph * up[j];
      ui1 += ph * up[NS + j];
    }
    ui0 *= s;
    ui1 *= s;
    R uo0 = ui0, uo1 = ui1;
    if (kd == kFacetInflow) {
      const double* uq = m.inflow_q + (size_t(f) * D::NQF + (canon ? q : D::NQF - 1 - q)) * 2;
      uo0 = R(uq[0]);
      uo1 = R(uq[1]);
    }
    const R vn = R(0.5) * ((ui0 + uo0) * n0 + (ui1 + uo1) * n1);
    const R w0 = vn >= R(0) ? ui0 : uo0, w1 = vn >= R(0) ? ui1 : uo1;
    const R w = T.fw[q] * len * s;
    const R A0 = -w * vn * w0, A1 = -w * vn * w1;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const R ph = T.fphi[e][q][j];
      acc[j] += A0 * ph;
      acc[NS + j] += A1 * ph;
    }
  }
}

// acc[i] = L(u)(phi_i) on triangle t: -C_h(u;u,phi_i) - B_h(u,phi_i) (eq. (7), eq. (18)).
// Volume: int (u x u - nu grad u) : grad phi. Facets: the upwind flux with u.n the
// average of both traces, and the SIPG consistency, symmetry and penalty terms,
// at the facet Gauss points (the neighbour traverses the facet the other way,
// so its point q is our point NQF-1-q). ug is the global coefficient array of u.
template <int K, typename R>
__device__ void element_residual(const DevMesh& m, const SmemTables<K, R>& T, int t, const double* __restrict__ ug,
                                 const R (&up)[Dims<K>::ND], R (&acc)[Dims<K>::ND]) {
  using D = Dims<K>;
  constexpr int NS = D::NS;
  const R nu = R(m.nu);
  const double* geo = m.geo + size_t(m.tri_class[t]) * kGeo;
  const R Ji[4] = {R(geo[G_JINV + 0]), R(geo[G_JINV + 1]), R(geo[G_JINV + 2]), R(geo[G_JINV + 3])};
  const R det = R(geo[G_DET]), s = R(geo[G_S]);
#pragma unroll
  for (int i = 0; i < D::ND; ++i) acc[i] = R(0);
  // ---- volume terms
#pragma unroll 1
  for (int q = 0; q < D::NQ; ++q) {
    R u0 = 0, u1 = 0, a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const R ph = T.vphi[q][j], d0 = T.vdphi[q][j][0], d1 = T.vdphi[q][j][1];
      u0 += ph * up[j];
      u1 += ph * up[NS + j];
      a00 += d0 * up[j];
      a01 += d1 * up[j];
      a10 += d0 * up[NS + j];
      a11 += d1 * up[NS + j];
    }
    u0 *= s;
    u1 *= s;
    // physical gradient du_c/dx_d = s sum_r a_cr Jinv[r][d]
    const R g00 = s * (a00 * Ji[0] + a01 * Ji[2]), g01 = s * (a00 * Ji[1] + a01 * Ji[3]);
    const R g10 = s * (a10 * Ji[0] + a11 * Ji[2]), g11 = s * (a10 * Ji[1] + a11 * Ji[3]);
    const R F00 = u0 * u0 - nu * g00, F01 = u0 * u1 - nu * g01;
    const R F10 = u1 * u0 - nu * g10, F11 = u1 * u1 - nu * g11;
    const R w = T.vw[q] * det * s;
    // H_cr = sum_d F_cd Jinv[r][d]
    const R H00 = w * (F00 * Ji[0] + F01 * Ji[1]), H01 = w * (F00 * Ji[2] + F01 * Ji[3]);
    const R H10 = w * (F10 * Ji[0] + F11 * Ji[1]), H11 = w * (F10 * Ji[2] + F11 * Ji[3]);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const R d0 = T.vdphi[q][j][0], d1 = T.vdphi[q][j][1];
      acc[j] += H00 * d0 + H01 * d1;
      acc[NS + j] += H10 * d0 + H11 * d1;
    }
  }
  // ---- facet terms
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    const int tn = m.tri_nbr[size_t(t) * 3 + e];
    if (tn < 0) {
      // a wall adds no term (u.n = 0 there; SIPG on interior facets only); inflow and outflow
      // facets add the convective flux against the exterior state (Sec. 2.5)
      if (m.facet_kind) boundary_flux<K, R>(m, T, t, e, Ji, s, up, acc);
      continue;
    }
    const int en = m.tri_nbr_loc[size_t(t) * 3 + e];
    const double* geon = m.geo + size_t(m.tri_class[tn]) * kGeo;
    const R sn = R(geon[G_S]);
    const R n0 = R(geo[G_NRM + 2 * e]), n1 = R(geo[G_NRM + 2 * e + 1]);
    const R len = R(geo[G_FLEN + e]);
    const R sig = R(m.facet_sigma[m.tri_facet[size_t(t) * 3 + e]]);
    // normal derivative in reference gradients: d_n psi = s sum_r d_r psihat (Jinv n)_r
    const R mo0 = Ji[0] * n0 + Ji[1] * n1, mo1 = Ji[2] * n0 + Ji[3] * n1;
    const R mn0 = R(geon[G_JINV + 0]) * n0 + R(geon[G_JINV + 1]) * n1;
    const R mn1 = R(geon[G_JINV + 2]) * n0 + R(geon[G_JINV + 3]) * n1;
    R un[D::ND];
    load_coef<D::ND>(ug + size_t(tn) * D::ND, un);
#pragma unroll 1
    for (int q = 0; q < D::NQF; ++q) {
      const int qn = D::NQF - 1 - q;
      R ui0 = 0, ui1 = 0, di0 = 0, di1 = 0, uo0 = 0, uo1 = 0, do0 = 0, do1 = 0;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const R ph = T.fphi[e][q][j];
        const R dn = T.fdphi[e][q][j][0] * mo0 + T.fdphi[e][q][j][1] * mo1;
        ui0 += ph * up[j];
        ui1 += ph * up[NS + j];
        di0 += dn * up[j];
        di1 += dn * up[NS + j];
        const R phn = T.fphi[en][qn][j];
        const R dnn = T.fdphi[en][qn][j][0] * mn0 + T.fdphi[en][qn][j][1] * mn1;
        uo0 += phn * un[j];
        uo1 += phn * un[NS + j];
        do0 += dnn * un[j];
        do1 += dnn * un[NS + j];
      }
      ui0 *= s;
      ui1 *= s;
      di0 *= s;
      di1 *= s;
      uo0 *= sn;
      uo1 *= sn;
      do0 *= sn;
      do1 *= sn;
      const R vn = R(0.5) * ((ui0 + uo0) * n0 + (ui1 + uo1) * n1);
      const R w0 = vn >= R(0) ? ui0 : uo0, w1 = vn >= R(0) ? ui1 : uo1;
      const R j0 = ui0 - uo0, j1 = ui1 - uo1;
      const R w = T.fw[q] * len * s;
      const R A0 = w * (-vn * w0 + nu * R(0.5) * (di0 + do0) - nu * sig * j0);
      const R A1 = w * (-vn * w1 + nu * R(0.5) * (di1 + do1) - nu * sig * j1);
      const R B0 = w * R(0.5) * nu * j0, B1 = w * R(0.5) * nu * j1;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const R ph = T.fphi[e][q][j];
        const R dn = T.fdphi[e][q][j][0] * mo0 + T.fdphi[e][q][j][1] * mo1;
        acc[j] += A0 * ph + B0 * dn;
        acc[NS + j] += A1 * ph + B1 * dn;
      }
    }
  }
}

// Transposed Jacobian of the residual (adjoint of the stage functional): for the
// state u and a functional w (coefficients), out = c_w w + c_J J_L(u)^T w with
//   (J_L(u)^T w)_j = d/du_j L(u)(w)
//     volume : int psi_j [(u.grad) w + (grad w)^T u]_c - nu int grad psi_j . grad w_c
//     facets : -int psi_j [n_c (u^up . [w]) / 2 + max(u.n, 0) [w]_c]        (upwind flux in its
//              1/2 (u.n)(u+ + u-) + 1/2 |u.n| (u+ - u-) form, sign(0) = 0)
//              + nu int [psi_j ({d_n w}_c - sigma [w]_c) + 1/2 d_n psi_j [w]_c]  (SIPG, symmetric)
// with [w] = w_T - w_neighbour and n the outward normal of T. The viscous part is the
// SIPG residual of w itself (eq. (18) is symmetric). Block partials of
// <u, dL/dnu(u)> = B_h(u, w)/nu with the sign of L, i.e. the nu-derivative of
// L(u)(w), go to red[blockIdx].
template <int K>
__device__ void element_adjoint(const DevMesh& m, const SmemTables<K, double>& T, int t, const double* __restrict__ ug,
                                const double* __restrict__ wg, double (&acc)[Dims<K>::ND], double& nupart) {
  using D = Dims<K>;
  constexpr int NS = D::NS, ND = D::ND;
  const double nu = m.nu;
  const double* geo = m.geo + size_t(m.tri_class[t]) * kGeo;
  const double Ji[4] = {geo[G_JINV + 0], geo[G_JINV + 1], geo[G_JINV + 2], geo[G_JINV + 3]};
  const double det = geo[G_DET], s = geo[G_S];
  double uc[ND], wc[ND];
  load_coef<ND>(ug + size_t(t) * ND, uc);
  load_coef<ND>(wg + size_t(t) * ND, wc);
#pragma unroll
  for (int i = 0; i < ND; ++i) acc[i] = 0.0;
  nupart = 0.0;
#pragma unroll 1
  for (int q = 0; q < D::NQ; ++q) {
    double u0 = 0, u1 = 0, a[2][2] = {{0, 0}, {0, 0}}, b[2][2] = {{0, 0}, {0, 0}};
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const double ph = T.vphi[q][j], d0 = T.vdphi[q][j][0], d1 = T.vdphi[q][j][1];
      u0 += ph * uc[j];
      u1 += ph * uc[NS + j];
      a[0][0] += d0 * wc[j];
      a[0][1] += d1 * wc[j];
      a[1][0] += d0 * wc[NS + j];
      a[1][1] += d1 * wc[NS + j];
      b[0][0] += d0 * uc[j];
      b[0][1] += d1 * uc[j];
      b[1][0] += d0 * uc[NS + j];
      b[1][1] += d1 * uc[NS + j];
    }
    u0 *= s;
    u1 *= s;
    double gw[2][2], gu[2][2];   // physical gradients d w_c / d x_d, d u_c / d x_d
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      gw[c][0] = s * (a[c][0] * Ji[0] + a[c][1] * Ji[2]);
      gw[c][1] = s * (a[c][0] * Ji[1] + a[c][1] * Ji[3]);
      gu[c][0] = s * (b[c][0] * Ji[0] + b[c][1] * Ji[2]);
      gu[c][1] = s * (b[c][0] * Ji[1] + b[c][1] * Ji[3]);
    }
    const double w = T.vw[q] * det;
    // value-type test terms A_c = (u.grad) w_c + sum_d u_d d_c w_d
    const double A0 = w * s * (u0 * gw[0][0] + u1 * gw[0][1] + u0 * gw[0][0] + u1 * gw[1][0]);
    const double A1 = w * s * (u0 * gw[1][0] + u1 * gw[1][1] + u0 * gw[0][1] + u1 * gw[1][1]);
    // gradient-type test terms: -nu grad w_c . grad psi_j, written through reference gradients
    const double H00 = -w * s * nu * (gw[0][0] * Ji[0] + gw[0][1] * Ji[1]);
    const double H01 = -w * s * nu * (gw[0][0] * Ji[2] + gw[0][1] * Ji[3]);
    const double H10 = -w * s * nu * (gw[1][0] * Ji[0] + gw[1][1] * Ji[1]);
    const double H11 = -w * s * nu * (gw[1][0] * Ji[2] + gw[1][1] * Ji[3]);
    nupart -= w * (gu[0][0] * gw[0][0] + gu[0][1] * gw[0][1] + gu[1][0] * gw[1][0] + gu[1][1] * gw[1][1]);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      const double ph = T.vphi[q][j], d0 = T.vdphi[q][j][0], d1 = T.vdphi[q][j][1];
      acc[j] += A0 * ph + H00 * d0 + H01 * d1;
      acc[NS + j] += A1 * ph + H10 * d0 + H11 * d1;
    }
  }
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    const int tn = m.tri_nbr[size_t(t) * 3 + e];
    if (tn < 0) continue;   // walls: no term in the forward residual, none in its transpose
    const int en = m.tri_nbr_loc[size_t(t) * 3 + e];
    const double* geon = m.geo + size_t(m.tri_class[tn]) * kGeo;
    const double sn = geon[G_S];
    const double n0 = geo[G_NRM + 2 * e], n1 = geo[G_NRM + 2 * e + 1];
    const double len = geo[G_FLEN + e];
    const double sig = m.facet_sigma[m.tri_facet[size_t(t) * 3 + e]];
    const double mo0 = Ji[0] * n0 + Ji[1] * n1, mo1 = Ji[2] * n0 + Ji[3] * n1;
    const double mn0 = geon[G_JINV + 0] * n0 + geon[G_JINV + 1] * n1;
    const double mn1 = geon[G_JINV + 2] * n0 + geon[G_JINV + 3] * n1;
    double un[ND], wn[ND];
    load_coef<ND>(ug + size_t(tn) * ND, un);
    load_coef<ND>(wg + size_t(tn) * ND, wn);
#pragma unroll 1
    for (int q = 0; q < D::NQF; ++q) {
      const int qn = D::NQF - 1 - q;
      double ui[2] = {0, 0}, uo[2] = {0, 0}, wi[2] = {0, 0}, wo[2] = {0, 0};
      double dwi[2] = {0, 0}, dwo[2] = {0, 0}, dui[2] = {0, 0};
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const double ph = T.fphi[e][q][j];
        const double dn = T.fdphi[e][q][j][0] * mo0 + T.fdphi[e][q][j][1] * mo1;
        const double phn = T.fphi[en][qn][j];
        const double dnn = T.fdphi[en][qn][j][0] * mn0 + T.fdphi[en][qn][j][1] * mn1;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          ui[c] += ph * uc[c * NS + j];
          wi[c] += ph * wc[c * NS + j];
          dwi[c] += dn * wc[c * NS + j];
          dui[c] += dn * uc[c * NS + j];
          uo[c] += phn * un[c * NS + j];
          wo[c] += phn * wn[c * NS + j];
          dwo[c] += dnn * wn[c * NS + j];
        }
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        ui[c] *= s;
        wi[c] *= s;
        dwi[c] *= s;
        dui[c] *= s;
        uo[c] *= sn;
        wo[c] *= sn;
        dwo[c] *= sn;
      }
      const double vn = 0.5 * ((ui[0] + uo[0]) * n0 + (ui[1] + uo[1]) * n1);
      const double sg = vn > 0.0 ? 1.0 : (vn < 0.0 ? -1.0 : 0.0);
      const double up0 = 0.5 * ((ui[0] + uo[0]) + sg * (ui[0] - uo[0]));
      const double up1 = 0.5 * ((ui[1] + uo[1]) + sg * (ui[1] - uo[1]));
      const double jw0 = wi[0] - wo[0], jw1 = wi[1] - wo[1];
      const double upj = up0 * jw0 + up1 * jw1;
      const double vp = vn > 0.0 ? vn : 0.0;
      const double w = T.fw[q] * len;
      // value-type: convective adjoint + SIPG consistency and penalty of w (nu)
      // u.n is the average of both traces: d(u.n)/du_T = n/2
      const double A0 = w * s * (-(0.5 * n0 * upj + vp * jw0) + nu * (0.5 * (dwi[0] + dwo[0]) - sig * jw0));
      const double A1 = w * s * (-(0.5 * n1 * upj + vp * jw1) + nu * (0.5 * (dwi[1] + dwo[1]) - sig * jw1));
      // normal-derivative test: SIPG symmetry term
      const double B0 = w * s * 0.5 * nu * jw0, B1 = w * s * 0.5 * nu * jw1;
      nupart += w * (ui[0] * (0.5 * (dwi[0] + dwo[0]) - sig * jw0) + ui[1] * (0.5 * (dwi[1] + dwo[1]) - sig * jw1) +
                     0.5 * (dui[0] * jw0 + dui[1] * jw1));
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const double ph = T.fphi[e][q][j];
        const double dn = T.fdphi[e][q][j][0] * mo0 + T.fdphi[e][q][j][1] * mo1;
        acc[j] += A0 * ph + B0 * dn;
        acc[NS + j] += A1 * ph + B1 * dn;
      }
    }
  }
}

template <int K>
__global__ void __launch_bounds__(128) k_adjoint(DevMesh m, const double* u, const double* w, double* out, double cw,
                                                 double cj, int accumulate) {
  using D = Dims<K>;
  constexpr int ND = D::ND;
  __shared__ SmemTables<K, double> T;
  load_tables<K, double>(m, T);
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double nupart = 0.0;
  if (t < m.n_tri) {
    double acc[ND];
    element_adjoint<K>(m, T, t, u, w, acc, nupart);
#pragma unroll
    for (int i = 0; i < ND; ++i) {
      const size_t o = size_t(t) * ND + i;
      const double v = cw * w[o] + cj * acc[i];
      out[o] = accumulate ? out[o] + v : v;
    }
  }
  nupart = block_sum(nupart);
  if (threadIdx.x == 0) m.red[blockIdx.x] = nupart;
}

// acc_dev += coef * (sum of the k_adjoint block partials), in fixed order.
__global__ void k_nu_accumulate(DevMesh m, int nparts, double coef, double* acc_dev) {
  if (threadIdx.x >= 32) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) v += m.red[i];
  v = warp_sum(v);
  if (threadIdx.x == 0) *acc_dev += coef * v;
}

// Stage kernel, FP64 form (the mixed form's is k_stage_df in k_stage_df.cu).
// Modes (StageMode): the stage functional and its condensation (h = P f,
// gl = G f), the residual alone, the pressure functional, or the projection
// functional.
template <int K, typename R>
__global__ void __launch_bounds__(128) k_stage(DevMesh m, StageArgs a) {
  using D = Dims<K>;
  constexpr int ND = D::ND, L3 = 3 * D::NL;
  __shared__ SmemTables<K, R> T;
  load_tables<K, R>(m, T);
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tri) return;
  R up[ND];
  load_coef<ND>(a.up + size_t(t) * ND, up);
  R f[ND];
  if (a.mode == MODE_PROJECT) {
#pragma unroll
    for (int i = 0; i < ND; ++i) f[i] = up[i];
  } else {
    element_residual<K, R>(m, T, t, a.up, up, f);
    if (a.mode == MODE_STAGE) {
      R un[ND];
      load_coef<ND>(a.un + size_t(t) * ND, un);
      const R ca = R(a.a), cb = R(a.b), cc = R(a.c);
#pragma unroll
      for (int i = 0; i < ND; ++i) f[i] = ca * un[i] + cb * up[i] + cc * f[i];
    }
  }
  if (a.mode == MODE_RESIDUAL || a.mode == MODE_PRESSURE) {
#pragma unroll
    for (int i = 0; i < ND; ++i) m.h[size_t(t) * ND + i] = double(f[i]);
  }
  if (a.mode == MODE_RESIDUAL) return;
  const int c = m.tri_class[t];
  if (a.mode != MODE_PRESSURE) {
    for (int i = 0; i < ND; ++i) {
      R v = R(0);
#pragma unroll
      for (int j = 0; j < ND; ++j) v += m.P[(size_t(c) * ND + i) * ND + j] * f[j];
      m.h[size_t(t) * ND + i] = double(v);
    }
  }
  for (int i = 0; i < L3; ++i) {
    R v = R(0);
#pragma unroll
    for (int j = 0; j < ND; ++j) v += m.G[(size_t(c) * L3 + i) * ND + j] * f[j];
    m.gl[size_t(t) * L3 + i] = double(v);
  }
}

// Recovery (eq. (12) eliminated locally): u_T = P_T f_T - G_T^T lam_T, with
// lam_T the multipliers of T's three facets mapped to T's own orientation.
template <int K>
__global__ void __launch_bounds__(128) k_recover(DevMesh m, double* out) {
  using D = Dims<K>;
  constexpr int ND = D::ND, NL = D::NL, L3 = 3 * NL;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tri) return;
  double lam[L3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int f = m.tri_facet[size_t(t) * 3 + e];
    const bool flip = m.tri_orient[size_t(t) * 3 + e] < 0;
#pragma unroll
    for (int mm = 0; mm < NL; ++mm) {
      const double v = m.lam[size_t(f) * NL + mm];
      lam[e * NL + mm] = (flip && (mm & 1)) ? -v : v;
    }
  }
  const double* G = m.G + size_t(m.tri_class[t]) * L3 * ND;
#pragma unroll 4
  for (int i = 0; i < ND; ++i) {
    double v = m.h[size_t(t) * ND + i];
#pragma unroll
    for (int l = 0; l < L3; ++l) v -= G[l * ND + i] * lam[l];
    out[size_t(t) * ND + i] = v;
  }
}

// Element pressure w_T = W_T f_T - (W C^T)_T lam_T; block partial sums of the
// integral of w for the L^2_0 shift go to red[0][block].
template <int K>
__global__ void __launch_bounds__(128) k_pressure(DevMesh m, double* w) {
  using D = Dims<K>;
  constexpr int ND = D::ND, NL = D::NL, L3 = 3 * NL, NW = D::NW;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double integral = 0.0;
  if (t < m.n_tri) {
    double lam[L3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int f = m.tri_facet[size_t(t) * 3 + e];
      const bool flip = m.tri_orient[size_t(t) * 3 + e] < 0;
#pragma unroll
      for (int mm = 0; mm < NL; ++mm) {
        const double v = m.lam[size_t(f) * NL + mm];
        lam[e * NL + mm] = (flip && (mm & 1)) ? -v : v;
      }
    }
    const int c = m.tri_class[t];
    const double* W = m.W + size_t(c) * NW * ND;
    const double* WC = m.WCt + size_t(c) * NW * L3;
    for (int i = 0; i < NW; ++i) {
      double v = 0.0;
      for (int j = 0; j < ND; ++j) v += W[i * ND + j] * m.h[size_t(t) * ND + j];
      for (int l = 0; l < L3; ++l) v -= WC[i * L3 + l] * lam[l];
      w[size_t(t) * NW + i] = v;
    }
    integral = w[size_t(t) * NW] * m.geo[size_t(c) * kGeo + G_ZINT0];
  }
  integral = block_sum(integral);
  if (threadIdx.x == 0) m.red[blockIdx.x] = integral;
}

// Lattice output of the shifted pressure: c = (integral of w) / |Omega| from the
// block partials, w <- w - c, lam <- lam - c (the constant is mode 0 on facets).
template <int K>
__global__ void __launch_bounds__(128) k_pressure_lattice(DevMesh m, const double* w, double* pe, double* pf,
                                                          int nparts) {
  using D = Dims<K>;
  constexpr int NW = D::NW, NL = D::NL;
  __shared__ double cshift;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) v += m.red[i];
    v = warp_sum(v);
    // with outflow facets p = 0 there fixes the constant (eq. (be)): no shift
    if (threadIdx.x == 0) cshift = m.has_kernel ? v / m.area_total : 0.0;
  }
  __syncthreads();
  const double c = cshift;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m.n_tri) {
    const double* geo = m.geo + size_t(m.tri_class[i]) * kGeo;
    double wl[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) wl[j] = w[size_t(i) * NW + j];
    wl[0] -= c * geo[G_CINV0];
    const double s = geo[G_S];
#pragma unroll
    for (int p = 0; p < NW; ++p) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < NW; ++j) v += m.plat_phi[p * NW + j] * wl[j];
      pe[size_t(i) * NW + p] = s * v;
    }
  }
  if (pf && i < m.n_facet) {
    const int fo = m.facet_ext ? m.facet_ext[i] : i;
    double lam[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) lam[j] = m.lam[size_t(i) * NL + j];
    lam[0] -= c;
#pragma unroll
    for (int p = 0; p < NL; ++p) {
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < NL; ++j) v += m.mu_lat[p * NL + j] * lam[j];
      pf[size_t(fo) * NL + p] = v;
    }
  }
}

// Lattice values -> orthonormal coefficients: coef = sqrt(det) Vhat^-1 vals per component.
template <int K>
__global__ void k_lattice_to_coef(DevMesh m, const double* vals, double* coef) {
  using D = Dims<K>;
  constexpr int NS = D::NS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tri) return;
  const double sq = 1.0 / m.geo[size_t(m.tri_class[t]) * kGeo + G_S];
  double v[NS][2];
#pragma unroll
  for (int p = 0; p < NS; ++p) {
    v[p][0] = vals[(size_t(t) * NS + p) * 2];
    v[p][1] = vals[(size_t(t) * NS + p) * 2 + 1];
  }
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    double c0 = 0.0, c1 = 0.0;
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      c0 += m.lat_inv[j * NS + p] * v[p][0];
      c1 += m.lat_inv[j * NS + p] * v[p][1];
    }
    coef[size_t(t) * 2 * NS + j] = sq * c0;
    coef[size_t(t) * 2 * NS + NS + j] = sq * c1;
  }
}

template <int K>
__global__ void k_coef_to_lattice(DevMesh m, const double* coef, double* vals) {
  using D = Dims<K>;
  constexpr int NS = D::NS;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.n_tri) return;
  const double s = m.geo[size_t(m.tri_class[t]) * kGeo + G_S];
  double c[2 * NS];
#pragma unroll
  for (int i = 0; i < 2 * NS; ++i) c[i] = coef[size_t(t) * 2 * NS + i];
#pragma unroll
  for (int p = 0; p < NS; ++p) {
    double v0 = 0.0, v1 = 0.0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      v0 += m.lat_phi[p * NS + j] * c[j];
      v1 += m.lat_phi[p * NS + j] * c[NS + j];
    }
    vals[(size_t(t) * NS + p) * 2] = s * v0;
    vals[(size_t(t) * NS + p) * 2 + 1] = s * v1;
  }
}

// The same conversions for the mixed form, in double-float arithmetic on the FP32 pipes (the
// FP64 pipe, 1/64 of the FP32 rate here, only splits the inputs and rounds the outputs). The
// tables are split into double-float pairs once per block; a block's 128 triangles pass through
// shared memory, so that global reads and writes are coalesced.
constexpr int kConvTris = 128;

template <int K>
__global__ void __launch_bounds__(kConvTris) k_lattice_to_coef_df(DevMesh m, const double* vals, double* coef) {
  using D = Dims<K>;
  constexpr int NS = D::NS, NV = 2 * NS, RS = NV + 1;
  __shared__ float2 tab[NS * NS];
  __shared__ double tile[kConvTris * RS];
  for (int i = threadIdx.x; i < NS * NS; i += kConvTris) tab[i] = to_float2(dfl(m.lat_inv[i]));
  const int t0 = blockIdx.x * kConvTris;
  const int nt = min(kConvTris, m.n_tri - t0);
  const double* vb = vals + size_t(t0) * NV;
  for (int e = threadIdx.x; e < nt * NV; e += kConvTris) tile[(e / NV) * RS + e % NV] = vb[e];
  __syncthreads();
  if (int(threadIdx.x) < nt) {
    const int t = t0 + threadIdx.x;
    const dfl sq(1.0 / m.geo[size_t(m.tri_class[t]) * kGeo + G_S]);
    double* row = tile + threadIdx.x * RS;
    dfl v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = dfl(row[i]);   // [p][c]
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      dacc c0 = dacc_zero(), c1 = dacc_zero();
#pragma unroll
      for (int p = 0; p < NS; ++p) {
        const dfl a = to_dfl(tab[j * NS + p]);
        mad(c0, a, v[2 * p]);
        mad(c1, a, v[2 * p + 1]);
      }
      row[j] = to_double(sq * val(c0));
      row[NS + j] = to_double(sq * val(c1));
    }
  }
  __syncthreads();
  double* cb = coef + size_t(t0) * NV;
  for (int e = threadIdx.x; e < nt * NV; e += kConvTris) cb[e] = tile[(e / NV) * RS + e % NV];
}

template <int K>
__global__ void __launch_bounds__(kConvTris) k_coef_to_lattice_df(DevMesh m, const double* coef, double* vals) {
  using D = Dims<K>;
  constexpr int NS = D::NS, NV = 2 * NS, RS = NV + 1;
  __shared__ float2 tab[NS * NS];
  __shared__ double tile[kConvTris * RS];
  for (int i = threadIdx.x; i < NS * NS; i += kConvTris) tab[i] = to_float2(dfl(m.lat_phi[i]));
  const int t0 = blockIdx.x * kConvTris;
  const int nt = min(kConvTris, m.n_tri - t0);
  const double* cb = coef + size_t(t0) * NV;
  for (int e = threadIdx.x; e < nt * NV; e += kConvTris) tile[(e / NV) * RS + e % NV] = cb[e];
  __syncthreads();
  if (int(threadIdx.x) < nt) {
    const int t = t0 + threadIdx.x;
    const dfl sc(m.geo[size_t(m.tri_class[t]) * kGeo + G_S]);
    double* row = tile + threadIdx.x * RS;
    dfl c[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) c[i] = dfl(row[i]);   // [c][j]
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      dacc v0 = dacc_zero(), v1 = dacc_zero();
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const dfl a = to_dfl(tab[p * NS + j]);
        mad(v0, a, c[j]);
        mad(v1, a, c[NS + j]);
      }
      row[2 * p] = to_double(sc * val(v0));
      row[2 * p + 1] = to_double(sc * val(v1));
    }
  }
  __syncthreads();
  double* vb = vals + size_t(t0) * NV;
  for (int e = threadIdx.x; e < nt * NV; e += kConvTris) vb[e] = tile[(e / NV) * RS + e % NV];
}

// Diagnostics partials per block: red[0] energy, red[1] enstrophy, red[2] max |div|,
// red[3] max |[u.n]| (each facet is seen from both sides).
template <int K>
__global__ void __launch_bounds__(128) k_diagnostics(DevMesh m, const double* coef) {
  using D = Dims<K>;
  constexpr int NS = D::NS, ND = D::ND;
  __shared__ SmemTables<K, double> T;
  load_tables<K, double>(m, T);
  __syncthreads();
  double en = 0.0, ens = 0.0, dmax = 0.0, jmax = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.n_tri; t += gridDim.x * blockDim.x) {
    double c[ND];
    load_coef<ND>(coef + size_t(t) * ND, c);
#pragma unroll
    for (int i = 0; i < ND; ++i) en += c[i] * c[i];
    const double* geo = m.geo + size_t(m.tri_class[t]) * kGeo;
    const double Ji[4] = {geo[0], geo[1], geo[2], geo[3]};
    const double det = geo[G_DET], s = geo[G_S];
    for (int q = 0; q < D::NQ; ++q) {
      double a00 = 0, a01 = 0, a10 = 0, a11 = 0;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        a00 += T.vdphi[q][j][0] * c[j];
        a01 += T.vdphi[q][j][1] * c[j];
        a10 += T.vdphi[q][j][0] * c[NS + j];
        a11 += T.vdphi[q][j][1] * c[NS + j];
      }
      const double g00 = s * (a00 * Ji[0] + a01 * Ji[2]), g01 = s * (a00 * Ji[1] + a01 * Ji[3]);
      const double g10 = s * (a10 * Ji[0] + a11 * Ji[2]), g11 = s * (a10 * Ji[1] + a11 * Ji[3]);
      const double om = g10 - g01;
      ens += T.vw[q] * det * om * om;
      dmax = fmax(dmax, fabs(g00 + g11));
    }
    for (int e = 0; e < 3; ++e) {
      // on a wall the jump is u.n itself: the missing side counts as zero; on an inflow facet
      // it is (u - u_in).n; on an outflow facet u.n is free (Sec. 2.5)
      const int tnr = m.tri_nbr[size_t(t) * 3 + e];
      const int fid = m.tri_facet[size_t(t) * 3 + e];
      const int kd = (tnr < 0 && m.facet_kind) ? int(m.facet_kind[fid]) : int(kFacetWall);
      if (kd == kFacetOutflow) continue;
      const bool canon = m.tri_orient[size_t(t) * 3 + e] > 0;
      const int tn = tnr < 0 ? t : tnr;
      const int el = tnr < 0 ? e : m.tri_nbr_loc[size_t(t) * 3 + e];
      const double sn = tnr < 0 ? 0.0 : m.geo[size_t(m.tri_class[tn]) * kGeo + G_S];
      const double n0 = geo[G_NRM + 2 * e], n1 = geo[G_NRM + 2 * e + 1];
      double cn[ND];
      load_coef<ND>(coef + size_t(tn) * ND, cn);
      for (int q = 0; q < D::NQF; ++q) {
        const int qn = D::NQF - 1 - q;
        double a0 = 0, a1 = 0, b0 = 0, b1 = 0;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          a0 += T.fphi[e][q][j] * c[j];
          a1 += T.fphi[e][q][j] * c[NS + j];
          b0 += T.fphi[el][qn][j] * cn[j];
          b1 += T.fphi[el][qn][j] * cn[NS + j];
        }
        double x0 = sn * b0, x1 = sn * b1;
        if (kd == kFacetInflow) {
          const double* uq = m.inflow_q + (size_t(fid) * D::NQF + (canon ? q : qn)) * 2;
          x0 = uq[0];
          x1 = uq[1];
        }
        jmax = fmax(jmax, fabs((s * a0 - x0) * n0 + (s * a1 - x1) * n1));
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

__global__ void k_diag_finish(DevMesh m, int nparts) {
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

__global__ void k_check_finite(const double* v, long long n, int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, kFlagNonFinite);
}

__global__ void __launch_bounds__(256) k_energy_part(const double* u, long long n, double* part) {
  double a = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = __ldcg(&u[i]);
    a = fma(v, v, a);
  }
  a = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void k_energy_watch(double* watch, int nparts, double tol, DevStats* st) {
  if (threadIdx.x >= 32) return;
  double e = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) e += watch[2 + i];
  e = warp_sum(e);
  if (threadIdx.x == 0) {
    const double prev = watch[0];
    if (prev >= 0.0) {
      watch[1] = prev > 0.0 ? e / prev : (e > 0.0 ? INFINITY : 1.0);
      if (!(e <= prev * (1.0 + tol))) atomicOr(&st->flags, kFlagEnergyGrowth);
    }
    watch[0] = e;
  }
}

// ------------------------------------------------------------------- launchers
namespace {
inline int blocks_for(long long n, int bs) { return int((n + bs - 1) / bs); }
}

#define DGDF_DISPATCH_K(kv, CALL) \
  switch (kv) {                   \
    case 1: { constexpr int K = 1; CALL; break; } \
    case 2: { constexpr int K = 2; CALL; break; } \
    case 3: { constexpr int K = 3; CALL; break; } \
    default: return cudaErrorInvalidValue;        \
  }

// Lattice conversions: FP64 arithmetic in the FP64 form, double-float in the mixed form.
cudaError_t launch_lattice_to_coef(const DevMesh& m, const double* vals, double* coef, cudaStream_t s) {
  if (m.elem_df)
    DGDF_DISPATCH_K(m.k, (k_lattice_to_coef_df<K><<<blocks_for(m.n_tri, kConvTris), kConvTris, 0, s>>>(m, vals, coef)))
  else
    DGDF_DISPATCH_K(m.k, (k_lattice_to_coef<K><<<blocks_for(m.n_tri, 128), 128, 0, s>>>(m, vals, coef)))
  return cudaGetLastError();
}

cudaError_t launch_coef_to_lattice(const DevMesh& m, const double* coef, double* vals, cudaStream_t s) {
  if (m.elem_df)
    DGDF_DISPATCH_K(m.k, (k_coef_to_lattice_df<K><<<blocks_for(m.n_tri, kConvTris), kConvTris, 0, s>>>(m, coef, vals)))
  else
    DGDF_DISPATCH_K(m.k, (k_coef_to_lattice<K><<<blocks_for(m.n_tri, 128), 128, 0, s>>>(m, coef, vals)))
  return cudaGetLastError();
}

cudaError_t launch_stage(const DevMesh& m, const StageArgs& a, cudaStream_t s) {
  if (m.elem_df) return launch_stage_df(m, a, s);
  DGDF_DISPATCH_K(m.k, (k_stage<K, double><<<blocks_for(m.n_tri, 128), 128, 0, s>>>(m, a)));
  return cudaGetLastError();
}

cudaError_t launch_recover(const DevMesh& m, double* out, float2* out_df, cudaStream_t s) {
  if (m.elem_df) return launch_recover_df(m, out, out_df, s);
  DGDF_DISPATCH_K(m.k, (k_recover<K><<<blocks_for(m.n_tri, 128), 128, 0, s>>>(m, out)));
  return cudaGetLastError();
}

cudaError_t launch_pressure(const DevMesh& m, double* w, cudaStream_t s) {
  DGDF_DISPATCH_K(m.k, (k_pressure<K><<<blocks_for(m.n_tri, 128), 128, 0, s>>>(m, w)));
  return cudaGetLastError();
}

cudaError_t launch_pressure_lattice(const DevMesh& m, const double* w, double* pe, double* pf, cudaStream_t s) {
  const int nparts = blocks_for(m.n_tri, 128);
  const long long n = m.n_tri > m.n_facet ? m.n_tri : m.n_facet;
  DGDF_DISPATCH_K(m.k, (k_pressure_lattice<K><<<blocks_for(n, 128), 128, 0, s>>>(m, w, pe, pf, nparts)));
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(const DevMesh& m, const double* coef, cudaStream_t s) {
  int nb = blocks_for(m.n_tri, 128);
  if (nb > kMaxSolverBlocks) nb = kMaxSolverBlocks;
  DGDF_DISPATCH_K(m.k, (k_diagnostics<K><<<nb, 128, 0, s>>>(m, coef)));
  k_diag_finish<<<1, 32, 0, s>>>(m, nb);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const DevMesh& m, const double* u, const double* w, double* out, double cw, double cj,
                           int accumulate, double nu_coef, double* nu_acc, cudaStream_t s) {
  const int nb = blocks_for(m.n_tri, 128);
  DGDF_DISPATCH_K(m.k, (k_adjoint<K><<<nb, 128, 0, s>>>(m, u, w, out, cw, cj, accumulate)));
  k_nu_accumulate<<<1, 32, 0, s>>>(m, nb, nu_coef, nu_acc);
  return cudaGetLastError();
}

cudaError_t launch_energy_watch(const double* u, long long n, double* watch, double tol, DevStats* st,
                                cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  k_energy_part<<<int(nb), 256, 0, s>>>(u, n, watch + 2);
  k_energy_watch<<<1, 32, 0, s>>>(watch, int(nb), tol, st);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* v, long long n, int* flag, cudaStream_t s) {
  long long nb = (n + 255) / 256;
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  k_check_finite<<<int(nb), 256, 0, s>>>(v, n, flag);
  return cudaGetLastError();
}

}  // namespace dgdf
