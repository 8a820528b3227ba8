// Element kernels of the mixed form: the stage residual + condensation (K1-K3)
// and the recovery (K5) in double-float arithmetic on the FP32 units.
//
// Two threads per triangle, one per velocity component c: the residual of
// eq. (7) + eq. (18) couples the components only through u (x) u and the normal
// velocity u.n, which the pair exchanges by warp shuffles at every quadrature
// point; every sum over basis functions belongs to one component. This halves
// the registers a thread holds (its component's coefficients, its neighbour
// traces and its accumulators) against one thread per triangle, so twice as many
// warps hide the FP32 latency. Inputs are the double-float twins of u^n and u'
// (no FP64 conversions on this path); sums of products use the compensated
// accumulator dacc (12 FP32 operations per multiply-add).
#include <algorithm>

#include "device.cuh"
#include "dfloat.cuh"
#include "kcommon.cuh"
#include "ktables.cuh"

namespace dgdf {

// 192 threads (96 triangles) per block and two blocks per SM leave 168 registers a thread,
// enough for either stage kernel at k = 3 without spills.
constexpr int kStageDfThreads = 192;

namespace {

__device__ __forceinline__ dfl shfl_pair(dfl v) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}

template <int N>
__device__ __forceinline__ void load_df(const float2* __restrict__ p, dfl (&c)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) c[i] = to_dfl(p[i]);
}

// Inflow and outflow facets of triangle t (Sec. 2.5, eq. (be)), component c: the convective
// flux of eq. (7) with u.n the average of the interior trace and the exterior state, which is
// u_in on an inflow facet (stored at the facet points in the canonical direction: our point q
// is its point q, or NQF-1-q when the triangle runs the facet the other way) and the interior
// trace on an outflow facet, and the upwind value from the side u.n leaves. The viscous form
// has no boundary terms. Whether a facet is taken depends on t alone, so both threads of a
// pair take it together, and they exchange u.n through a shuffle over the pair only. ui(e, q)
// returns the interior trace of component c; add(e, q, F) adds -w_q F phi_j(e, q) to acc.
template <int NQF, typename Trace, typename Add>
__device__ __forceinline__ void boundary_terms(const DevMesh& m, const float2* geo, int t, int c, dfl s, Trace ui,
                                               Add add) {
  const unsigned pair_mask = 3u << ((threadIdx.x & 31) & ~1u);
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    if (__ldg(&m.tri_nbr[size_t(t) * 3 + e]) >= 0) continue;
    const int fid = __ldg(&m.tri_facet[size_t(t) * 3 + e]);
    const int kd = __ldg(&m.facet_kind[fid]);
    if (kd == kFacetWall) continue;
    const bool canon = __ldg(&m.tri_orient[size_t(t) * 3 + e]) > 0;
    const dfl nc = to_dfl(geo[G_NRM + 2 * e + c]);
    const dfl lens = to_dfl(geo[G_FLEN + e]) * s;
#pragma unroll 1
    for (int q = 0; q < NQF; ++q) {
      const dfl u = ui(e, q);
      const dfl uo =
          kd == kFacetInflow ? dfl(__ldg(&m.inflow_q[(size_t(fid) * NQF + (canon ? q : NQF - 1 - q)) * 2 + c])) : u;
      const dfl pc = (u + uo) * nc;
      const dfl po(__shfl_xor_sync(pair_mask, pc.hi, 1), __shfl_xor_sync(pair_mask, pc.lo, 1));
      const dfl vn = half(c ? po + pc : pc + po);
      const dfl wup = vn >= dfl(0) ? u : uo;
      add(e, q, lens * vn * wup);
    }
  }
}

// acc[j] += the component-c part of L(u')(phi_j): -C_h(u;u,phi) - B_h(u,phi) of
// eq. (7) and eq. (18). Volume: int (u_c u - nu grad u_c) . grad phi_j. Facets: the
// upwind flux (u.n) u_c^up with u.n the average of both traces, and the SIPG
// consistency, symmetry and penalty terms, at the facet Gauss points (the
// neighbour's point q is our point NQF-1-q).
template <int K>
__device__ __forceinline__ void residual_component(const DevMesh& m, const SmemTables<K, dfl>& T, int t, int c,
                                                   const float2* __restrict__ ug, const dfl (&up)[Dims<K>::NS],
                                                   dacc (&acc)[Dims<K>::NS]) {
  using D = Dims<K>;
  constexpr int NS = D::NS, ND = D::ND;
  const dfl nu(m.nu);
  const int cls = __ldg(&m.tri_class[t]);
  const float2* geo = m.geo_df + size_t(cls) * kGeo;
  const dfl Ji0 = to_dfl(geo[G_JINV + 0]), Ji1 = to_dfl(geo[G_JINV + 1]);
  const dfl Ji2 = to_dfl(geo[G_JINV + 2]), Ji3 = to_dfl(geo[G_JINV + 3]);
  const dfl s = to_dfl(geo[G_S]);
  const dfl ds = to_dfl(geo[G_DET]) * s;
  // ---- volume terms
#pragma unroll 1
  for (int q = 0; q < D::NQ; ++q) {
    dacc U = dacc_zero(), A0 = dacc_zero(), A1 = dacc_zero();
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      mad(U, T.vphi[q][j], up[j]);
      mad(A0, T.vdphi[q][j][0], up[j]);
      mad(A1, T.vdphi[q][j][1], up[j]);
    }
    const dfl uc = s * val(U), a0 = val(A0), a1 = val(A1);
    // physical gradient d u_c / d x_d = s sum_r a_r Jinv[r][d]
    const dfl g0 = s * (a0 * Ji0 + a1 * Ji2), g1 = s * (a0 * Ji1 + a1 * Ji3);
    const dfl uo = shfl_pair(uc);
    const dfl u0 = c ? uo : uc, u1 = c ? uc : uo;
    const dfl F0 = uc * u0 - nu * g0, F1 = uc * u1 - nu * g1;
    const dfl w = T.vw[q] * ds;
    // H_r = w sum_d F_d Jinv[r][d]
    const dfl H0 = w * (F0 * Ji0 + F1 * Ji1), H1 = w * (F0 * Ji2 + F1 * Ji3);
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      mad(acc[j], H0, T.vdphi[q][j][0]);
      mad(acc[j], H1, T.vdphi[q][j][1]);
    }
  }
  // ---- facet terms
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    // A boundary facet (no neighbour) adds no term here. It is evaluated against its own trace
    // with weight zero, so that both threads of every pair still reach each shuffle; inflow and
    // outflow facets add their convective flux in boundary_component.
    const int tnr = __ldg(&m.tri_nbr[size_t(t) * 3 + e]);
    const bool wall = tnr < 0;
    const int tn = wall ? t : tnr;
    const int en = wall ? e : __ldg(&m.tri_nbr_loc[size_t(t) * 3 + e]);
    const int ncls = __ldg(&m.tri_class[tn]);
    const float2* geon = m.geo_df + size_t(ncls) * kGeo;
    const dfl sn = to_dfl(geon[G_S]);
    const dfl n0 = to_dfl(geo[G_NRM + 2 * e]), n1 = to_dfl(geo[G_NRM + 2 * e + 1]);
    const dfl nc = c ? n1 : n0;
    const dfl lens = wall ? dfl(0) : to_dfl(geo[G_FLEN + e]) * s;
    const dfl sig = to_dfl(m.sigma_df[__ldg(&m.tri_facet[size_t(t) * 3 + e])]);
    const dfl nusig = nu * sig, hnu = half(nu);
    dfl un[NS];
    load_df<NS>(ug + size_t(tn) * ND + c * NS, un);
    // normal derivative in reference gradients: d_n psi = s sum_r d_r psihat (Jinv n)_r
    const dfl mo0 = Ji0 * n0 + Ji1 * n1, mo1 = Ji2 * n0 + Ji3 * n1;
    const dfl mn0 = to_dfl(geon[G_JINV + 0]) * n0 + to_dfl(geon[G_JINV + 1]) * n1;
    const dfl mn1 = to_dfl(geon[G_JINV + 2]) * n0 + to_dfl(geon[G_JINV + 3]) * n1;
#pragma unroll 1
    for (int q = 0; q < D::NQF; ++q) {
      const int qn = D::NQF - 1 - q;
      dacc V = dacc_zero(), D0 = dacc_zero(), D1 = dacc_zero();
      dacc Vn = dacc_zero(), Dn0 = dacc_zero(), Dn1 = dacc_zero();
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        mad(V, T.fphi[e][q][j], up[j]);
        mad(D0, T.fdphi[e][q][j][0], up[j]);
        mad(D1, T.fdphi[e][q][j][1], up[j]);
        mad(Vn, T.fphi[en][qn][j], un[j]);
        mad(Dn0, T.fdphi[en][qn][j][0], un[j]);
        mad(Dn1, T.fdphi[en][qn][j][1], un[j]);
      }
      const dfl ui = s * val(V), di = s * (mo0 * val(D0) + mo1 * val(D1));
      const dfl uo = sn * val(Vn), dn = sn * (mn0 * val(Dn0) + mn1 * val(Dn1));
      // u.n = 1/2 (u_in + u_out) . n, summed in the same order by both threads of the pair
      const dfl pc = (ui + uo) * nc, po = shfl_pair(pc);
      const dfl vn = half(c ? po + pc : pc + po);
      const dfl wup = vn >= dfl(0) ? ui : uo;
      const dfl jc = ui - uo;
      const dfl w = T.fw[q] * lens;
      const dfl A = w * (hnu * (di + dn) - vn * wup - nusig * jc);
      const dfl B = w * hnu * jc;
      const dfl B0 = B * mo0, B1 = B * mo1;
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        mad(acc[j], A, T.fphi[e][q][j]);
        mad(acc[j], B0, T.fdphi[e][q][j][0]);
        mad(acc[j], B1, T.fdphi[e][q][j][1]);
      }
    }
  }
  if (m.facet_kind)
    boundary_terms<D::NQF>(
        m, geo, t, c, s,
        [&](int e, int q) {
          dacc V = dacc_zero();
#pragma unroll
          for (int j = 0; j < NS; ++j) mad(V, T.fphi[e][q][j], up[j]);
          return s * val(V);
        },
        [&](int e, int q, dfl F) {
          const dfl A = -(T.fw[q] * F);
#pragma unroll
          for (int j = 0; j < NS; ++j) mad(acc[j], A, T.fphi[e][q][j]);
        });
}

// Stage kernel, mixed form (all modes, see StageMode): reads the double-float
// twins a.up_df / a.un_df; writes h_df = P f and gl_df = G f (MODE_STAGE,
// MODE_PROJECT), h = f in FP64 (MODE_RESIDUAL, MODE_PRESSURE) and gl_df
// (MODE_PRESSURE). Thread c of a pair owns rows c*NS.. of f and h, and the rows
// i = c (mod 2) of gl.
template <int K>
__global__ void __launch_bounds__(kStageDfThreads, 2) k_stage_df(DevMesh m, StageArgs a) {
  using D = Dims<K>;
  constexpr int NS = D::NS, ND = D::ND, L3 = 3 * D::NL;
  __shared__ SmemTables<K, dfl> T;
  load_tables_df<K>(m, T);
  __syncthreads();
  const int c = threadIdx.x & 1;
  const int traw = blockIdx.x * (kStageDfThreads / 2) + (threadIdx.x >> 1);
  const bool live = traw < m.n_tri;
  const int t = live ? traw : m.n_tri - 1;   // both threads of a pair stay for the shuffles
  dfl up[NS];
  load_df<NS>(a.up_df + size_t(t) * ND + c * NS, up);
  dfl f[NS];
  if (a.mode == MODE_PROJECT) {
#pragma unroll
    for (int j = 0; j < NS; ++j) f[j] = up[j];
  } else {
    dacc acc[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) acc[j] = dacc_zero();
    residual_component<K>(m, T, t, c, a.up_df, up, acc);
    if (a.mode == MODE_STAGE) {
      dfl un[NS];
      load_df<NS>(a.un_df + size_t(t) * ND + c * NS, un);
      const dfl ca(a.a), cb(a.b), cc(a.c);
#pragma unroll
      for (int j = 0; j < NS; ++j) f[j] = ca * un[j] + cb * up[j] + cc * val(acc[j]);
    } else {
#pragma unroll
      for (int j = 0; j < NS; ++j) f[j] = val(acc[j]);
    }
  }
  if (a.mode == MODE_RESIDUAL || a.mode == MODE_PRESSURE) {
    if (live)
#pragma unroll
      for (int j = 0; j < NS; ++j) m.h[size_t(t) * ND + c * NS + j] = to_double(f[j]);
  }
  if (a.mode == MODE_RESIDUAL) return;   // uniform over the block
  dfl fo[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) fo[j] = shfl_pair(f[j]);
  const int cls = __ldg(&m.tri_class[t]);
  // F[i] = f_i in triangle order: component 0 first
  auto F = [&](int i) -> dfl { return (i < NS) == (c == 0) ? f[i % NS] : fo[i % NS]; };
  if (a.mode != MODE_PRESSURE) {
    const float2* P = m.Pdf + size_t(cls) * ND * ND;
    for (int r = 0; r < NS; ++r) {
      const int i = c * NS + r;
      dacc v = dacc_zero();
#pragma unroll
      for (int j = 0; j < ND; ++j) mad(v, to_dfl(__ldg(&P[i * ND + j])), F(j));
      if (live) m.h_df[size_t(t) * ND + i] = to_float2(val(v));
    }
  }
  const float2* G = m.Gdf + size_t(cls) * L3 * ND;
  for (int i = c; i < L3; i += 2) {
    dacc v = dacc_zero();
#pragma unroll
    for (int j = 0; j < ND; ++j) mad(v, to_dfl(__ldg(&G[i * ND + j])), F(j));
    if (live) m.gl_df[size_t(t) * L3 + i] = to_float2(val(v));
  }
}

// ---- paired form (meshes with at most kDnClasses geometry classes). The normal
// derivatives of the basis at the facet points come from a per-class table, so a trace
// takes two sums (value, normal derivative) instead of three and the test derivative one
// instead of two. Every sum over basis functions takes two consecutive indices j, j+1 at
// once in the packed FP32x2 instructions (dacc2 / mad2), with the tables laid out as
// pairs {hi_j, hi_j+1, lo_j, lo_j+1}. The terms and the per-point arithmetic are those of
// k_stage_df; only the order of summation inside each dot product differs (even and odd
// j apart).
template <int K>
struct PairTables {
  static constexpr int NS2 = (Dims<K>::NS + 1) / 2, NQ = Dims<K>::NQ, NQF = Dims<K>::NQF;
  float4 vphi[NQ][NS2];
  float4 vd0[NQ][NS2];   // d/dxi1 of the reference basis
  float4 vd1[NQ][NS2];   // d/dxi2
  float4 fphi[3][NQF][NS2];
  float4 dn[kDnClasses][3][NQF][NS2];   // d/dn of the basis at the facet points, per class
  float2 vw[NQ], fw[NQF];
};

__device__ __forceinline__ dfl2 pair(float4 v) { return dfl2{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }

// coefficients j = 0..N-1 of a double-float row as pairs (a missing j+1 is zero)
template <int N>
__device__ __forceinline__ void load_pairs(const float2* __restrict__ p, dfl2 (&c)[(N + 1) / 2]) {
#pragma unroll
  for (int jp = 0; jp < (N + 1) / 2; ++jp) {
    const float2 x = p[2 * jp];
    const float2 y = 2 * jp + 1 < N ? p[2 * jp + 1] : make_float2(0.f, 0.f);
    c[jp] = dfl2{make_float2(x.x, y.x), make_float2(x.y, y.y)};
  }
}

__device__ __forceinline__ dfl lane(const dfl2& v, int l) { return l ? dfl(v.hi.y, v.lo.y) : dfl(v.hi.x, v.lo.x); }

template <int K>
__device__ __forceinline__ void residual_pairs(const DevMesh& m, const PairTables<K>& T, int t, int c,
                                               const float2* __restrict__ ug, const dfl2 (&up)[PairTables<K>::NS2],
                                               dacc2 (&acc)[PairTables<K>::NS2]) {
  using D = Dims<K>;
  constexpr int NS = D::NS, ND = D::ND, NS2 = PairTables<K>::NS2;
  const dfl nu(m.nu);
  const int cls = __ldg(&m.tri_class[t]);
  const float2* geo = m.geo_df + size_t(cls) * kGeo;
  const dfl Ji0 = to_dfl(geo[G_JINV + 0]), Ji1 = to_dfl(geo[G_JINV + 1]);
  const dfl Ji2 = to_dfl(geo[G_JINV + 2]), Ji3 = to_dfl(geo[G_JINV + 3]);
  const dfl s = to_dfl(geo[G_S]);
  const dfl ds = to_dfl(geo[G_DET]) * s;
  // ---- volume terms
#pragma unroll 1
  for (int q = 0; q < D::NQ; ++q) {
    dacc2 U = dacc2_zero(), A0 = dacc2_zero(), A1 = dacc2_zero();
#pragma unroll
    for (int jp = 0; jp < NS2; ++jp) {
      mad2(U, pair(T.vphi[q][jp]), up[jp]);
      mad2(A0, pair(T.vd0[q][jp]), up[jp]);
      mad2(A1, pair(T.vd1[q][jp]), up[jp]);
    }
    const dfl uc = s * val_sum(U), a0 = val_sum(A0), a1 = val_sum(A1);
    const dfl g0 = s * (a0 * Ji0 + a1 * Ji2), g1 = s * (a0 * Ji1 + a1 * Ji3);
    const dfl uo = shfl_pair(uc);
    const dfl u0 = c ? uo : uc, u1 = c ? uc : uo;
    const dfl F0 = uc * u0 - nu * g0, F1 = uc * u1 - nu * g1;
    const dfl w = to_dfl(T.vw[q]) * ds;
    const dfl2 H0 = splat(w * (F0 * Ji0 + F1 * Ji1)), H1 = splat(w * (F0 * Ji2 + F1 * Ji3));
#pragma unroll
    for (int jp = 0; jp < NS2; ++jp) {
      mad2(acc[jp], H0, pair(T.vd0[q][jp]));
      mad2(acc[jp], H1, pair(T.vd1[q][jp]));
    }
  }
  // ---- facet terms
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    // a boundary facet: own trace, weight zero (see residual_component)
    const int tnr = __ldg(&m.tri_nbr[size_t(t) * 3 + e]);
    const bool wall = tnr < 0;
    const int tn = wall ? t : tnr;
    const int en = wall ? e : __ldg(&m.tri_nbr_loc[size_t(t) * 3 + e]);
    const int ncls = __ldg(&m.tri_class[tn]);
    const dfl sn = to_dfl(m.geo_df[size_t(ncls) * kGeo + G_S]);
    const dfl n0 = to_dfl(geo[G_NRM + 2 * e]), n1 = to_dfl(geo[G_NRM + 2 * e + 1]);
    const dfl nc = c ? n1 : n0;
    const dfl lens = wall ? dfl(0) : to_dfl(geo[G_FLEN + e]) * s;
    const dfl sig = to_dfl(m.sigma_df[__ldg(&m.tri_facet[size_t(t) * 3 + e])]);
    const dfl nusig = nu * sig, hnu = half(nu);
    const dfl msn = -sn;   // the neighbour's table holds derivatives along its own normal, -n
    dfl2 un[NS2];
    load_pairs<NS>(ug + size_t(tn) * ND + c * NS, un);
#pragma unroll 1
    for (int q = 0; q < D::NQF; ++q) {
      const int qn = D::NQF - 1 - q;
      dacc2 V = dacc2_zero(), Dd = dacc2_zero(), Vn = dacc2_zero(), Dnd = dacc2_zero();
#pragma unroll
      for (int jp = 0; jp < NS2; ++jp) {
        mad2(V, pair(T.fphi[e][q][jp]), up[jp]);
        mad2(Dd, pair(T.dn[cls][e][q][jp]), up[jp]);
        mad2(Vn, pair(T.fphi[en][qn][jp]), un[jp]);
        mad2(Dnd, pair(T.dn[ncls][en][qn][jp]), un[jp]);
      }
      const dfl ui = s * val_sum(V), di = s * val_sum(Dd);
      const dfl uo = sn * val_sum(Vn), dn = msn * val_sum(Dnd);
      const dfl pc = (ui + uo) * nc, po = shfl_pair(pc);
      const dfl vn = half(c ? po + pc : pc + po);
      const dfl wup = vn >= dfl(0) ? ui : uo;
      const dfl jc = ui - uo;
      const dfl w = to_dfl(T.fw[q]) * lens;
      const dfl2 A = splat(w * (hnu * (di + dn) - vn * wup - nusig * jc));
      const dfl2 B = splat(w * hnu * jc);
#pragma unroll
      for (int jp = 0; jp < NS2; ++jp) {
        mad2(acc[jp], A, pair(T.fphi[e][q][jp]));
        mad2(acc[jp], B, pair(T.dn[cls][e][q][jp]));
      }
    }
  }
  if (m.facet_kind)
    boundary_terms<D::NQF>(
        m, geo, t, c, s,
        [&](int e, int q) {
          dacc2 V = dacc2_zero();
#pragma unroll
          for (int jp = 0; jp < NS2; ++jp) mad2(V, pair(T.fphi[e][q][jp]), up[jp]);
          return s * val_sum(V);
        },
        [&](int e, int q, dfl F) {
          const dfl2 A = splat(-(to_dfl(T.fw[q]) * F));
#pragma unroll
          for (int jp = 0; jp < NS2; ++jp) mad2(acc[jp], A, pair(T.fphi[e][q][jp]));
        });
}

// Stage kernel, paired form: the modes, inputs and outputs of k_stage_df; the class
// operators P and G are read as column pairs (m.P2, m.G2).
template <int K>
__global__ void __launch_bounds__(kStageDfThreads, 2) k_stage_df2(DevMesh m, StageArgs a) {
  using D = Dims<K>;
  using PT = PairTables<K>;
  constexpr int NS = D::NS, ND = D::ND, L3 = 3 * D::NL, NS2 = PT::NS2, NDP = ND / 2;
  __shared__ PT T;
  {
    float4* dst = reinterpret_cast<float4*>(&T);
    for (int i = threadIdx.x; i < int(sizeof(PT) / sizeof(float4)); i += blockDim.x) dst[i] = __ldg(&m.ptab[i]);
  }
  __syncthreads();
  const int c = threadIdx.x & 1;
  const int traw = blockIdx.x * (kStageDfThreads / 2) + (threadIdx.x >> 1);
  const bool live = traw < m.n_tri;
  const int t = live ? traw : m.n_tri - 1;   // both threads of a pair stay for the shuffles
  dfl2 up[NS2];
  load_pairs<NS>(a.up_df + size_t(t) * ND + c * NS, up);
  dfl f[NS];
  if (a.mode == MODE_PROJECT) {
#pragma unroll
    for (int j = 0; j < NS; ++j) f[j] = lane(up[j / 2], j & 1);
  } else {
    dacc2 acc[NS2];
#pragma unroll
    for (int jp = 0; jp < NS2; ++jp) acc[jp] = dacc2_zero();
    residual_pairs<K>(m, T, t, c, a.up_df, up, acc);
    if (a.mode == MODE_STAGE) {
      dfl un[NS];
      load_df<NS>(a.un_df + size_t(t) * ND + c * NS, un);
      const dfl ca(a.a), cb(a.b), cc(a.c);
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const dfl r = (j & 1) ? val_y(acc[j / 2]) : val_x(acc[j / 2]);
        f[j] = ca * un[j] + cb * lane(up[j / 2], j & 1) + cc * r;
      }
    } else {
#pragma unroll
      for (int j = 0; j < NS; ++j) f[j] = (j & 1) ? val_y(acc[j / 2]) : val_x(acc[j / 2]);
    }
  }
  if (a.mode == MODE_RESIDUAL || a.mode == MODE_PRESSURE) {
    if (live)
#pragma unroll
      for (int j = 0; j < NS; ++j) m.h[size_t(t) * ND + c * NS + j] = to_double(f[j]);
  }
  if (a.mode == MODE_RESIDUAL) return;   // uniform over the block
  // F = f in triangle order (component 0 first), as column pairs
  dfl2 F[NDP];
  {
    dfl fo[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) fo[j] = shfl_pair(f[j]);
#pragma unroll
    for (int jp = 0; jp < NDP; ++jp) {
      const int i0 = 2 * jp, i1 = 2 * jp + 1;
      const dfl x = (i0 < NS) == (c == 0) ? f[i0 % NS] : fo[i0 % NS];
      const dfl y = (i1 < NS) == (c == 0) ? f[i1 % NS] : fo[i1 % NS];
      F[jp] = dfl2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
    }
  }
  const int cls = __ldg(&m.tri_class[t]);
  if (a.mode != MODE_PRESSURE && m.tc_rec) {
    // the tensor-core recovery applies P itself: keep f
    if (live)
#pragma unroll
      for (int j = 0; j < NS; ++j) m.h_df[size_t(t) * ND + c * NS + j] = to_float2(f[j]);
  } else if (a.mode != MODE_PRESSURE) {
    const float4* P = m.P2 + size_t(cls) * ND * NDP;
    for (int r = 0; r < NS; ++r) {
      const int i = c * NS + r;
      dacc2 v = dacc2_zero();
#pragma unroll
      for (int jp = 0; jp < NDP; ++jp) mad2(v, pair(__ldg(&P[i * NDP + jp])), F[jp]);
      if (live) m.h_df[size_t(t) * ND + i] = to_float2(val_sum(v));
    }
  }
  const float4* G = m.G2 + size_t(cls) * L3 * NDP;
  for (int i = c; i < L3; i += 2) {
    dacc2 v = dacc2_zero();
#pragma unroll
    for (int jp = 0; jp < NDP; ++jp) mad2(v, pair(__ldg(&G[i * NDP + jp])), F[jp]);
    if (live) m.gl_df[size_t(t) * L3 + i] = to_float2(val_sum(v));
  }
}

// Recovery, mixed form: u_T = h_T - G_T^T lam_T (h = P f from the stage kernel) in
// double-float, with lam from the double-float solver (lam_is_df) or the FP64 one.
// Writes the double-float twin out_df and, if out is given, u in FP64. A block's rows of
// h and u pass through shared memory (padded rows), so that global reads and writes are
// coalesced; a thread issues all its tile loads before its shared-memory stores. For k = 3,
// two threads per triangle, one per velocity component (warp-uniform): twice the threads
// with half the compensated sums each hide more of the gathers' latency (33.1 -> 30.8 us per
// launch at 256^2); for k <= 2 the second thread's repeated gathers cost more than that.
constexpr int kRecoverTris = 128;
template <int K>
struct RecoverShape {
  static constexpr int TPT = K == 3 ? 2 : 1;           // threads per triangle
  static constexpr int THREADS = TPT * kRecoverTris;
};

template <int K>
__global__ void __launch_bounds__(RecoverShape<K>::THREADS) k_recover_df(DevMesh m, double* out, float2* out_df) {
  using D = Dims<K>;
  constexpr int ND = D::ND, NL = D::NL, L3 = 3 * NL, RS = ND + 1;
  constexpr int TPT = RecoverShape<K>::TPT, kRecoverThreads = RecoverShape<K>::THREADS;
  constexpr int PER = kRecoverTris * ND / kRecoverThreads;   // tile values per thread
  __shared__ float2 tile[kRecoverTris * RS];
  const int t0 = blockIdx.x * kRecoverTris;
  const int nt = min(kRecoverTris, m.n_tri - t0);
  const float2* hb = m.h_df + size_t(t0) * ND;
  if (nt == kRecoverTris) {
    float2 v[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) v[q] = __ldg(&hb[q * kRecoverThreads + threadIdx.x]);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = q * kRecoverThreads + threadIdx.x;
      tile[(e / ND) * RS + e % ND] = v[q];
    }
  } else {
    for (int e = threadIdx.x; e < nt * ND; e += kRecoverThreads) tile[(e / ND) * RS + e % ND] = hb[e];
  }
  __syncthreads();
  const int r = threadIdx.x % kRecoverTris, c = threadIdx.x / kRecoverTris;
  constexpr int NOUT = ND / TPT;   // outputs per thread: one component (TPT = 2) or both
  if (r < nt) {
    const int t = t0 + r;
    dfl lam[L3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int f = __ldg(&m.tri_facet[size_t(t) * 3 + e]);
      const bool flip = __ldg(&m.tri_orient[size_t(t) * 3 + e]) < 0;
#pragma unroll
      for (int mm = 0; mm < NL; ++mm) {
        const dfl v = m.lam_is_df ? to_dfl(m.lam_df[size_t(f) * m.lat_vs + mm]) : dfl(m.lam[size_t(f) * NL + mm]);
        lam[e * NL + mm] = (flip && (mm & 1)) ? v : -v;   // negated: u = h + sum (-G) lam
      }
    }
    const float2* G = m.Gdf + size_t(__ldg(&m.tri_class[t])) * L3 * ND;
    float2* row = tile + r * RS;
#pragma unroll 5
    for (int j = 0; j < NOUT; ++j) {
      const int i = c * NOUT + j;
      dacc v = dacc_of(to_dfl(row[i]));
#pragma unroll
      for (int l = 0; l < L3; ++l) mad(v, to_dfl(__ldg(&G[l * ND + i])), lam[l]);
      row[i] = to_float2(val(v));
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nt * ND; e += kRecoverThreads) {
    const float2 u = tile[(e / ND) * RS + e % ND];
    if (out_df) out_df[size_t(t0) * ND + e] = u;
    if (out) out[size_t(t0) * ND + e] = to_double(u);
  }
}

__global__ void k_to_dfl(const double* __restrict__ x, float2* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = to_float2(dfl(x[i]));
}

// y[f][j] = x[f][j] for j < ny: facet-major rows of stride sx (double-float) and ny (FP64)
__global__ void k_to_double(const float2* __restrict__ x, int sx, double* __restrict__ y, int ny, long long nrow) {
  const long long n = nrow * ny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = to_double(x[(i / ny) * sx + i % ny]);
}

// z = alpha x + beta y in double-float (the RK4 combination of stage states)
__global__ void k_axpby_df(const float2* x, const float2* __restrict__ y, float2* z, double alpha, double beta,
                           long long n) {
  const dfl al(alpha), be(beta);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = to_float2(al * to_dfl(x[i]) + be * to_dfl(y[i]));
}

__global__ void k_axpby64(const double* x, const double* __restrict__ y, double* z, double alpha, double beta,
                          long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    z[i] = alpha * x[i] + beta * y[i];
}

inline int blocks_for(long long n, int bs) { return int((n + bs - 1) / bs); }

}  // namespace

template <int K>
cudaError_t launch_pairs(const DevMesh& m, const StageArgs& a, cudaStream_t s) {
  // the host image must have the layout of PairTables<K>
  if (m.ptab_words != int(sizeof(PairTables<K>) / sizeof(float4))) return cudaErrorInvalidValue;
  k_stage_df2<K><<<blocks_for(m.n_tri, kStageDfThreads / 2), kStageDfThreads, 0, s>>>(m, a);
  return cudaSuccess;
}

#define DGDF_DISPATCH_K(kv, CALL) \
  switch (kv) {                   \
    case 1: { constexpr int K = 1; CALL; break; } \
    case 2: { constexpr int K = 2; CALL; break; } \
    case 3: { constexpr int K = 3; CALL; break; } \
    default: return cudaErrorInvalidValue;        \
  }

cudaError_t launch_stage_df(const DevMesh& m, const StageArgs& a, cudaStream_t s) {
  if (!a.up_df || (a.mode == MODE_STAGE && !a.un_df)) return cudaErrorInvalidValue;
  const int nb = blocks_for(m.n_tri, kStageDfThreads / 2);
  if (m.ptab) {
    cudaError_t e = cudaSuccess;
    DGDF_DISPATCH_K(m.k, (e = launch_pairs<K>(m, a, s)));
    if (e != cudaSuccess) return e;
  } else {
    DGDF_DISPATCH_K(m.k, (k_stage_df<K><<<nb, kStageDfThreads, 0, s>>>(m, a)));
  }
  return cudaGetLastError();
}

cudaError_t launch_recover_df(const DevMesh& m, double* out, float2* out_df, cudaStream_t s) {
  if (m.tc_rec) return launch_recover_tc(m, out, out_df, s);
  DGDF_DISPATCH_K(m.k, (k_recover_df<K><<<blocks_for(m.n_tri, kRecoverTris), RecoverShape<K>::THREADS, 0, s>>>(m, out, out_df)));
  return cudaGetLastError();
}

cudaError_t launch_axpby_df(const float2* x, const float2* y, float2* z, double alpha, double beta, long long n,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_axpby_df<<<int(std::min<long long>((n + 255) / 256, 152 * 16)), 256, 0, s>>>(x, y, z, alpha, beta, n);
  return cudaGetLastError();
}

cudaError_t launch_axpby64(const double* x, const double* y, double* z, double alpha, double beta, long long n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_axpby64<<<int(std::min<long long>((n + 255) / 256, 152 * 16)), 256, 0, s>>>(x, y, z, alpha, beta, n);
  return cudaGetLastError();
}

cudaError_t launch_to_dfl(const double* x, float2* y, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long nb = (n + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_to_dfl<<<int(nb), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_to_double(const float2* x, int sx, double* y, int ny, long long nrow, cudaStream_t s) {
  if (nrow <= 0) return cudaSuccess;
  long long nb = (nrow * ny + 255) / 256;
  if (nb > 4096) nb = 4096;
  k_to_double<<<int(nb), 256, 0, s>>>(x, sx, y, ny, nrow);
  return cudaGetLastError();
}

}  // namespace dgdf
