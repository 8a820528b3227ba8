// C-ABI of the three-dimensional path (include/dgdf3.h): closed tetrahedral meshes, FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/dgdf.h"
#include "../../include/dgdf3.h"
#include "device3.cuh"
#include "multilevel.hpp"
#include "setup3.hpp"

namespace dgdf {
int api_fail(int code, const std::string& msg);
void api_clear_error();
}  // namespace dgdf

struct dg_mesh3 {
  dgdf::HostMesh3 hm;
  dgdf::DevMesh3 dm{};
  dg_params p{};
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  int solver_blocks = 1;
  bool use_ml = false;            // multilevel PCG (k_solve3_ml), else block Jacobi (k_solve3)
  int ml_blocks = 1;
  dgdf::DevMesh mv{};             // the hierarchy and the PCG vectors for the multilevel kernel
  bool has_lam = false;
  double last_c = 0.0;
  // multipliers of each SSP-RK3 stage in the last kHist steps (warm starts; the layout of lam),
  // their step sizes, and how many are valid
  static constexpr int kHist = 3;
  double* hist[3][kHist] = {};
  double hist_dt[3][kHist] = {};
  int hist_n[3] = {};
  double* lattice = nullptr;          // [n_tet][ns][3] staging
  dgdf::DevStats* host_stats = nullptr;
  double *pe = nullptr, *pf = nullptr, *ppart = nullptr;   // pressure outputs and scratch (first use)
  double volume = 0.0;                // of the domain
};

namespace {

using dgdf::api_fail;

#define CK3(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return api_fail(e_ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,                     \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename T>
int dalloc3(dg_mesh3* M, T** out, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) return api_fail(DG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  M->allocs.push_back(p);
  *out = static_cast<T*>(p);
  return DG_OK;
}

template <typename T>
int upload3(dg_mesh3* M, const T** out, const std::vector<T>& v) {
  T* p = nullptr;
  int rc = dalloc3(M, &p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK3(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = p;
  return DG_OK;
}

int check3(const dg_mesh3* M) { return M ? DG_OK : api_fail(DG_ERR_INVALID_ARG, "NULL mesh"); }

int finish3(dg_mesh3* M, bool check_solver) {
  CK3(cudaStreamSynchronize(M->stream));
  if (!check_solver) return DG_OK;
  CK3(cudaMemcpy(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost));
  const int fl = M->host_stats->flags;
  if (fl & dgdf::kFlagBarrierTimeout) return api_fail(DG_ERR_CUDA, "solver grid barrier timed out");
  if (fl & dgdf::kFlagNonFinite) return api_fail(DG_ERR_NONFINITE, "non-finite residual in the face solve");
  if (fl & dgdf::kFlagNotConverged) return api_fail(DG_ERR_NOT_CONVERGED, "face solve reached cg_maxit");
  return DG_OK;
}

int reset3(dg_mesh3* M) {
  CK3(cudaMemsetAsync(&M->dm.stats->flags, 0, sizeof(int), M->stream));
  return DG_OK;
}

// stage >= 0: a solve of SSP-RK3 stage `stage` with step size dt. The multipliers of the
// stage are c dt times a smooth function of time: with three earlier entries taken with this
// step size, the warm start is the quadratic extrapolation 3 lam(n-1) - 3 lam(n-2) + lam(n-3),
// with two the linear one, else lam(n-1) rescaled by dt / dt(n-1); with none, warm_scale lam.
int solve3(dg_mesh3* M, double warm_scale, int stage = -1, double dt = 0.0) {
  dgdf::SolveArgs a{};
  a.warm_scale = warm_scale;
  if (stage >= 0 && M->hist_n[stage] >= 1) {
    const double* hd = M->hist_dt[stage];
    const int n = M->hist_n[stage];
    a.hist1 = M->hist[stage][0];
    a.hist2 = M->hist[stage][1];
    a.hist3 = M->hist[stage][2];
    a.c1 = dt / hd[0];
    if (n >= 3 && hd[0] == dt && hd[1] == dt && hd[2] == dt) {
      a.c1 = 3.0;
      a.c2 = -3.0;
      a.c3 = 1.0;
    } else if (n >= 2 && hd[0] == dt && hd[1] == dt) {
      a.c1 = 2.0;
      a.c2 = -1.0;
    }
  }
  a.rtol = M->p.cg_rtol;
  a.maxit = M->p.cg_maxit;
  a.floor_rtol = 1e-9;
  if (M->use_ml) CK3(dgdf::launch_solve3_ml(M->dm, M->mv, a, M->ml_blocks, M->stream));
  else CK3(dgdf::launch_solve3(M->dm, a, M->solver_blocks, M->stream));
  return DG_OK;
}

// After the solve of stage s with step size dt: the new multipliers become the newest history
// entry (the solver already moved the older ones down one slot).
int push_history3(dg_mesh3* M, int s, double dt) {
  const size_t bytes = size_t(M->dm.n_face) * M->hm.nl * sizeof(double);
  CK3(cudaMemcpyAsync(M->hist[s][0], M->dm.lam, bytes, cudaMemcpyDeviceToDevice, M->stream));
  for (int h = dg_mesh3::kHist - 1; h > 0; --h) M->hist_dt[s][h] = M->hist_dt[s][h - 1];
  M->hist_dt[s][0] = dt;
  M->hist_n[s] = std::min(M->hist_n[s] + 1, dg_mesh3::kHist);
  return DG_OK;
}

}  // namespace

extern "C" {

int dg3_mesh_create(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords, const dg_params* params,
                    dg_mesh3** out) {
  dgdf::api_clear_error();
  if (!out || !params || !tet_vertex_ids || !tet_coords) return api_fail(DG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  dg_params p = *params;
  if (p.k < 1 || p.k > dgdf::kMaxDegree3) return api_fail(DG_ERR_UNSUPPORTED, "3-D path: k must be 1..2");
  if (!(p.nu >= 0.0) || !std::isfinite(p.nu)) return api_fail(DG_ERR_INVALID_ARG, "nu must be finite and >= 0");
  if (!(p.alpha > 0.0) || !std::isfinite(p.alpha)) return api_fail(DG_ERR_INVALID_ARG, "alpha must be > 0");
  if (p.precision != DG_PRECISION_FP64) return api_fail(DG_ERR_UNSUPPORTED, "3-D path: FP64 form only");
  if (!(p.cg_rtol > 0.0)) p.cg_rtol = 1e-13;
  if (p.cg_maxit <= 0) p.cg_maxit = 20000;
  dg_mesh3* M = new dg_mesh3();
  M->p = p;
  M->stream = static_cast<cudaStream_t>(p.cuda_stream);
  std::string err;
  int rc = dgdf::build_host_mesh3(n_tet, tet_vertex_ids, tet_coords, p.k, p.alpha, M->hm, err);
  if (rc) {
    delete M;
    return api_fail(rc, err);
  }
  auto cleanup = [&](int code) {
    dg3_mesh_destroy(M);
    return code;
  };
  if (!dgdf::tet_tables_match(M->hm.k, M->hm.ref.nq, M->hm.ref.nqf))
    return cleanup(api_fail(DG_ERR_MESH, "3-D set-up: quadrature sizes differ from the kernels'"));
  const dgdf::HostMesh3& hm = M->hm;
  const dgdf::Ref3& ref = hm.ref;
  dgdf::DevMesh3& d = M->dm;
  d.k = hm.k;
  d.ns = hm.ns;
  d.nd = hm.nd;
  d.nw = hm.nw;
  d.nl = hm.nl;
  d.nq = ref.nq;
  d.nqf = ref.nqf;
  d.n_tet = int(hm.n_tet);
  d.n_face = int(hm.n_face);
  d.n_class = int(hm.classes.size());
  d.n_stencil = hm.n_stencil;
  d.nu = p.nu;
  const int nd = hm.nd, L4 = 4 * hm.nl;
  std::vector<double> geo(size_t(d.n_class) * dgdf::kGeo3, 0.0), P, G, W, WC;
  for (int c = 0; c < d.n_class; ++c) {
    const dgdf::Class3& co = hm.classes[c];
    double* g = &geo[size_t(c) * dgdf::kGeo3];
    for (int i = 0; i < 9; ++i) g[dgdf::G3_JINV + i] = co.Jinv[i];
    g[dgdf::G3_DET] = co.det;
    g[dgdf::G3_S] = 1.0 / std::sqrt(co.det);
    for (int e = 0; e < 4; ++e) {
      for (int x = 0; x < 3; ++x) g[dgdf::G3_NRM + 3 * e + x] = co.normal[e][x];
      g[dgdf::G3_AREA + e] = co.area[e];
      g[dgdf::G3_PERM + e] = co.perm[e];
    }
    P.insert(P.end(), co.P.begin(), co.P.end());
    G.insert(G.end(), co.G.begin(), co.G.end());
    W.insert(W.end(), co.W.begin(), co.W.end());
    WC.insert(WC.end(), co.WC.begin(), co.WC.end());
  }
  for (int64_t t = 0; t < hm.n_tet; ++t) M->volume += hm.classes[hm.tet_class[t]].det / 6.0;
  if ((rc = upload3(M, &d.vw, ref.vw)) || (rc = upload3(M, &d.vphi, ref.vphi)) ||
      (rc = upload3(M, &d.vdphi, ref.vdphi)) || (rc = upload3(M, &d.fw, ref.fw)) ||
      (rc = upload3(M, &d.fphi, ref.fphi)) || (rc = upload3(M, &d.fdphi, ref.fdphi)) ||
      (rc = upload3(M, &d.lat_phi, ref.lat_phi)) || (rc = upload3(M, &d.lat_inv, ref.lat_inv)) ||
      (rc = upload3(M, &d.geo, geo)) || (rc = upload3(M, &d.P, P)) || (rc = upload3(M, &d.G, G)) ||
      (rc = upload3(M, &d.W, W)) || (rc = upload3(M, &d.WC, WC)) || (rc = upload3(M, &d.plat_phi, ref.plat_phi)) ||
      (rc = upload3(M, &d.mu_lat, ref.mu_lat)) ||
      (rc = upload3(M, &d.tet_class, hm.tet_class)) || (rc = upload3(M, &d.tet_nbr, hm.tet_nbr)) ||
      (rc = upload3(M, &d.tet_face, hm.tet_face)) || (rc = upload3(M, &d.tet_nbr_loc, hm.tet_nbr_loc)) ||
      (rc = upload3(M, &d.face_sigma, hm.face_sigma)) || (rc = upload3(M, &d.face_tet, hm.face_tet)) ||
      (rc = upload3(M, &d.face_nbr, hm.face_nbr)) || (rc = upload3(M, &d.face_stencil, hm.face_stencil)) ||
      (rc = upload3(M, &d.face_loc, hm.face_loc)) || (rc = upload3(M, &d.st_blk, hm.stencil_blocks)) ||
      (rc = upload3(M, &d.st_binv, hm.stencil_binv)))
    return cleanup(rc);
  const size_t nT = size_t(d.n_tet), nF = size_t(d.n_face), nl = size_t(hm.nl);
  if ((rc = dalloc3(M, &d.u, nT * nd)) || (rc = dalloc3(M, &d.ustage, nT * nd)) || (rc = dalloc3(M, &d.h, nT * nd)) ||
      (rc = dalloc3(M, &d.gl, nT * L4)) || (rc = dalloc3(M, &d.lam, nF * nl)) || (rc = dalloc3(M, &d.g, nF * nl)) ||
      (rc = dalloc3(M, &d.r, nF * nl)) || (rc = dalloc3(M, &d.z, nF * nl)) || (rc = dalloc3(M, &d.pa, nF * nl)) ||
      (rc = dalloc3(M, &d.pb, nF * nl)) || (rc = dalloc3(M, &d.q, nF * nl)) ||
      (rc = dalloc3(M, &d.red, size_t(dgdf::kRedSlots) * dgdf::kMaxSolverBlocks)) || (rc = dalloc3(M, &d.bar, 1)) ||
      (rc = dalloc3(M, &d.stats, 1)) || (rc = dalloc3(M, &d.diag, 8)) ||
      (rc = dalloc3(M, &M->lattice, nT * hm.ns * 3)))
    return cleanup(rc);
  for (int s = 0; s < 3; ++s)
    for (int h = 0; h < dg_mesh3::kHist; ++h)
      if ((rc = dalloc3(M, &M->hist[s][h], nF * nl))) return cleanup(rc);
  cudaError_t e = cudaMallocHost(&M->host_stats, sizeof(dgdf::DevStats));
  if (e != cudaSuccess) return cleanup(api_fail(DG_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e)));
  e = cudaMemsetAsync(d.u, 0, nT * nd * sizeof(double), M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.lam, 0, nF * nl * sizeof(double), M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.stats, 0, sizeof(dgdf::DevStats), M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  if (e != cudaSuccess) return cleanup(api_fail(DG_ERR_CUDA, std::string("initialise: ") + cudaGetErrorString(e)));
  M->solver_blocks = dgdf::solver3_blocks(d);
  // multilevel preconditioner (default; DG_PRECOND_BLOCK_JACOBI keeps block Jacobi): block-Jacobi
  // Chebyshev smoothing on the face stencil, injection to the face-constant multipliers, smoothed
  // aggregation with point-Jacobi smoothing on their assembled operator (multilevel.hpp,
  // build_multilevel_csr)
  if (p.precond != DG_PRECOND_BLOCK_JACOBI) {
    dgdf::CsrHost A0 = dgdf::stencil_csr(d.n_face, hm.nl, 6, hm.face_stencil.data(), hm.face_nbr.data(),
                                         hm.stencil_blocks.data());
    dgdf::MLHost mlh;
    std::string merr;
    if ((rc = dgdf::build_multilevel_csr(A0, hm.nl, hm.face_stencil.data(), &hm.stencil_binv, mlh, merr)))
      return cleanup(api_fail(rc, merr));
    // the V-cycle runs in FP32 (a preconditioner needs no more; the PCG vectors and S stay FP64):
    // level operators, transfers, Chebyshev coefficients and the coarsest pseudo-inverse rounded
    // once; level 0 has vectors of its own, filled from r and written back to z
    auto f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    std::vector<dgdf::MLLevelT<float>> lv(mlh.lv.size());
    const float* blk32 = nullptr;
    if ((rc = upload3(M, &blk32, f32(hm.stencil_blocks)))) return cleanup(rc);
    for (size_t l = 0; l < mlh.lv.size(); ++l) {
      const dgdf::MLHostLevel& H = mlh.lv[l];
      dgdf::MLLevelT<float>& L = lv[l];
      L.stencil = H.stencil ? 1 : 0;
      L.bs = H.bs;
      L.n = H.n;
      L.inject = H.inject ? 1 : 0;
      L.n_next = H.n_next;
      L.bs_next = H.bs_next;
      L.modes = 1;
      L.c0 = float(H.cheb[0]);
      L.c1 = float(H.cheb[1]);
      L.c2 = float(H.cheb[2]);
      if ((rc = upload3(M, &L.binv, f32(H.binv)))) return cleanup(rc);
      if (H.stencil) {   // level 0: block Jacobi on the seven-block face stencil
        L.st_cls = d.face_stencil;
        L.st_nbr = d.face_nbr;
        L.st_nnb = 6;
        L.st_blk = blk32;
      } else if ((rc = upload3(M, &L.a_rp, H.A.rp)) || (rc = upload3(M, &L.a_ci, H.A.ci)) ||
                 (rc = upload3(M, &L.a_v, f32(H.A.v)))) {
        return cleanup(rc);
      }
      if (!H.inject && ((rc = upload3(M, &L.p_rp, H.P.rp)) || (rc = upload3(M, &L.p_ci, H.P.ci)) ||
                        (rc = upload3(M, &L.p_v, f32(H.P.v))) || (rc = upload3(M, &L.r_rp, H.R.rp)) ||
                        (rc = upload3(M, &L.r_ci, H.R.ci)) || (rc = upload3(M, &L.r_v, f32(H.R.v)))))
        return cleanup(rc);
      const size_t nv = size_t(H.n) * H.bs;
      if ((rc = dalloc3(M, &L.b, nv)) || (rc = dalloc3(M, &L.x, nv)) || (rc = dalloc3(M, &L.r, nv)) ||
          (rc = dalloc3(M, &L.d, nv)))
        return cleanup(rc);
    }
    dgdf::DevMesh& v = M->mv;
    const dgdf::MLLevelT<float>* lvd = nullptr;
    if ((rc = upload3(M, &lvd, lv)) || (rc = upload3(M, &v.ml_cpinv_f, f32(mlh.cpinv))) ||
        (rc = dalloc3(M, &v.ml_xc_f, size_t(mlh.nc))) || (rc = dalloc3(M, &v.ml_bc_f, size_t(mlh.nc))))
      return cleanup(rc);
    v.ml_lv_f = lvd;
    v.ml_nlev = int(lv.size());
    v.ml_nc = mlh.nc;
    v.k = d.k;
    v.n_facet = d.n_face;
    v.r = d.r;
    v.z = d.z;
    v.red = d.red;
    v.bar = d.bar;
    v.stats = d.stats;
    M->use_ml = true;
    M->ml_blocks = dgdf::solver3_ml_blocks(d, true);
  }
  *out = M;
  return DG_OK;
}

int dg3_mesh_destroy(dg_mesh3* M) {
  if (!M) return DG_OK;
  for (void* p : M->allocs) cudaFree(p);
  if (M->host_stats) cudaFreeHost(M->host_stats);
  delete M;
  return DG_OK;
}

int dg3_mesh_info(const dg_mesh3* M, int64_t out[8]) {
  if (int rc = check3(M)) return rc;
  if (!out) return api_fail(DG_ERR_INVALID_ARG, "NULL out");
  const dgdf::HostMesh3& hm = M->hm;
  out[0] = hm.n_tet;
  out[1] = hm.n_face;
  out[2] = hm.k;
  out[3] = dgdf::n_lat3(hm.k);
  out[4] = int64_t(hm.classes.size());
  out[5] = hm.n_stencil;
  out[6] = hm.n_tet * hm.nd;
  out[7] = hm.n_face * hm.nl;
  return DG_OK;
}

int dg3_set_velocity(dg_mesh3* M, const double* vals, int on_device) {
  if (int rc = check3(M)) return rc;
  if (!vals) return api_fail(DG_ERR_INVALID_ARG, "NULL vals");
  const size_t n = size_t(M->dm.n_tet) * M->hm.ns * 3;
  if (!on_device)
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(vals[i])) return api_fail(DG_ERR_NONFINITE, "non-finite velocity value");
  CK3(cudaMemcpyAsync(M->lattice, vals, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      M->stream));
  CK3(dgdf::launch_lattice_to_coef3(M->dm, M->lattice, M->dm.u, M->stream));
  M->has_lam = false;
  return finish3(M, false);
}

int dg3_get_velocity(dg_mesh3* M, double* vals, int on_device) {
  if (int rc = check3(M)) return rc;
  if (!vals) return api_fail(DG_ERR_INVALID_ARG, "NULL vals");
  const size_t n = size_t(M->dm.n_tet) * M->hm.ns * 3;
  CK3(dgdf::launch_coef_to_lattice3(M->dm, M->dm.u, M->lattice, M->stream));
  CK3(cudaMemcpyAsync(vals, M->lattice, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      M->stream));
  return finish3(M, false);
}

int dg3_project_divfree(dg_mesh3* M) {
  if (int rc = check3(M)) return rc;
  int rc = reset3(M);
  if (rc) return rc;
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_PROJECT;
  a.up = M->dm.u;
  a.un = M->dm.u;
  CK3(dgdf::launch_stage3(M->dm, a, M->stream));
  if ((rc = solve3(M, 0.0))) return rc;
  CK3(dgdf::launch_recover3(M->dm, M->dm.u, M->stream));
  M->has_lam = false;
  for (int s = 0; s < 3; ++s) M->hist_n[s] = 0;
  return finish3(M, true);
}

int dg3_rk3_step(dg_mesh3* M, double dt, int64_t nsteps) {
  if (int rc = check3(M)) return rc;
  if (!(dt > 0.0) || !std::isfinite(dt)) return api_fail(DG_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (nsteps < 0) return api_fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  int rc = reset3(M);
  if (rc) return rc;
  // SSP-RK3, eq. (8): u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1)); u = 1/3 u + 2/3 (u2 + dt L(u2))
  const double co[3][2] = {{0.0, 1.0}, {0.75, 0.25}, {1.0 / 3.0, 2.0 / 3.0}};
  dgdf::DevMesh3& d = M->dm;
  for (int64_t n = 0; n < nsteps; ++n)
    for (int s = 0; s < 3; ++s) {
      dgdf::StageArgs a{};
      a.mode = dgdf::MODE_STAGE;
      a.a = co[s][0];
      a.b = co[s][1];
      a.c = co[s][1] * dt;
      a.un = d.u;
      a.up = s == 0 ? d.u : d.ustage;
      CK3(dgdf::launch_stage3(d, a, M->stream));
      // warm start from the stage's history, else from the previous stage's multipliers
      // rescaled by the ratio of the L coefficients
      if ((rc = solve3(M, M->has_lam ? a.c / M->last_c : 0.0, s, dt)) || (rc = push_history3(M, s, dt))) return rc;
      CK3(dgdf::launch_recover3(d, s == 2 ? d.u : d.ustage, M->stream));
      M->last_c = a.c;
      M->has_lam = true;
    }
  return finish3(M, true);
}

int dg3_get_pressure(dg_mesh3* M, double* p_elem, double* p_face, int on_device) {
  if (int rc = check3(M)) return rc;
  if (!p_elem) return api_fail(DG_ERR_INVALID_ARG, "NULL p_elem");
  int rc = reset3(M);
  if (rc) return rc;
  dgdf::DevMesh3& d = M->dm;
  const size_t npe = size_t(d.n_tet) * d.nw, npf = size_t(d.n_face) * d.nl;
  if (!M->pe && ((rc = dalloc3(M, &M->pe, npe)) || (rc = dalloc3(M, &M->pf, npf)) ||
                 (rc = dalloc3(M, &M->ppart, size_t(dgdf::pressure3_parts(d))))))
    return rc;
  // the functional L(u) alone (eq. (12) with F = L(u), Theorem 2, Remark 2)
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_PRESSURE;
  a.up = d.u;
  a.un = d.u;
  CK3(dgdf::launch_stage3(d, a, M->stream));
  if ((rc = solve3(M, 0.0))) return rc;
  CK3(dgdf::launch_pressure3(d, M->pe, p_face ? M->pf : nullptr, M->ppart, M->volume, M->stream));
  M->has_lam = false;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK3(cudaMemcpyAsync(p_elem, M->pe, npe * sizeof(double), kind, M->stream));
  if (p_face) CK3(cudaMemcpyAsync(p_face, M->pf, npf * sizeof(double), kind, M->stream));
  return finish3(M, true);
}

int dg3_eval_residual(dg_mesh3* M, double* vals, int on_device) {
  if (int rc = check3(M)) return rc;
  if (!vals) return api_fail(DG_ERR_INVALID_ARG, "NULL vals");
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_RESIDUAL;
  a.up = M->dm.u;
  a.un = M->dm.u;
  CK3(dgdf::launch_stage3(M->dm, a, M->stream));
  const size_t n = size_t(M->dm.n_tet) * M->hm.ns * 3;
  CK3(dgdf::launch_coef_to_lattice3(M->dm, M->dm.h, M->lattice, M->stream));
  CK3(cudaMemcpyAsync(vals, M->lattice, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      M->stream));
  return finish3(M, false);
}

int dg3_get_diagnostics(dg_mesh3* M, double out[8]) {
  if (int rc = check3(M)) return rc;
  if (!out) return api_fail(DG_ERR_INVALID_ARG, "NULL out");
  CK3(dgdf::launch_diagnostics3(M->dm, M->dm.u, M->stream));
  double d4[4];
  CK3(cudaMemcpyAsync(d4, M->dm.diag, sizeof(d4), cudaMemcpyDeviceToHost, M->stream));
  CK3(cudaMemcpyAsync(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost, M->stream));
  if (int rc = finish3(M, false)) return rc;
  out[0] = d4[0];
  out[1] = d4[1];
  out[2] = d4[2];
  out[3] = d4[3];
  out[4] = M->host_stats->last_iters;
  out[5] = M->host_stats->last_relres;
  out[6] = double(M->host_stats->total_iters);
  out[7] = double(M->host_stats->solves);
  return DG_OK;
}

}  // extern "C"
