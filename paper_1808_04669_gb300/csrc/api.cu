// C ABI of libdgdf (declared in include/dgdf.h): mesh set-up, state I/O and
// the stage pipeline. Host code here only orchestrates; every step of the
// method runs in the kernels of k_element.cu and k_solver.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dgdf.h"
#include "device.cuh"
#include "kcommon.cuh"
#include "multilevel.hpp"
#include "setup.hpp"

static_assert(dgdf::Dims<1>::NQ == dgdf::kVolumePoints(1) && dgdf::Dims<2>::NQ == dgdf::kVolumePoints(2) &&
                  dgdf::Dims<3>::NQ == dgdf::kVolumePoints(3),
              "host and device volume rules differ in size");

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

enum KernelClass {
  KC_STAGE = 0,
  KC_SOLVE64,
  KC_SOLVE_MIXED,
  KC_RECOVER,
  KC_PROJECT_RHS,
  KC_LATTICE,
  KC_DIAG,
  KC_PRESSURE,
  KC_SOLVE_LAT64,
  KC_SOLVE_LAT32,
  KC_ADJOINT,
  KC_COMBINE,
  KC_WATCH,
  KC_SOLVE_ML,
  KC_COUNT
};
const char* kKernelNames[KC_COUNT] = {"stage_residual", "facet_pcg_fp64",
                                      "facet_pcg_mixed",     "recover",              "project_rhs",
                                      "lattice",             "diagnostics",          "pressure",
                                      "facet_pcg_fft_fp64",  "facet_pcg_fft_fp32",   "adjoint",
                                      "combine",             "energy_watchdog",      "facet_pcg_multilevel"};

}  // namespace

namespace dgdf {
// error reporting of the other C-ABI translation units (api3.cu): the same thread-local message
int api_fail(int code, const std::string& msg) { return fail(code, msg); }
void api_clear_error() { g_err.clear(); }
}  // namespace dgdf

struct dg_mesh {
  dgdf::HostMesh hm;
  dgdf::DevMesh dm{};
  dg_params p{};
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  int solver_blocks[2] = {1, 1};
  bool use_lattice = false;
  int lattice_blocks = 0;
  bool tc_available = false;      // the tensor-core recovery is set up (mixed form, <= 2 classes)
  bool use_ml = false;            // multilevel-preconditioned PCG (k_multilevel.cu)
  int grid_div = 1;               // solver grid divided by this while a batch runs lanes
  int ml_blocks = 0;
  std::string lattice_why;
  double last_c = 0.0;            // coefficient of L(u') in the last stage solved
  long long gen = 0;              // bumped by every setter that changes a kernel argument
                                  // (dg_set_viscosity): batch graphs captured earlier are stale
  bool has_lam = false;
  // multipliers of each stage of the current scheme in the last hist_len steps (device, the
  // layout of the solver's lam), their step sizes, and how many are valid
  static constexpr int kMaxStages = 4;
  static constexpr int kHist = 3;
  int hist_len = 0;
  void* hist[kMaxStages][kHist] = {};
  double hist_dt[kMaxStages][kHist] = {};
  int hist_n[kMaxStages] = {};
  int hist_scheme = -1;           // the scheme the history belongs to
  size_t hist_bytes = 0;
  // classical RK4: the running combination of the stage states (FP64 form, or its
  // double-float twin in the mixed form), allocated at the first RK4 step
  double* rk_w = nullptr;
  float2* rk_w_df = nullptr;
  bool udf_valid = false;        // mixed form: u_df holds the double-float image of u
  // energy watchdog (dg_set_energy_watchdog): after every step, flag a growth of ||u||^2 by
  // more than watch_tol (relative); watch = [E of the last step (< 0: none yet), ratio, partials]
  double watch_tol = 0.0;
  double* watch = nullptr;
  double* lattice = nullptr;     // [n_tri][ns][2] staging for lattice I/O
  double* wbuf = nullptr;        // [n_tri][nw] element pressure
  double* pe = nullptr;          // [n_tri][nw] pressure lattice staging
  double* pfac = nullptr;        // [n_facet][nl]
  int* dflag = nullptr;          // finite check
  dgdf::DevStats* host_stats = nullptr;
  // profiling
  bool prof = false;
  struct Rec {
    int kc;
    cudaEvent_t a, b;
    bool owns_a;   // false: a is the previous record's b (chained launches)
  };
  // inside a step, consecutive launches share one event: the end of a launch is the start of
  // the next (a non-kernel operation between them clears prof_prev)
  bool prof_chain = false;
  cudaEvent_t prof_prev = nullptr;
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[KC_COUNT] = {};
  long long prof_n[KC_COUNT] = {};
};

namespace {

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,                         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                \
  } while (0)

template <typename T>
int dalloc(dg_mesh* M, T** out, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(&p, n * sizeof(T));
  if (e != cudaSuccess) return fail(DG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  M->allocs.push_back(p);
  *out = static_cast<T*>(p);
  return DG_OK;
}

template <typename T>
int upload(dg_mesh* M, const T** out, const std::vector<T>& v) {
  T* p = nullptr;
  int rc = dalloc(M, &p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = p;
  return DG_OK;
}

// a float vector (a multiple of 4 long) as float4 words
int upload_f4(dg_mesh* M, const float4** out, const std::vector<float>& v) {
  float4* p = nullptr;
  int rc = dalloc(M, &p, v.size() / 4);
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(float), cudaMemcpyHostToDevice));
  *out = p;
  return DG_OK;
}

std::vector<float> to_float(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

// double -> (hi, lo) float pairs with hi + lo = v to about 48 bits
std::vector<float2> to_dfloat(const std::vector<double>& v) {
  std::vector<float2> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float h = float(v[i]);
    out[i] = make_float2(h, float(v[i] - double(h)));
  }
  return out;
}

cudaEvent_t get_event(dg_mesh* M) {
  if (!M->pool.empty()) {
    cudaEvent_t e = M->pool.back();
    M->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Launch wrapper: records an event pair around the launch when profiling. Inside a step
// (prof_chain) a launch that directly follows another starts at that launch's end event, so
// that a step records one event per kernel boundary; the launch gap is then counted in the
// following kernel's time.
template <typename F>
int launch(dg_mesh* M, int kc, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  bool owns_a = true;
  if (M->prof) {
    if (M->prof_chain && M->prof_prev) {
      a = M->prof_prev;
      owns_a = false;
    } else {
      a = get_event(M);
      cudaEventRecord(a, M->stream);
    }
    b = get_event(M);
  }
  M->prof_prev = nullptr;
  cudaError_t e = f();
  if (e != cudaSuccess) {
    if (M->prof) {   // give back the events of the failed launch
      if (owns_a) M->pool.push_back(a);
      M->pool.push_back(b);
    }
    return fail(DG_ERR_CUDA, std::string("kernel launch (") + kKernelNames[kc] + "): " + cudaGetErrorString(e));
  }
  if (M->prof) {
    cudaEventRecord(b, M->stream);
    M->pending.push_back({kc, a, b, owns_a});
    if (M->prof_chain) M->prof_prev = b;
  }
  return DG_OK;
}

void collect_profile(dg_mesh* M) {
  for (auto& r : M->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      M->prof_ms[r.kc] += ms;
      M->prof_n[r.kc] += 1;
    }
    if (r.owns_a) M->pool.push_back(r.a);
    M->pool.push_back(r.b);
  }
  M->pending.clear();
  M->prof_prev = nullptr;
}

// Synchronise the stream, gather profiling, translate device flags to a status.
int finish(dg_mesh* M, bool check_solver) {
  CK(cudaStreamSynchronize(M->stream));
  collect_profile(M);
  if (!check_solver) return DG_OK;
  CK(cudaMemcpy(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost));
  const int fl = M->host_stats->flags;
  if (fl & dgdf::kFlagBarrierTimeout) return fail(DG_ERR_CUDA, "solver grid barrier timed out");
  if (fl & dgdf::kFlagNonFinite) return fail(DG_ERR_NONFINITE, "non-finite residual in the facet solve");
  if (fl & dgdf::kFlagNotConverged) return fail(DG_ERR_NOT_CONVERGED, "facet solve reached cg_maxit");
  if (fl & dgdf::kFlagEnergyGrowth) {
    double w[2] = {0.0, 0.0};
    CK(cudaMemcpy(w, M->watch, sizeof(w), cudaMemcpyDeviceToHost));
    char buf[192];
    std::snprintf(buf, sizeof(buf),
                  "energy watchdog: ||u||^2 grew by a factor %.6g in one step (tolerance %.3g): the step size "
                  "exceeds the stability limit of the scheme", w[1], M->watch_tol);
    return fail(DG_ERR_UNSTABLE, buf);
  }
  return DG_OK;
}

// Forget the watchdog's last energy (a new state was set): the next step only records it.
int reset_watch(dg_mesh* M) {
  if (!M->watch) return DG_OK;
  const double none = -1.0;
  CK(cudaMemcpyAsync(M->watch, &none, sizeof(double), cudaMemcpyHostToDevice, M->stream));
  return DG_OK;
}

int reset_flags(dg_mesh* M) {
  CK(cudaMemsetAsync(&M->dm.stats->flags, 0, sizeof(int), M->stream));
  return DG_OK;
}

// Mixed form: refresh the double-float twin of u after u was written by anything
// but the recovery (which writes both).
int ensure_udf(dg_mesh* M) {
  if (!M->dm.elem_df || M->udf_valid) return DG_OK;
  const long long n = (long long)M->dm.n_tri * M->dm.nd;
  int rc = launch(M, KC_LATTICE, [&] { return dgdf::launch_to_dfl(M->dm.u, M->dm.u_df, n, M->stream); });
  if (rc == DG_OK) M->udf_valid = true;
  return rc;
}

void forget_history(dg_mesh* M) {
  for (int s = 0; s < dg_mesh::kMaxStages; ++s) M->hist_n[s] = 0;
}

// Persistent solver blocks: the mesh's maximum, divided by the ensemble's lanes while a batch
// runs members on parallel graph branches (so that every solver grid that can run at the
// same time fits on the device together, and no grid barrier waits for another grid's blocks).
int capped(const dg_mesh* M, int nb) {
  if (M->grid_div > 1) nb = std::max(1, nb / M->grid_div);
  return nb;
}

int solve(dg_mesh* M, double warm_scale, int stage = -1, double dt = 0.0, bool homog = false) {
  dgdf::SolveArgs a{};
  a.warm_scale = warm_scale;
  a.homog = homog ? 1 : 0;
  // inside a step: warm start from the same stage of the last steps. lam_s is c_s dt times a
  // smooth function of time, so with equal step sizes the quadratic extrapolation
  // 3 lam(n-1) - 3 lam(n-2) + lam(n-3) is third-order accurate and the linear
  // 2 lam(n-1) - lam(n-2) second-order; one entry, or a changed step size, gives lam(n-1)
  // rescaled by dt / dt(n-1).
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
  a.mixed = M->p.precision == DG_PRECISION_MIXED;
  a.inner_rtol = 1e-3;
  a.max_sweeps = 40;
  a.inner_maxit = M->p.cg_maxit;
  a.floor_rtol = 1e-9;
  if (M->use_lattice) {
    const int nb = capped(M, M->lattice_blocks);
    return launch(M, a.mixed ? KC_SOLVE_LAT32 : KC_SOLVE_LAT64,
                  [&] { return dgdf::launch_solve_lattice(M->dm, a, nb, a.mixed, M->stream); });
  }
  if (M->use_ml) {
    const int nb = capped(M, M->ml_blocks);
    return launch(M, KC_SOLVE_ML, [&] { return dgdf::launch_solve_ml(M->dm, a, nb, M->stream); });
  }
  const int nb = capped(M, M->solver_blocks[a.mixed]);
  return launch(M, a.mixed ? KC_SOLVE_MIXED : KC_SOLVE64, [&] { return dgdf::launch_solve(M->dm, a, nb, M->stream); });
}

// After the solve of RK stage s with step size dt: the new multipliers become the newest
// history entry (the solver already moved the older ones down one slot).
int push_history(dg_mesh* M, int s, double dt) {
  if (M->hist_len == 0) return DG_OK;
  const void* lam = M->dm.lam_is_df ? static_cast<const void*>(M->dm.lam_df) : static_cast<const void*>(M->dm.lam);
  M->prof_prev = nullptr;   // a copy between two launches: no chained profiling event across it
  CK(cudaMemcpyAsync(M->hist[s][0], lam, M->hist_bytes, cudaMemcpyDeviceToDevice, M->stream));
  for (int h = M->hist_len - 1; h > 0; --h) M->hist_dt[s][h] = M->hist_dt[s][h - 1];
  M->hist_dt[s][0] = dt;
  M->hist_n[s] = std::min(M->hist_n[s] + 1, M->hist_len);
  return DG_OK;
}

int check_mesh(const dg_mesh* M) {
  if (!M) return fail(DG_ERR_INVALID_ARG, "NULL mesh");
  return DG_OK;
}

}  // namespace

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

const char* dg_kernel_name(int i) { return (i >= 0 && i < KC_COUNT) ? kKernelNames[i] : nullptr; }

int dg_mesh_create(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, const dg_params* params,
                   dg_mesh** out) {
  return dg_mesh_create_ex(n_tri, tri_vertex_ids, tri_coords, nullptr, params, out);
}

int dg_mesh_create_ex(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, const int8_t* edge_kind,
                      const dg_params* params, dg_mesh** out) {
  g_err.clear();
  if (!out || !params || !tri_vertex_ids || !tri_coords) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  dg_params p = *params;
  if (p.k < 1 || p.k > dgdf::kMaxDegree) return fail(DG_ERR_UNSUPPORTED, "k must be 1..3");
  if (!(p.nu >= 0.0) || !std::isfinite(p.nu)) return fail(DG_ERR_INVALID_ARG, "nu must be finite and >= 0");
  if (!(p.alpha > 0.0) || !std::isfinite(p.alpha)) return fail(DG_ERR_INVALID_ARG, "alpha must be > 0");
  if (p.precision != DG_PRECISION_FP64 && p.precision != DG_PRECISION_MIXED)
    return fail(DG_ERR_INVALID_ARG, "precision must be 0 (FP64) or 1 (mixed)");
  if (!(p.cg_rtol > 0.0)) p.cg_rtol = 1e-13;
  if (p.cg_maxit <= 0) p.cg_maxit = 20000;
  if (p.precond != DG_PRECOND_AUTO && p.precond != DG_PRECOND_BLOCK_JACOBI && p.precond != DG_PRECOND_MULTILEVEL)
    return fail(DG_ERR_INVALID_ARG,
                "precond must be DG_PRECOND_AUTO, DG_PRECOND_BLOCK_JACOBI or DG_PRECOND_MULTILEVEL");
  dg_mesh* M = new dg_mesh();
  M->p = p;
  M->stream = static_cast<cudaStream_t>(p.cuda_stream);
  std::string err;
  int rc = dgdf::build_host_mesh(n_tri, tri_vertex_ids, tri_coords, p.k, p.alpha, M->hm, err, edge_kind);
  if (rc) {
    delete M;
    return fail(rc, err);
  }
  auto cleanup = [&](int code) {
    dg_mesh_destroy(M);
    return code;
  };
  // lattice structure (translation-invariant split-square mesh): renumber facets in lattice
  // order before anything facet-indexed is uploaded
  dgdf::Lattice lat;
  const int lat_fp32 = p.precision == DG_PRECISION_MIXED;
  int lat_blocks = 0;
  if (p.precond == DG_PRECOND_AUTO) {
    dgdf::build_lattice(M->hm, tri_coords, lat, lat_fp32);
    if (lat.ok) lat_blocks = dgdf::lattice_blocks(M->hm.k, lat.N, lat_fp32);
    if (lat.ok && lat_blocks > 0) dgdf::renumber_facets_lattice(M->hm, lat);
    else M->lattice_why = lat.ok ? "lattice solver does not fit on this device" : lat.why;
  }
  const dgdf::HostMesh& hm = M->hm;
  const dgdf::RefTables& ref = hm.ref;
  dgdf::DevMesh& d = M->dm;
  d.k = hm.k;
  d.ns = hm.ns;
  d.nd = hm.nd;
  d.nw = hm.nw;
  d.nl = hm.nl;
  d.nq = ref.nq;
  d.nqf = ref.nqf;
  d.n_tri = int(hm.topo.n_tri);
  d.n_facet = int(hm.topo.n_facet);
  d.n_class = int(hm.classes.size());
  d.n_stencil = hm.n_stencil;
  d.nu = p.nu;
  d.area_total = hm.area_total;
  d.elem_df = p.precision == DG_PRECISION_MIXED ? 1 : 0;
  const int nd = hm.nd, nw = hm.nw, nl = hm.nl, L3 = 3 * nl;
  // class data
  std::vector<double> geo(size_t(d.n_class) * dgdf::kGeo, 0.0), P, G, W, WC;
  for (int c = 0; c < d.n_class; ++c) {
    const dgdf::ClassOps& co = hm.classes[c];
    double* g = &geo[size_t(c) * dgdf::kGeo];
    for (int i = 0; i < 4; ++i) g[dgdf::G_JINV + i] = co.Jinv[i];
    g[dgdf::G_DET] = co.det;
    g[dgdf::G_S] = 1.0 / std::sqrt(co.det);
    for (int e = 0; e < 3; ++e) {
      g[dgdf::G_NRM + 2 * e] = co.normal[e][0];
      g[dgdf::G_NRM + 2 * e + 1] = co.normal[e][1];
      g[dgdf::G_FLEN + e] = co.flen[e];
    }
    // integral over T of the first (constant) basis function, and 1 / its value
    double psi0 = ref.vphi[0];
    double s = 1.0 / std::sqrt(co.det);
    g[dgdf::G_ZINT0] = co.det * 0.5 * psi0 * s;   // psi0 constant; reference area 1/2
    g[dgdf::G_CINV0] = 1.0 / (psi0 * s);
    P.insert(P.end(), co.P.begin(), co.P.end());
    G.insert(G.end(), co.G.begin(), co.G.end());
    W.insert(W.end(), co.W.begin(), co.W.end());
    WC.insert(WC.end(), co.WCt.begin(), co.WCt.end());
  }
  if ((rc = upload(M, &d.vw, ref.vw)) || (rc = upload(M, &d.vphi, ref.vphi)) || (rc = upload(M, &d.vdphi, ref.vdphi)) ||
      (rc = upload(M, &d.fw, ref.fw)) || (rc = upload(M, &d.fphi, ref.fphi)) || (rc = upload(M, &d.fdphi, ref.fdphi)) ||
      (rc = upload(M, &d.lat_inv, ref.lat_inv)) || (rc = upload(M, &d.lat_phi, ref.lat_phi)) ||
      (rc = upload(M, &d.plat_phi, ref.plat_phi)) || (rc = upload(M, &d.mu_lat, ref.mu_lat)) ||
      (rc = upload(M, &d.geo, geo)) || (rc = upload(M, &d.P, P)) || (rc = upload(M, &d.G, G)) ||
      (rc = upload(M, &d.W, W)) || (rc = upload(M, &d.WCt, WC)) || (rc = upload(M, &d.Pdf, to_dfloat(P))) ||
      (rc = upload(M, &d.Gdf, to_dfloat(G))) || (rc = upload(M, &d.tri_class, hm.tri_class)) ||
      (rc = upload(M, &d.tri_nbr, hm.tri_nbr)) || (rc = upload(M, &d.tri_facet, hm.topo.tri_facet)) ||
      (rc = upload(M, &d.tri_nbr_loc, hm.tri_nbr_loc)) || (rc = upload(M, &d.tri_orient, hm.topo.tri_orient)) ||
      (rc = upload(M, &d.facet_sigma, hm.facet_sigma)) || (rc = upload(M, &d.facet_nbr, hm.facet_nbr)) ||
      (rc = upload(M, &d.facet_stencil, hm.facet_stencil)) || (rc = upload(M, &d.facet_tri, hm.topo.facet_tri)) ||
      (rc = upload(M, &d.facet_loc, hm.topo.facet_loc)) || (rc = upload(M, &d.st_blk, hm.stencil_blocks)) ||
      (rc = upload(M, &d.st_binv, hm.stencil_binv)) || (rc = upload(M, &d.st_blk_f, to_float(hm.stencil_blocks))) ||
      (rc = upload(M, &d.st_binv_f, to_float(hm.stencil_binv))))
    return cleanup(rc);
  // inflow / outflow boundaries (Sec. 2.5): facet kinds, and zero inflow data until
  // dg_set_inflow; with outflow facets S has no kernel
  d.has_kernel = hm.has_outflow ? 0 : 1;
  if (hm.has_inflow || hm.has_outflow) {
    if ((rc = upload(M, &d.facet_kind, hm.facet_kind))) return cleanup(rc);
    if (hm.has_inflow) {
      std::vector<double> uq(size_t(d.n_facet) * ref.nqf * 2, 0.0), dm(size_t(d.n_facet) * nl, 0.0);
      if ((rc = upload(M, &d.inflow_q, uq)) || (rc = upload(M, &d.inflow_d, dm))) return cleanup(rc);
    }
  }
  if (d.elem_df && d.n_class <= dgdf::kDnClasses) {
    // normal derivatives of the basis at the facet points, per class
    const int nqf = ref.nqf, ns = hm.ns;
    std::vector<double> dn(size_t(d.n_class) * 3 * nqf * ns);
    for (int c = 0; c < d.n_class; ++c) {
      const dgdf::ClassOps& co = hm.classes[c];
      for (int e = 0; e < 3; ++e) {
        const double m0 = co.Jinv[0] * co.normal[e][0] + co.Jinv[1] * co.normal[e][1];
        const double m1 = co.Jinv[2] * co.normal[e][0] + co.Jinv[3] * co.normal[e][1];
        for (int q = 0; q < nqf; ++q)
          for (int j = 0; j < ns; ++j) {
            const double* g = &ref.fdphi[((size_t(e) * nqf + q) * ns + j) * 2];
            dn[((size_t(c) * 3 + e) * nqf + q) * ns + j] = g[0] * m0 + g[1] * m1;
          }
      }
    }
    // paired image for k_stage_df2: rows of ns values as ceil(ns/2) pairs
    // {hi_j, hi_j+1, lo_j, lo_j+1} (a missing j+1 is 0), in the order of PairTables<K>
    const int ns2 = (ns + 1) / 2, nq = ref.nq;
    std::vector<float> pt;
    auto split = [](double v, float& h, float& l) {
      h = float(v);
      l = float(v - double(h));
    };
    // value (r, j) = src[r * rstride + j * jstride]
    auto rows = [&](const double* src, int nrow, int rstride, int jstride) {
      for (int r = 0; r < nrow; ++r)
        for (int jp = 0; jp < ns2; ++jp) {
          float h0, l0, h1 = 0.f, l1 = 0.f;
          const int j = 2 * jp;
          split(src[size_t(r) * rstride + size_t(j) * jstride], h0, l0);
          if (j + 1 < ns) split(src[size_t(r) * rstride + size_t(j + 1) * jstride], h1, l1);
          pt.insert(pt.end(), {h0, h1, l0, l1});
        }
    };
    rows(ref.vphi.data(), nq, ns, 1);                  // vphi[q][j]
    rows(ref.vdphi.data(), nq, 2 * ns, 2);             // d/dxi1 psi_j at q
    rows(ref.vdphi.data() + 1, nq, 2 * ns, 2);         // d/dxi2
    rows(ref.fphi.data(), 3 * nqf, ns, 1);             // fphi[e][q][j]
    {
      std::vector<double> dnfull(size_t(dgdf::kDnClasses) * 3 * nqf * ns, 0.0);
      std::copy(dn.begin(), dn.end(), dnfull.begin());
      rows(dnfull.data(), dgdf::kDnClasses * 3 * nqf, ns, 1);
    }
    for (int q = 0; q < nq; ++q) {
      float h, l;
      split(ref.vw[q], h, l);
      pt.push_back(h);
      pt.push_back(l);
    }
    for (int q = 0; q < nqf; ++q) {
      float h, l;
      split(ref.fw[q], h, l);
      pt.push_back(h);
      pt.push_back(l);
    }
    while (pt.size() % 4) pt.push_back(0.f);
    d.ptab_words = int(pt.size() / 4);
    // class operators, pairs of consecutive columns
    auto pairs = [&](const std::vector<double>& Mx, int nrow) {
      std::vector<float> out;
      const int nc2 = nd / 2;
      for (int c = 0; c < d.n_class; ++c)
        for (int r = 0; r < nrow; ++r)
          for (int jp = 0; jp < nc2; ++jp) {
            float h0, l0, h1, l1;
            split(Mx[(size_t(c) * nrow + r) * nd + 2 * jp], h0, l0);
            split(Mx[(size_t(c) * nrow + r) * nd + 2 * jp + 1], h1, l1);
            out.insert(out.end(), {h0, h1, l0, l1});
          }
      return out;
    };
    std::vector<float> p2 = pairs(P, nd), g2 = pairs(G, L3);
    if ((rc = upload_f4(M, &d.ptab, pt)) || (rc = upload_f4(M, &d.P2, p2)) || (rc = upload_f4(M, &d.G2, g2)))
      return cleanup(rc);
  }
  if (d.elem_df && d.ptab && d.n_class <= 2) {
    // tensor-core recovery: per class, tiles of 128 triangles, and the class operator
    // B = [P, -G^T] (B[n][k], n < n_u output, k < n_u + 3(k+1) input) split into kTcSlices
    // signed 8-bit digits per column scale, stored in the kernel's K-major tile layout
    constexpr int S = 7;
    int KP = 0, NP = 0;
    dgdf::tc_dims(hm.k, &KP, &NP);
    std::vector<int32_t> rows, tcls;
    for (int c = 0; c < d.n_class; ++c) {
      std::vector<int32_t> mine;
      for (int t = 0; t < d.n_tri; ++t)
        if (hm.tri_class[t] == c) mine.push_back(t);
      for (size_t i = 0; i < mine.size(); i += 128) {
        for (size_t j = 0; j < 128; ++j) rows.push_back(i + j < mine.size() ? mine[i + j] : -1);
        tcls.push_back(c);
      }
    }
    auto core_off = [&](int row, int k) {
      return size_t((row >> 3) * (KP / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2) / 2;
    };
    std::vector<uint16_t> bb(size_t(d.n_class) * S * NP * KP, 0);
    std::vector<int32_t> ec(size_t(d.n_class) * NP, 0);
    for (int c = 0; c < d.n_class; ++c) {
      const dgdf::ClassOps& co = hm.classes[c];
      for (int n = 0; n < NP; ++n) {
        std::vector<double> col(KP, 0.0);
        if (n < nd)
          for (int k = 0; k < nd + L3; ++k)
            col[k] = k < nd ? co.P[size_t(n) * nd + k] : -co.G[size_t(k - nd) * nd + n];
        double mx = 0.0;
        for (double v : col) mx = std::max(mx, std::fabs(v));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);
        ec[size_t(c) * NP + n] = e;
        for (int k = 0; k < KP; ++k) {
          double t = std::ldexp(col[k], -e);
          for (int sl = 0; sl < S; ++sl) {
            const double x = t * 256.0, dg = std::nearbyint(x);
            t = x - dg;
            const float df = float(dg);
            uint32_t bits;
            std::memcpy(&bits, &df, 4);
            bb[(size_t(c) * S + sl) * NP * KP + core_off(n, k)] = uint16_t(bits >> 16);
          }
        }
      }
    }
    if ((rc = upload(M, &d.tc_rows, rows)) || (rc = upload(M, &d.tc_tile_cls, tcls)) ||
        (rc = upload(M, &d.tc_b, bb)) || (rc = upload(M, &d.tc_ec, ec)))
      return cleanup(rc);
    d.tc_tiles = int(tcls.size());
    d.tc_rec = 0;   // off by default: the double-float recovery is faster (dg_set_tensor_cores)
    M->tc_available = true;
  }
  if (d.elem_df) {
    // reference tables in the field order of the kernels' shared-memory image
    std::vector<double> tab;
    for (const std::vector<double>* v : {&ref.vw, &ref.vphi, &ref.vdphi, &ref.fw, &ref.fphi, &ref.fdphi})
      tab.insert(tab.end(), v->begin(), v->end());
    if ((rc = upload(M, &d.tab_df, to_dfloat(tab))) || (rc = upload(M, &d.geo_df, to_dfloat(geo))) ||
        (rc = upload(M, &d.sigma_df, to_dfloat(hm.facet_sigma))))
      return cleanup(rc);
  }
  const size_t nT = size_t(d.n_tri), nF = size_t(d.n_facet);
  const size_t nred = std::max<size_t>(size_t(dgdf::kRedSlots) * dgdf::kMaxSolverBlocks, nT / 128 + 2);
  if ((rc = dalloc(M, &d.u, nT * nd)) || (rc = dalloc(M, &d.ustage, nT * nd)) || (rc = dalloc(M, &d.h, nT * nd)) ||
      (rc = dalloc(M, &d.gl, nT * L3)) ||
      (rc = dalloc(M, &d.lam, nF * nl)) || (rc = dalloc(M, &d.g, nF * nl)) || (rc = dalloc(M, &d.r, nF * nl)) ||
      (rc = dalloc(M, &d.z, nF * nl)) || (rc = dalloc(M, &d.pa, nF * nl)) || (rc = dalloc(M, &d.pb, nF * nl)) ||
      (rc = dalloc(M, &d.q, nF * nl)) || (rc = dalloc(M, &d.rf, nF * nl)) || (rc = dalloc(M, &d.zf, nF * nl)) ||
      (rc = dalloc(M, &d.paf, nF * nl)) || (rc = dalloc(M, &d.pbf, nF * nl)) || (rc = dalloc(M, &d.qf, nF * nl)) ||
      (rc = dalloc(M, &d.xf, nF * nl)) || (rc = dalloc(M, &d.red, nred)) || (rc = dalloc(M, &d.bar, 1)) ||
      (rc = dalloc(M, &d.stats, 1)) || (rc = dalloc(M, &d.diag, 8)) ||
      (rc = dalloc(M, &M->lattice, nT * hm.ns * 2)) || (rc = dalloc(M, &M->wbuf, nT * nw)) ||
      (rc = dalloc(M, &M->pe, nT * nw)) || (rc = dalloc(M, &M->pfac, nF * nl)) || (rc = dalloc(M, &M->dflag, 1)))
    return cleanup(rc);
  if (d.elem_df && ((rc = dalloc(M, &d.u_df, nT * nd)) || (rc = dalloc(M, &d.ustage_df, nT * nd)) ||
                    (rc = dalloc(M, &d.h_df, nT * nd)) || (rc = dalloc(M, &d.gl_df, nT * L3))))
    return cleanup(rc);
  cudaError_t e = cudaMallocHost(&M->host_stats, sizeof(dgdf::DevStats));
  if (e != cudaSuccess) return cleanup(fail(DG_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e)));
  e = cudaMemsetAsync(d.u, 0, nT * nd * sizeof(double), M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.lam, 0, nF * nl * sizeof(double), M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.stats, 0, sizeof(dgdf::DevStats), M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  if (e != cudaSuccess) return cleanup(fail(DG_ERR_CUDA, std::string("initialise: ") + cudaGetErrorString(e)));
  M->solver_blocks[0] = dgdf::solver_max_blocks(d, 0);
  M->solver_blocks[1] = dgdf::solver_max_blocks(d, 1);
  // multilevel preconditioner: asked for, or the default where the lattice path is not taken
  if (p.precond == DG_PRECOND_MULTILEVEL || (p.precond == DG_PRECOND_AUTO && !(lat.ok && lat_blocks > 0))) {
    dgdf::MLHost mlh;
    std::string merr;
    if ((rc = dgdf::build_multilevel(M->hm, mlh, merr))) return cleanup(fail(rc, merr));
    // the V-cycle's precision: FP32 in the mixed form (a preconditioner needs no more; the PCG
    // vectors and S stay FP64), FP64 in the FP64 form
    const bool ml32 = p.precision == DG_PRECISION_MIXED;
    auto f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    auto fill = [&](auto& lv, auto conv, auto* cpinv_out, auto** xc, auto** bc) -> int {
      for (size_t l = 0; l < mlh.lv.size(); ++l) {
        const dgdf::MLHostLevel& H = mlh.lv[l];
        auto& L = lv[l];
        using T = std::remove_pointer_t<decltype(L.x)>;
        L.stencil = H.stencil ? 1 : 0;
        L.bs = H.bs;
        L.n = H.n;
        L.inject = H.inject ? 1 : 0;
        L.n_next = H.n_next;
        L.bs_next = H.bs_next;
        L.c0 = T(H.cheb[0]);
        L.c1 = T(H.cheb[1]);
        L.c2 = T(H.cheb[2]);
        int rc2 = 0;
        if ((rc2 = upload(M, &L.binv, conv(H.binv)))) return rc2;
        if (!H.stencil && ((rc2 = upload(M, &L.a_rp, H.A.rp)) || (rc2 = upload(M, &L.a_ci, H.A.ci)) ||
                           (rc2 = upload(M, &L.a_v, conv(H.A.v)))))
          return rc2;
        if (!H.inject && ((rc2 = upload(M, &L.p_rp, H.P.rp)) || (rc2 = upload(M, &L.p_ci, H.P.ci)) ||
                          (rc2 = upload(M, &L.p_v, conv(H.P.v))) || (rc2 = upload(M, &L.r_rp, H.R.rp)) ||
                          (rc2 = upload(M, &L.r_ci, H.R.ci)) || (rc2 = upload(M, &L.r_v, conv(H.R.v)))))
          return rc2;
        const size_t nv = size_t(H.n) * H.bs;
        if constexpr (std::is_same<T, double>::value) {
          if (l == 0) {   // level 0 works on the PCG vectors: b = r, x = z
            L.b = d.r;
            L.x = d.z;
          }
        }
        if (!L.b && ((rc2 = dalloc(M, &L.b, nv)) || (rc2 = dalloc(M, &L.x, nv)))) return rc2;
        if ((rc2 = dalloc(M, &L.r, nv)) || (rc2 = dalloc(M, &L.d, nv))) return rc2;
      }
      int rc2 = 0;
      if ((rc2 = upload(M, cpinv_out, conv(mlh.cpinv))) || (rc2 = dalloc(M, xc, size_t(mlh.nc))) ||
          (rc2 = dalloc(M, bc, size_t(mlh.nc))))
        return rc2;
      return 0;
    };
    if (ml32) {
      std::vector<dgdf::MLLevelT<float>> lv(mlh.lv.size());
      if ((rc = fill(lv, f32, &d.ml_cpinv_f, &d.ml_xc_f, &d.ml_bc_f))) return cleanup(rc);
      const dgdf::MLLevelT<float>* lvd = nullptr;
      if ((rc = upload(M, &lvd, lv))) return cleanup(rc);
      d.ml_lv_f = lvd;
    } else {
      std::vector<dgdf::MLLevelDev> lv(mlh.lv.size());
      if ((rc = fill(lv, [](const std::vector<double>& v) { return v; }, &d.ml_cpinv, &d.ml_xc, &d.ml_bc)))
        return cleanup(rc);
      const dgdf::MLLevelDev* lvd = nullptr;
      if ((rc = upload(M, &lvd, lv))) return cleanup(rc);
      d.ml_lv = lvd;
    }
    d.ml_nlev = int(mlh.lv.size());
    d.ml_nc = mlh.nc;
    M->use_ml = d.ml_nlev >= 1;
    M->ml_blocks = dgdf::solver_ml_blocks(d);
    if (M->use_ml && M->ml_blocks < 1) return cleanup(fail(DG_ERR_CUDA, "multilevel solver does not fit"));
  }
  if (lat.ok && lat_blocks > 0) {
    const int fp32 = lat_fp32;
    const int C = lat.C, N = lat.N;
    // device layout [ki < N/2+1][entry][kj] complex: the residual is real, so only half the
    // wavenumbers along i are needed.
    //  FP32: the deflated eigen form of each Hermitian block: the eigen-pair of its largest
    //        eigenvalue (v1, 1/mu1), then the packed upper triangle of the rest. The one
    //        near-singular direction of the symbol at small kappa is applied on its own,
    //        so no cancellation happens in FP32; the explicit inverse rounded to FP32 loses
    //        accuracy there;
    //  FP64: all C*C entries of the inverse, the self-conjugate columns ki = 0 and ki = N/2
    //        symmetrised (the half-spectrum transform takes S^(-kappa) = conj S^(kappa) for
    //        granted, and the host inverts each wavenumber on its own).
    const int NK = N / 2 + 1, NP = fp32 ? C + 1 + C * (C + 1) / 2 : C * C;
    // split column pass: within a wavenumber row the even kj come first, then the odd ones
    const bool split = dgdf::lattice_split(N);
    auto kjs = [&](int kj) { return split ? (kj & 1) * (N / 2) + (kj >> 1) : kj; };
    const size_t nS = dgdf::lattice_symbol_elems(hm.k, N, fp32);
    std::vector<double> sd;
    std::vector<float> sf;
    if (fp32) {
      // deflated eigen form: the dominant pair (v1, 1/mu1) of the inverse, kept apart, and
      // the packed upper triangle of the remainder sum_{i != 1} v_i v_i^H / mu_i (cond ~ 10)
      sf.resize(2 * nS);
      const int NE = C * C + C;
      std::vector<double> Hr(size_t(C) * C * 2);
      for (int ki = 0; ki < NK; ++ki)
        for (int kj = 0; kj < N; ++kj) {
          const double* E = &lat.seig[(size_t(ki) * N + kj) * NE * 2];
          auto V = [&](int b, int i, int ri) { return E[(b * C + i) * 2 + ri]; };
          auto dinv = [&](int i) { return E[(C * C + i) * 2]; };
          int i1 = 0;
          for (int i = 1; i < C; ++i)
            if (dinv(i) > dinv(i1)) i1 = i;
          std::fill(Hr.begin(), Hr.end(), 0.0);
          for (int i = 0; i < C; ++i) {
            if (i == i1) continue;
            for (int ca = 0; ca < C; ++ca)
              for (int cb = 0; cb < C; ++cb) {
                // V_ai conj(V_bi) d_i
                const double ar = V(ca, i, 0), ai = V(ca, i, 1), br = V(cb, i, 0), bi = V(cb, i, 1);
                Hr[(ca * C + cb) * 2] += dinv(i) * (ar * br + ai * bi);
                Hr[(ca * C + cb) * 2 + 1] += dinv(i) * (ai * br - ar * bi);
              }
          }
          auto put = [&](int e, double re, double im) {
            const size_t o = ((size_t(ki) * NP + e) * N + kjs(kj)) * 2;
            sf[o] = float(re);
            sf[o + 1] = float(im);
          };
          for (int b = 0; b < C; ++b) put(b, V(b, i1, 0), V(b, i1, 1));
          put(C, dinv(i1), 0.0);
          int pi = C + 1;
          for (int ca = 0; ca < C; ++ca)
            for (int cb = ca; cb < C; ++cb, ++pi)
              put(pi, Hr[(ca * C + cb) * 2], ca == cb ? 0.0 : Hr[(ca * C + cb) * 2 + 1]);
        }
    } else {
      sd.resize(2 * nS);
      auto H = [&](int ki, int kj, int ca, int cb, int ri) {
        return lat.sinv[((size_t(ki) * N + kj) * C * C + size_t(ca) * C + cb) * 2 + ri];
      };
      for (int ki = 0; ki < NK; ++ki) {
        const bool selfconj = ki == 0 || 2 * ki == N;
        for (int kj = 0; kj < N; ++kj) {
          const int mj = (N - kj) % N;
          for (int ca = 0; ca < C; ++ca)
            for (int cb = 0; cb < C; ++cb) {
              double re = H(ki, kj, ca, cb, 0), im = H(ki, kj, ca, cb, 1);
              if (selfconj) {
                re = 0.5 * (re + H(ki, mj, ca, cb, 0));
                im = 0.5 * (im - H(ki, mj, ca, cb, 1));
              }
              const size_t o = ((size_t(ki) * NP + ca * C + cb) * N + kjs(kj)) * 2;
              sd[o] = re;
              sd[o + 1] = im;
            }
        }
      }
    }
    std::vector<double>().swap(lat.sinv);
    std::vector<double>().swap(lat.seig);
    const int32_t* fo = nullptr;
    const int32_t* fe = nullptr;
    const double* tw = nullptr;
    if ((rc = upload(M, &fo, lat.facet_of)) || (rc = upload(M, &tw, lat.twiddle)) ||
        (rc = upload(M, &fe, hm.facet_ext)))
      return cleanup(rc);
    if (fp32) {
      const float* sp = nullptr;
      if ((rc = upload(M, &sp, sf))) return cleanup(rc);
      d.lat_sinv = sp;
      float* xp = nullptr;
      if ((rc = dalloc(M, &xp, 2 * dgdf::lattice_spectrum_elems(hm.k, N)))) return cleanup(rc);
      d.lat_x = xp;
      if (split) {
        float* x2 = nullptr;
        if ((rc = dalloc(M, &x2, 2 * dgdf::lattice_spectrum_elems(hm.k, N)))) return cleanup(rc);
        d.lat_x2 = x2;
      }
      // the mixed lattice solver keeps its multipliers and work vectors in double-float,
      // facet stride padded to an aligned access (4 for k = 2)
      d.lat_vs = nl == 3 ? 4 : nl;
      const size_t nv = nF * size_t(d.lat_vs);
      if ((rc = dalloc(M, &d.lam_df, nv)) || (rc = dalloc(M, &d.lv_g, nv)) || (rc = dalloc(M, &d.lv_r, nv)) ||
          (rc = dalloc(M, &d.lv_q, nv)) || (rc = dalloc(M, &d.lv_p, nv)) || (rc = dalloc(M, &d.lv_z, nv)) ||
          (rc = upload(M, &d.st_blk_df, to_dfloat(hm.stencil_blocks))))
        return cleanup(rc);
      if (cudaMemsetAsync(d.lam_df, 0, nv * sizeof(float2), M->stream) != cudaSuccess)
        return cleanup(fail(DG_ERR_CUDA, "initialise the double-float multipliers"));
      d.lam_is_df = 1;
    } else {
      const double* sp = nullptr;
      if ((rc = upload(M, &sp, sd))) return cleanup(rc);
      d.lat_sinv = sp;
      double* xp = nullptr;
      if ((rc = dalloc(M, &xp, 2 * dgdf::lattice_spectrum_elems(hm.k, N)))) return cleanup(rc);
      d.lat_x = xp;
      if (split) {
        double* x2 = nullptr;
        if ((rc = dalloc(M, &x2, 2 * dgdf::lattice_spectrum_elems(hm.k, N)))) return cleanup(rc);
        d.lat_x2 = x2;
      }
    }
    d.lat_facet_of = fo;
    d.facet_ext = fe;
    d.lat_tw = tw;
    d.lat_N = N;
    d.lat_bufsz = int(dgdf::lattice_buffer_elems(hm.k, N, fp32));
    d.lat_grp = dgdf::lattice_group_rows(hm.k, N, fp32);
    d.lat_split = split ? 1 : 0;
    d.lat_tw2_off = int(dgdf::lattice_tw2_offset(hm.k, N, fp32, d.lat_grp));
    int logn = 0;
    while ((1 << logn) < N) ++logn;
    d.lat_logn = logn;
    M->use_lattice = true;
    M->lattice_blocks = lat_blocks;
  }
  // multiplier history of the stages (warm starts), in the layout of the solver's lam: two
  // entries on the lattice path (its solves take two PCG iterations from the linear
  // extrapolation already; a third entry did not lower that count), three for the others
  M->hist_len = M->use_lattice ? 2 : 3;
  M->hist_bytes = size_t(M->dm.n_facet) * size_t(M->use_lattice && lat_fp32 ? M->dm.lat_vs : M->hm.k + 1) * 8;
  for (int s = 0; s < dg_mesh::kMaxStages; ++s)
    for (int h = 0; h < M->hist_len; ++h) {
      double* p = nullptr;
      if ((rc = dalloc(M, &p, M->hist_bytes / 8))) return cleanup(rc);
      M->hist[s][h] = p;
    }
  *out = M;
  return DG_OK;
}

int dg_mesh_destroy(dg_mesh* M) {
  if (!M) return DG_OK;
  cudaStreamSynchronize(M->stream);
  for (void* p : M->allocs) cudaFree(p);
  for (auto& r : M->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : M->pool) cudaEventDestroy(e);
  if (M->host_stats) cudaFreeHost(M->host_stats);
  delete M;
  return DG_OK;
}

int dg_mesh_info(const dg_mesh* M, int64_t out[8]) {
  if (int rc = check_mesh(M)) return rc;
  if (!out) return fail(DG_ERR_INVALID_ARG, "NULL out");
  out[0] = M->hm.topo.n_tri;
  out[1] = M->hm.topo.n_facet;
  out[2] = M->hm.k;
  out[3] = M->hm.ns;
  out[4] = int64_t(M->hm.classes.size());
  out[5] = M->hm.n_stencil;
  out[6] = M->hm.topo.n_tri * M->hm.nd;
  out[7] = M->hm.topo.n_facet * M->hm.nl;
  return DG_OK;
}

int dg_set_velocity(dg_mesh* M, const double* vals, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!vals) return fail(DG_ERR_INVALID_ARG, "NULL vals");
  const size_t n = size_t(M->dm.n_tri) * M->hm.ns * 2;
  CK(cudaMemcpyAsync(M->lattice, vals, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     M->stream));
  CK(cudaMemsetAsync(M->dflag, 0, sizeof(int), M->stream));
  int rc = launch(M, KC_LATTICE, [&] { return dgdf::launch_check_finite(M->lattice, (long long)n, M->dflag, M->stream); });
  if (rc) return rc;
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, M->dflag, sizeof(int), cudaMemcpyDeviceToHost, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  if (flag) return fail(DG_ERR_NONFINITE, "non-finite velocity value");
  rc = launch(M, KC_LATTICE, [&] { return dgdf::launch_lattice_to_coef(M->dm, M->lattice, M->dm.u, M->stream); });
  if (rc) return rc;
  // the solver's multipliers of the last stages and steps stay: they only set the initial guess
  // of the next solves (a state that continues the trajectory keeps its short solves)
  M->udf_valid = false;
  if ((rc = reset_watch(M))) return rc;
  return finish(M, false);
}

int dg_get_velocity(dg_mesh* M, double* vals, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!vals) return fail(DG_ERR_INVALID_ARG, "NULL vals");
  const size_t n = size_t(M->dm.n_tri) * M->hm.ns * 2;
  int rc = launch(M, KC_LATTICE, [&] { return dgdf::launch_coef_to_lattice(M->dm, M->dm.u, M->lattice, M->stream); });
  if (rc) return rc;
  CK(cudaMemcpyAsync(vals, M->lattice, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     M->stream));
  return finish(M, false);
}

int dg_project_divfree(dg_mesh* M) {
  if (int rc = check_mesh(M)) return rc;
  int rc = reset_flags(M);
  if (rc) return rc;
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_PROJECT;
  a.up = M->dm.u;
  a.un = M->dm.u;
  if ((rc = ensure_udf(M))) return rc;
  a.up_df = M->dm.u_df;
  a.un_df = M->dm.u_df;
  if ((rc = launch(M, KC_PROJECT_RHS, [&] { return dgdf::launch_stage(M->dm, a, M->stream); }))) return rc;
  if ((rc = solve(M, 0.0))) return rc;
  if ((rc = launch(M, KC_RECOVER, [&] { return dgdf::launch_recover(M->dm, M->dm.u, M->dm.u_df, M->stream); })))
    return rc;
  M->has_lam = false;
  forget_history(M);
  if ((rc = reset_watch(M))) return rc;
  return finish(M, true);
}

}  // extern "C"

namespace {

// Explicit schemes in stage form. Stage s solves M u_s = a M x + b M u' + c dt L(u') on the
// divergence-free space, with u' = u^n for s = 0 and the previous stage's state otherwise,
// and x = u^n, or (xw) the running combination W. After stage s, W <- wx X + wb u_s with
// X = u^n, or (wacc) X = W. The last stage's state is u^(n+1).
struct StageCoef {
  bool xw;
  double a, b, c;
  int wop;   // 0: W unchanged; 1: W = wx u^n + wb u_s; 2: W = wx W + wb u_s
  double wx, wb;
};
struct Scheme {
  int n;
  StageCoef st[dg_mesh::kMaxStages];
};
const Scheme kSchemes[3] = {
    // SSP-RK3, eq. (8): u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1));
    // u^(n+1) = 1/3 u + 2/3 (u2 + dt L(u2))
    {3,
     {{false, 0.0, 1.0, 1.0, 0, 0.0, 0.0},
      {false, 0.75, 0.25, 0.25, 0, 0.0, 0.0},
      {false, 1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0, 0.0, 0.0}}},
    // forward Euler, eq. (FE) of Sec. 3.1 (with the full L, viscous terms included)
    {1, {{false, 0.0, 1.0, 1.0, 0, 0.0, 0.0}}},
    // classical RK4 (Example 1b): u1 = u + dt/2 k1, u2 = u + dt/2 k2, u3 = u + dt k3 with
    // k_i the projected L of the previous state; u^(n+1) = u + dt/6 (k1 + 2 k2 + 2 k3 + k4)
    // = W + 1/3 u3 + dt/6 L(u3) with W = (-u + u1 + 2 u2) / 3
    {4,
     {{false, 0.0, 1.0, 0.5, 1, -1.0 / 3.0, 1.0 / 3.0},
      {false, 1.0, 0.0, 0.5, 2, 1.0, 2.0 / 3.0},
      {false, 1.0, 0.0, 1.0, 0, 0.0, 0.0},
      {true, 1.0, 1.0 / 3.0, 1.0 / 6.0, 0, 0.0, 0.0}}},
};

// the warm-start history holds multipliers of one scheme's stages
void use_scheme(dg_mesh* M, int scheme) {
  if (M->hist_scheme != scheme) {
    forget_history(M);
    M->hist_scheme = scheme;
  }
}

int ensure_rk_w(dg_mesh* M) {
  const size_t n = size_t(M->dm.n_tri) * M->dm.nd;
  if (M->dm.elem_df) return M->rk_w_df ? DG_OK : dalloc(M, &M->rk_w_df, n);
  return M->rk_w ? DG_OK : dalloc(M, &M->rk_w, n);
}

// Enqueue one step of the given scheme on M's stream: per stage the residual +
// condensation kernel, the facet solve (warm-started from the previous stage's
// multipliers rescaled by the ratio of the L coefficients, or from the same stage of the
// last steps) and the recovery. No synchronisation.
struct ProfChain {   // chained profiling events for the launches of one step
  dg_mesh* M;
  explicit ProfChain(dg_mesh* m) : M(m) { M->prof_chain = true; }
  ~ProfChain() {
    M->prof_chain = false;
    M->prof_prev = nullptr;
  }
};

int enqueue_step(dg_mesh* M, double dt, int scheme = DG_SCHEME_SSPRK3) {
  ProfChain chain(M);
  dgdf::DevMesh& d = M->dm;
  const Scheme& sc = kSchemes[scheme];
  int rc = ensure_udf(M);
  if (rc) return rc;
  if (sc.st[sc.n - 1].xw || sc.st[0].wop) {
    if ((rc = ensure_rk_w(M))) return rc;
  }
  use_scheme(M, scheme);
  const long long n = (long long)d.n_tri * d.nd;
  for (int s = 0; s < sc.n; ++s) {
    const StageCoef& k = sc.st[s];
    const bool last = s == sc.n - 1;
    // mixed form: the next stage reads only the double-float twin, so the FP64 copy of an
    // intermediate stage is not written
    double* out = last ? d.u : (d.elem_df ? nullptr : d.ustage);
    float2* out_df = last ? d.u_df : d.ustage_df;
    dgdf::StageArgs sa{};
    sa.mode = dgdf::MODE_STAGE;
    sa.a = k.a;
    sa.b = k.b;
    sa.c = k.c * dt;
    sa.un = k.xw ? M->rk_w : d.u;
    sa.up = (s == 0) ? d.u : d.ustage;
    sa.un_df = k.xw ? M->rk_w_df : d.u_df;
    sa.up_df = (s == 0) ? d.u_df : d.ustage_df;
    if ((rc = launch(M, KC_STAGE, [&] { return dgdf::launch_stage(d, sa, M->stream); }))) return rc;
    const double warm = M->has_lam ? sa.c / M->last_c : 0.0;
    if ((rc = solve(M, warm, s, dt))) return rc;
    if ((rc = launch(M, KC_RECOVER, [&] { return dgdf::launch_recover(d, out, out_df, M->stream); }))) return rc;
    if ((rc = push_history(M, s, dt))) return rc;
    M->last_c = sa.c;
    M->has_lam = true;
    if (k.wop) {
      const bool acc = k.wop == 2;
      rc = launch(M, KC_COMBINE, [&] {
        return d.elem_df ? dgdf::launch_axpby_df(acc ? M->rk_w_df : d.u_df, d.ustage_df, M->rk_w_df, k.wx, k.wb, n,
                                                 M->stream)
                         : dgdf::launch_axpby64(acc ? M->rk_w : d.u, d.ustage, M->rk_w, k.wx, k.wb, n, M->stream);
      });
      if (rc) return rc;
    }
  }
  if (M->watch_tol > 0.0) {
    rc = launch(M, KC_WATCH, [&] {
      return dgdf::launch_energy_watch(d.u, n, M->watch, M->watch_tol, d.stats, M->stream);
    });
    if (rc) return rc;
  }
  return DG_OK;
}

}  // namespace

struct dg_batch {
  std::vector<dg_mesh*> members;
  cudaStream_t user = nullptr;     // the caller's stream
  cudaStream_t stream = nullptr;   // the batch's own stream: graphs are captured and replayed here
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double> graph_dt;
  std::vector<long long> graph_gen;   // each member's gen when the graph was captured
  // lanes: members are dealt out to this many parallel branches of the captured step (0: the
  // autotuner picks it on the next call); the branch streams, their join events
  int lanes = 0;
  int graph_lanes = 0;                 // lanes of the captured graph
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_events;
  double tune_ms[5] = {-1.0, -1.0, -1.0, -1.0, -1.0};   // measured step time for 1, 2, 4, 8, 16 lanes
};

extern "C" {

int dg_step(dg_mesh* M, int scheme, double dt, int64_t nsteps) {
  if (int rc = check_mesh(M)) return rc;
  if (scheme != DG_SCHEME_SSPRK3 && scheme != DG_SCHEME_EULER && scheme != DG_SCHEME_RK4)
    return fail(DG_ERR_INVALID_ARG, "scheme must be DG_SCHEME_SSPRK3, DG_SCHEME_EULER or DG_SCHEME_RK4");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  int rc = reset_flags(M);
  if (rc) return rc;
  for (int64_t n = 0; n < nsteps; ++n)
    if ((rc = enqueue_step(M, dt, scheme))) return rc;
  return finish(M, true);
}

int dg_rk3_step(dg_mesh* M, double dt, int64_t nsteps) { return dg_step(M, DG_SCHEME_SSPRK3, dt, nsteps); }

int dg_batch_create(int n, dg_mesh* const* meshes, void* cuda_stream, dg_batch** out) {
  g_err.clear();
  if (!out || n < 1 || !meshes) return fail(DG_ERR_INVALID_ARG, "need n >= 1 meshes and an output pointer");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return fail(DG_ERR_INVALID_ARG, "NULL member mesh");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == meshes[i]) return fail(DG_ERR_INVALID_ARG, "a mesh appears twice in the batch");
  }
  dg_batch* B = new dg_batch();
  B->members.assign(meshes, meshes + n);
  B->user = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    dg_batch_destroy(B);
    return fail(DG_ERR_CUDA, std::string("dg_batch_create: ") + cudaGetErrorString(e));
  }
  *out = B;
  return DG_OK;
}

int dg_batch_destroy(dg_batch* B) {
  if (!B) return DG_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->ev) cudaEventDestroy(B->ev);
  for (cudaEvent_t e : B->lane_events) cudaEventDestroy(e);
  for (cudaStream_t st : B->lane_streams) cudaStreamDestroy(st);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
  return DG_OK;
}

int dg_batch_set_lanes(dg_batch* B, int lanes) {
  if (!B) return fail(DG_ERR_INVALID_ARG, "NULL batch");
  if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16)
    return fail(DG_ERR_INVALID_ARG, "lanes must be 0 (autotune), 1, 2, 4, 8 or 16");
  B->lanes = lanes;
  if (lanes == 0)
    for (double& t : B->tune_ms) t = -1.0;
  return DG_OK;
}

int dg_batch_get_tuning(dg_batch* B, int* lanes, double ms[5]) {
  if (!B) return fail(DG_ERR_INVALID_ARG, "NULL batch");
  if (lanes) *lanes = B->lanes;
  if (ms)
    for (int i = 0; i < 5; ++i) ms[i] = B->tune_ms[i];
  return DG_OK;
}

namespace {

// Capture one SSP-RK3 step of every member as B's graph: members dealt out (largest first, to
// the least loaded) to `lanes` parallel branches forked from and joined into the batch stream;
// each member's solver grid is divided by the lanes for the capture.
int capture_batch_step(dg_batch* B, const double* dt, int lanes) {
  const size_t n = B->members.size();
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
  B->graph_lanes = 0;
  lanes = std::max(1, std::min(lanes, int(n)));
  while (int(B->lane_streams.size()) < lanes) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(DG_ERR_CUDA, "dg_batch_rk3_step: lane stream");
    B->lane_streams.push_back(st);
    B->lane_events.push_back(ev);
  }
  // largest members first, each to the lane with the least work so far
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  auto work = [&](size_t i) { return double(B->members[i]->dm.n_tri) * B->members[i]->dm.nd; };
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work(a) > work(b); });
  std::vector<double> load(lanes, 0.0);
  std::vector<int> lane_of(n, 0);
  for (size_t i : order) {
    const int l = int(std::min_element(load.begin(), load.end()) - load.begin());
    lane_of[i] = l;
    load[l] += work(i);
  }
  for (dg_mesh* M : B->members) M->prof = false;   // no timing events inside the graph
  cudaError_t e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  int rc = DG_OK;
  if (lanes > 1) {
    e = cudaEventRecord(B->ev, B->stream);
    for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(B->lane_streams[l], B->ev, 0);
    if (e != cudaSuccess) rc = fail(DG_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
  }
  for (size_t i = 0; i < n && rc == DG_OK; ++i) {
    dg_mesh* M = B->members[i];
    M->stream = lanes > 1 ? B->lane_streams[lane_of[i]] : B->stream;
    M->grid_div = lanes;
    rc = enqueue_step(M, dt[i]);
    M->grid_div = 1;
    M->stream = B->stream;
  }
  if (lanes > 1 && rc == DG_OK) {
    for (int l = 0; l < lanes && e == cudaSuccess; ++l) {
      e = cudaEventRecord(B->lane_events[l], B->lane_streams[l]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->lane_events[l], 0);
    }
    if (e != cudaSuccess) rc = fail(DG_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(B->stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&B->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(DG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  B->graph = g;
  B->graph_lanes = lanes;
  B->graph_dt.assign(dt, dt + n);
  B->graph_gen.resize(n);
  for (size_t i = 0; i < n; ++i) B->graph_gen[i] = B->members[i]->gen;
  return DG_OK;
}

}  // namespace

int dg_batch_rk3_step(dg_batch* B, const double* dt, int64_t nsteps) {
  if (!B) return fail(DG_ERR_INVALID_ARG, "NULL batch");
  if (!dt) return fail(DG_ERR_INVALID_ARG, "NULL dt");
  if (nsteps < 0) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 0");
  const size_t n = B->members.size();
  for (size_t i = 0; i < n; ++i)
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(DG_ERR_INVALID_ARG, "every dt must be finite and > 0");
  if (nsteps == 0) return DG_OK;
  // every member runs on the batch stream for the duration of the call
  std::vector<cudaStream_t> saved(n);
  std::vector<bool> saved_prof(n);
  for (size_t i = 0; i < n; ++i) {
    saved[i] = B->members[i]->stream;
    saved_prof[i] = B->members[i]->prof;
    B->members[i]->stream = B->stream;
  }
  auto restore = [&](int code) {
    for (size_t i = 0; i < n; ++i) {
      B->members[i]->stream = saved[i];
      B->members[i]->prof = saved_prof[i];
    }
    return code;
  };
  int rc = DG_OK;
  // order after the caller's stream, then work on the batch's own stream
  cudaError_t e0 = cudaEventRecord(B->ev, B->user);
  if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(B->stream, B->ev, 0);
  if (e0 != cudaSuccess) return restore(fail(DG_ERR_CUDA, std::string("dg_batch_rk3_step: ") + cudaGetErrorString(e0)));
  for (dg_mesh* M : B->members)
    if ((rc = reset_flags(M)) || (rc = ensure_udf(M))) return restore(rc);
  // The captured step assumes warm-started solves with a fixed step size: run one step
  // eagerly when any member is cold or the step sizes changed.
  // The graph holds every member's kernel arguments by value (nu among them): it is
  // replayed only if no step size and no member's arguments changed since the capture.
  bool same_dt = B->exec && B->graph_dt.size() == n && B->graph_gen.size() == n;
  for (size_t i = 0; same_dt && i < n; ++i)
    same_dt = B->graph_dt[i] == dt[i] && B->graph_gen[i] == B->members[i]->gen;
  // A member is in steady mode when its solves are warm and every stage has a full
  // multiplier history taken with the current step size; the captured step
  // replays that mode, so steps run eagerly until all members reach it.
  auto steady = [&](size_t i) {
    const dg_mesh* M = B->members[i];
    if (!M->has_lam) return false;
    for (int s = 0; s < 3; ++s) {
      if (M->hist_n[s] < M->hist_len) return false;
      for (int h = 0; h < M->hist_len; ++h)
        if (M->hist_dt[s][h] != dt[i]) return false;
    }
    return true;
  };
  int64_t done = 0;
  for (;;) {
    bool all = true;
    for (size_t i = 0; i < n; ++i) all = all && steady(i);
    if ((all && same_dt) || done >= nsteps) break;
    if (all && !same_dt) break;   // capture below
    for (size_t i = 0; i < n; ++i)
      if ((rc = enqueue_step(B->members[i], dt[i]))) return restore(rc);
    ++done;
    same_dt = false;              // the graph (if any) predates these eager steps
  }
  // The autotuner: with lanes = 0, capture the step for 1, 2, 4, 8 and 16 lanes in turn, time one
  // replay of each (each a real step of the run) and keep the fastest. Member results do not
  // depend on the lanes beyond the rounding of the solver's block-wise reductions.
  if (done < nsteps && B->lanes == 0) {
    const int cands[5] = {1, 2, 4, 8, 16};
    int best = 1;
    double best_ms = -1.0;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    for (int ci = 0; ci < 5 && done < nsteps; ++ci) {
      const int L = cands[ci];
      if (L > 1 && L > int(n)) break;
      if ((rc = capture_batch_step(B, dt, L))) break;
      // one untimed replay uploads the graph, one timed replay measures it (when steps remain)
      cudaError_t e = cudaGraphLaunch(B->exec, B->stream);
      ++done;
      if (e == cudaSuccess && done < nsteps) {
        cudaEventRecord(t0, B->stream);
        e = cudaGraphLaunch(B->exec, B->stream);
        cudaEventRecord(t1, B->stream);
        ++done;
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) {
          B->tune_ms[ci] = ms;
          if (best_ms < 0.0 || ms < best_ms) {
            best_ms = ms;
            best = L;
          }
        }
      }
      if (e != cudaSuccess) {
        rc = fail(DG_ERR_CUDA, std::string("dg_batch_rk3_step (tuning): ") + cudaGetErrorString(e));
        break;
      }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc) return restore(rc);
    B->lanes = best;
    same_dt = B->exec && B->graph_lanes == best;
  }
  if (done < nsteps && (!same_dt || B->graph_lanes != B->lanes)) {
    if ((rc = capture_batch_step(B, dt, B->lanes))) return restore(rc);
  }
  for (int64_t s = done; s < nsteps; ++s) {
    cudaError_t e = cudaGraphLaunch(B->exec, B->stream);
    if (e != cudaSuccess) return restore(fail(DG_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e)));
  }
  cudaError_t e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return restore(fail(DG_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e)));
  restore(DG_OK);
  int first = DG_OK;
  for (dg_mesh* M : B->members) {
    const int r = finish(M, true);
    if (r != DG_OK && first == DG_OK) first = r;
  }
  return first;
}

int dg_set_coefficients(dg_mesh* M, const double* coef, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!coef) return fail(DG_ERR_INVALID_ARG, "NULL coef");
  const size_t n = size_t(M->dm.n_tri) * M->hm.nd;
  CK(cudaMemcpyAsync(M->dm.u, coef, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     M->stream));
  M->udf_valid = false;   // the solver's warm-start multipliers stay (as in dg_set_velocity)
  if (int rc = reset_watch(M)) return rc;
  return finish(M, false);
}

int dg_get_coefficients(dg_mesh* M, double* coef, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!coef) return fail(DG_ERR_INVALID_ARG, "NULL coef");
  const size_t n = size_t(M->dm.n_tri) * M->hm.nd;
  CK(cudaMemcpyAsync(coef, M->dm.u, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     M->stream));
  return finish(M, false);
}

int dg_set_viscosity(dg_mesh* M, double nu) {
  if (int rc = check_mesh(M)) return rc;
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(DG_ERR_INVALID_ARG, "nu must be finite and >= 0");
  M->p.nu = nu;
  M->dm.nu = nu;
  ++M->gen;
  return DG_OK;
}

}  // extern "C"

namespace {

// y = Q x: the hybrid-mixed solve of eq. (12) applied to the functional with
// coefficients x (orthonormal basis, M = I); Q is symmetric.
int apply_Q(dg_mesh* M, const double* x, double* y) {
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_PROJECT;
  a.up = x;
  a.un = x;
  int rc = DG_OK;
  if (M->dm.elem_df) {
    // the stage buffer's twin is free outside a step: it takes the double-float image of x
    const long long n = (long long)M->dm.n_tri * M->dm.nd;
    if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_to_dfl(x, M->dm.ustage_df, n, M->stream); })))
      return rc;
    a.up_df = M->dm.ustage_df;
    a.un_df = M->dm.ustage_df;
  }
  if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_stage(M->dm, a, M->stream); }))) return rc;
  if ((rc = solve(M, 0.0))) return rc;
  return launch(M, KC_ADJOINT, [&] { return dgdf::launch_recover(M->dm, y, nullptr, M->stream); });
}

// One SSP-RK3 step that also keeps the stage inputs u^n, u^(1), u^(2) in st[0..2].
int enqueue_step_keep(dg_mesh* M, double dt, double* const st[3]) {
  dgdf::DevMesh& d = M->dm;
  const size_t bytes = size_t(d.n_tri) * d.nd * sizeof(double);
  int rc = ensure_udf(M);
  if (rc) return rc;
  use_scheme(M, DG_SCHEME_SSPRK3);
  for (int s = 0; s < 3; ++s) {
    const double* up = (s == 0) ? d.u : d.ustage;
    CK(cudaMemcpyAsync(st[s], up, bytes, cudaMemcpyDeviceToDevice, M->stream));
    dgdf::StageArgs sa{};
    sa.mode = dgdf::MODE_STAGE;
    const StageCoef& k = kSchemes[DG_SCHEME_SSPRK3].st[s];
    sa.a = k.a;
    sa.b = k.b;
    sa.c = k.c * dt;
    sa.un = d.u;
    sa.up = up;
    sa.un_df = d.u_df;
    sa.up_df = (s == 0) ? d.u_df : d.ustage_df;
    if ((rc = launch(M, KC_STAGE, [&] { return dgdf::launch_stage(d, sa, M->stream); }))) return rc;
    const double warm = M->has_lam ? sa.c / M->last_c : 0.0;
    if ((rc = solve(M, warm, s, dt)) || (rc = push_history(M, s, dt))) return rc;
    double* out = (s == 2) ? d.u : d.ustage;
    float2* out_df = (s == 2) ? d.u_df : d.ustage_df;
    if ((rc = launch(M, KC_RECOVER, [&] { return dgdf::launch_recover(d, out, out_df, M->stream); }))) return rc;
    M->last_c = sa.c;
    M->has_lam = true;
  }
  return DG_OK;
}

struct DevBuffers {
  std::vector<void*> p;
  ~DevBuffers() {
    for (void* q : p) cudaFree(q);
  }
  double* get(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(double)) != cudaSuccess) return nullptr;
    p.push_back(q);
    return static_cast<double*>(q);
  }
};

}  // namespace

extern "C" {

int dg_rk3_vjp(dg_mesh* M, double dt, int64_t nsteps, int64_t checkpoint_every, const double* ubar, double* u0bar,
               double* nubar, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (M->dm.facet_kind)
    return fail(DG_ERR_UNSUPPORTED, "dg_rk3_vjp: meshes with inflow or outflow facets are not supported");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DG_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (nsteps < 1) return fail(DG_ERR_INVALID_ARG, "nsteps must be >= 1");
  if (!ubar || !u0bar) return fail(DG_ERR_INVALID_ARG, "NULL ubar or u0bar");
  if (checkpoint_every < 1 || checkpoint_every > nsteps) checkpoint_every = nsteps;
  int rc = reset_flags(M);
  if (rc) return rc;
  dgdf::DevMesh& d = M->dm;
  const size_t n = size_t(d.n_tri) * d.nd, bytes = n * sizeof(double);
  const int64_t nseg = (nsteps + checkpoint_every - 1) / checkpoint_every;
  DevBuffers buf;
  double* ck = buf.get(size_t(nseg) * n);                      // segment start states
  double* stg = buf.get(size_t(checkpoint_every) * 3 * n);     // stage inputs of one segment
  double* ub = buf.get(n);
  double* acc = buf.get(n);
  double* fb = buf.get(n);
  double* uK = buf.get(n);
  double* nu_acc = buf.get(1);
  if (!ck || !stg || !ub || !acc || !fb || !uK || !nu_acc) return fail(DG_ERR_OOM, "dg_rk3_vjp: device memory for checkpoints");
  // forward sweep, keeping the state at the start of every segment
  for (int64_t s = 0; s < nsteps; ++s) {
    if (s % checkpoint_every == 0)
      CK(cudaMemcpyAsync(ck + size_t(s / checkpoint_every) * n, d.u, bytes, cudaMemcpyDeviceToDevice, M->stream));
    if ((rc = enqueue_step(M, dt))) return rc;
  }
  CK(cudaMemcpyAsync(uK, d.u, bytes, cudaMemcpyDeviceToDevice, M->stream));
  CK(cudaMemcpyAsync(ub, ubar, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, M->stream));
  CK(cudaMemsetAsync(nu_acc, 0, sizeof(double), M->stream));
  // reverse sweep: recompute each segment's stage inputs, then walk its steps backwards
  for (int64_t g = nseg - 1; g >= 0; --g) {
    const int64_t s0 = g * checkpoint_every;
    const int64_t len = std::min<int64_t>(checkpoint_every, nsteps - s0);
    CK(cudaMemcpyAsync(d.u, ck + size_t(g) * n, bytes, cudaMemcpyDeviceToDevice, M->stream));
    M->has_lam = false;
    M->udf_valid = false;
    forget_history(M);
    for (int64_t i = 0; i < len; ++i) {
      double* const st[3] = {stg + (size_t(i) * 3 + 0) * n, stg + (size_t(i) * 3 + 1) * n, stg + (size_t(i) * 3 + 2) * n};
      if ((rc = enqueue_step_keep(M, dt, st))) return rc;
    }
    for (int64_t i = len - 1; i >= 0; --i) {
      const double* U[3] = {stg + (size_t(i) * 3 + 0) * n, stg + (size_t(i) * 3 + 1) * n, stg + (size_t(i) * 3 + 2) * n};
      // stage s: u_s = Q(a_s u^n + b_s u' + c_s L(u')), u' = U[s], c_s = b_s dt
      for (int s = 2; s >= 0; --s) {
        if ((rc = apply_Q(M, ub, fb))) return rc;                       // F-bar = Q u_s-bar
        const StageCoef& k = kSchemes[DG_SCHEME_SSPRK3].st[s];
        const double a = k.a, b = k.b, c = k.c * dt;
        if (s == 2) {
          if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_adjoint(d, U[s], fb, acc, a, 0.0, 0, 0.0, nu_acc, M->stream); })))
            return rc;                                                   // acc = a F-bar
        } else if (a != 0.0) {
          if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_adjoint(d, U[s], fb, acc, a, 0.0, 1, 0.0, nu_acc, M->stream); })))
            return rc;                                                   // acc += a F-bar
        }
        if (s > 0) {
          // u'-bar = b (F-bar + dt J_L(u')^T F-bar); nu-bar += b dt dL/dnu(u').F-bar
          if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_adjoint(d, U[s], fb, ub, b, c, 0, c, nu_acc, M->stream); })))
            return rc;
        } else {
          // u' = u^n at the first stage: add into acc, which becomes u^n-bar
          if ((rc = launch(M, KC_ADJOINT, [&] { return dgdf::launch_adjoint(d, U[s], fb, acc, b, c, 1, c, nu_acc, M->stream); })))
            return rc;
          CK(cudaMemcpyAsync(ub, acc, bytes, cudaMemcpyDeviceToDevice, M->stream));
        }
      }
    }
  }
  CK(cudaMemcpyAsync(d.u, uK, bytes, cudaMemcpyDeviceToDevice, M->stream));
  M->has_lam = false;
  M->udf_valid = false;
  forget_history(M);
  CK(cudaMemcpyAsync(u0bar, ub, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, M->stream));
  double nb = 0.0;
  CK(cudaMemcpyAsync(&nb, nu_acc, sizeof(double), cudaMemcpyDeviceToHost, M->stream));
  rc = finish(M, true);
  if (nubar) *nubar = nb;
  return rc;
}

int dg_get_pressure(dg_mesh* M, double* p_elem, double* p_facet, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!p_elem) return fail(DG_ERR_INVALID_ARG, "NULL p_elem");
  int rc = reset_flags(M);
  if (rc) return rc;
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_PRESSURE;
  a.up = M->dm.u;
  a.un = M->dm.u;
  if ((rc = ensure_udf(M))) return rc;
  a.up_df = M->dm.u_df;
  a.un_df = M->dm.u_df;
  if ((rc = launch(M, KC_PRESSURE, [&] { return dgdf::launch_stage(M->dm, a, M->stream); }))) return rc;
  if ((rc = solve(M, 0.0, -1, 0.0, true))) return rc;   // L(u) alone: u.n = 0 on inflow facets
  if (M->dm.lam_is_df) {   // the pressure kernels read the multipliers in FP64
    if ((rc = launch(M, KC_PRESSURE, [&] {
           return dgdf::launch_to_double(M->dm.lam_df, M->dm.lat_vs, M->dm.lam, M->dm.nl, M->dm.n_facet, M->stream);
         })))
      return rc;
  }
  if ((rc = launch(M, KC_PRESSURE, [&] { return dgdf::launch_pressure(M->dm, M->wbuf, M->stream); }))) return rc;
  if ((rc = launch(M, KC_PRESSURE, [&] {
         return dgdf::launch_pressure_lattice(M->dm, M->wbuf, M->pe, p_facet ? M->pfac : nullptr, M->stream);
       })))
    return rc;
  M->has_lam = false;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(p_elem, M->pe, size_t(M->dm.n_tri) * M->hm.nw * sizeof(double), kind, M->stream));
  if (p_facet)
    CK(cudaMemcpyAsync(p_facet, M->pfac, size_t(M->dm.n_facet) * M->hm.nl * sizeof(double), kind, M->stream));
  return finish(M, true);
}

int dg_eval_residual(dg_mesh* M, double* vals, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!vals) return fail(DG_ERR_INVALID_ARG, "NULL vals");
  dgdf::StageArgs a{};
  a.mode = dgdf::MODE_RESIDUAL;
  a.up = M->dm.u;
  a.un = M->dm.u;
  int rc = ensure_udf(M);
  if (rc) return rc;
  a.up_df = M->dm.u_df;
  a.un_df = M->dm.u_df;
  rc = launch(M, KC_STAGE, [&] { return dgdf::launch_stage(M->dm, a, M->stream); });
  if (rc) return rc;
  if ((rc = launch(M, KC_LATTICE, [&] { return dgdf::launch_coef_to_lattice(M->dm, M->dm.h, M->lattice, M->stream); })))
    return rc;
  const size_t n = size_t(M->dm.n_tri) * M->hm.ns * 2;
  CK(cudaMemcpyAsync(vals, M->lattice, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     M->stream));
  return finish(M, false);
}

int dg_get_diagnostics(dg_mesh* M, double out[8]) {
  if (int rc = check_mesh(M)) return rc;
  if (!out) return fail(DG_ERR_INVALID_ARG, "NULL out");
  int rc = launch(M, KC_DIAG, [&] { return dgdf::launch_diagnostics(M->dm, M->dm.u, M->stream); });
  if (rc) return rc;
  double d4[4];
  CK(cudaMemcpyAsync(d4, M->dm.diag, 4 * sizeof(double), cudaMemcpyDeviceToHost, M->stream));
  CK(cudaMemcpyAsync(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost, M->stream));
  if ((rc = finish(M, false))) return rc;
  for (int i = 0; i < 4; ++i) out[i] = d4[i];
  out[4] = M->host_stats->last_iters;
  out[5] = double(M->host_stats->total_iters);
  out[6] = double(M->host_stats->solves);
  out[7] = M->host_stats->last_relres;
  return DG_OK;
}

int dg_get_solver_stats(dg_mesh* M, double out[8]) {
  if (int rc = check_mesh(M)) return rc;
  if (!out) return fail(DG_ERR_INVALID_ARG, "NULL out");
  CK(cudaMemcpyAsync(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost, M->stream));
  if (int rc = finish(M, false)) return rc;
  const dgdf::DevStats& s = *M->host_stats;
  out[0] = s.last_iters;
  out[1] = double(s.total_iters);
  out[2] = double(s.solves);
  out[3] = s.last_relres;
  out[4] = s.last_sweeps;
  out[5] = double(s.total_sweeps);
  out[6] = M->use_lattice ? 1.0 : (M->use_ml ? 2.0 : 0.0);
  out[7] = M->use_lattice ? M->lattice_blocks
                          : (M->use_ml ? M->ml_blocks : M->solver_blocks[M->p.precision == DG_PRECISION_MIXED]);
  return DG_OK;
}

int dg_facet_solve_noalloc(int k, int64_t n_facet, const int32_t* facet_nbr, const int32_t* stencil,
                           const double* blocks, const double* binv, const double* g, double* lam, double rtol,
                           int maxit, void* cuda_stream, int* iterations, double* relres) {
  g_err.clear();
  if (k < 1 || k > dgdf::kMaxDegree) return fail(DG_ERR_UNSUPPORTED, "k must be 1..3");
  if (!facet_nbr || !stencil || !blocks || !binv || !g || !lam) return fail(DG_ERR_INVALID_ARG, "NULL argument");
  if (n_facet < 1) return fail(DG_ERR_INVALID_ARG, "n_facet must be >= 1");
  const long long dofs = (long long)n_facet * (k + 1);
  if (dofs > dgdf::noalloc_max_dofs())
    return fail(DG_ERR_INVALID_ARG, "dg_facet_solve_noalloc: n_facet*(k+1) = " + std::to_string(dofs) +
                                        " exceeds the static scratch limit of " +
                                        std::to_string(dgdf::noalloc_max_dofs()) + " multiplier DOFs");
  if (!(rtol > 0.0) || maxit < 1) return fail(DG_ERR_INVALID_ARG, "need rtol > 0 and maxit >= 1");
  dgdf::DevStats st{};
  cudaError_t e = dgdf::solve_noalloc(k, int(n_facet), facet_nbr, stencil, blocks, binv, g, lam, rtol, maxit,
                                      static_cast<cudaStream_t>(cuda_stream), &st);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, std::string("dg_facet_solve_noalloc: ") + cudaGetErrorString(e));
  if (iterations) *iterations = st.last_iters;
  if (relres) *relres = st.last_relres;
  if (st.flags & dgdf::kFlagBarrierTimeout) return fail(DG_ERR_CUDA, "solver grid barrier timed out");
  if (st.flags & dgdf::kFlagNonFinite) return fail(DG_ERR_NONFINITE, "non-finite residual in the facet solve");
  if (st.flags & dgdf::kFlagNotConverged) return fail(DG_ERR_NOT_CONVERGED, "facet solve reached maxit");
  return DG_OK;
}

int dg_set_inflow(dg_mesh* M, const double* vals) {
  if (int rc = check_mesh(M)) return rc;
  if (!vals) return fail(DG_ERR_INVALID_ARG, "NULL vals");
  if (!M->hm.has_inflow) return fail(DG_ERR_INVALID_ARG, "dg_set_inflow: the mesh has no inflow facets");
  const size_t nv = size_t(M->dm.n_tri) * 3 * (M->hm.k + 1) * 2;
  for (size_t i = 0; i < nv; ++i)
    if (!std::isfinite(vals[i])) return fail(DG_ERR_INVALID_ARG, "dg_set_inflow: values must be finite");
  std::vector<double> uq, dm;
  dgdf::inflow_data(M->hm, vals, uq, dm);
  CK(cudaMemcpyAsync(const_cast<double*>(M->dm.inflow_q), uq.data(), uq.size() * sizeof(double),
                     cudaMemcpyHostToDevice, M->stream));
  CK(cudaMemcpyAsync(const_cast<double*>(M->dm.inflow_d), dm.data(), dm.size() * sizeof(double),
                     cudaMemcpyHostToDevice, M->stream));
  CK(cudaStreamSynchronize(M->stream));
  return DG_OK;
}

int dg_set_tensor_cores(dg_mesh* M, int enable) {
  if (int rc = check_mesh(M)) return rc;
  if (enable != 0 && enable != 1) return fail(DG_ERR_INVALID_ARG, "enable must be 0 or 1");
  if (enable && !M->tc_available)
    return fail(DG_ERR_UNSUPPORTED, "the tensor-core recovery needs the mixed form and at most two geometry classes");
  M->dm.tc_rec = enable;
  ++M->gen;
  return DG_OK;
}

int dg_set_energy_watchdog(dg_mesh* M, double rel_tol) {
  if (int rc = check_mesh(M)) return rc;
  if (!(rel_tol >= 0.0) || !std::isfinite(rel_tol)) return fail(DG_ERR_INVALID_ARG, "rel_tol must be finite and >= 0");
  if (rel_tol > 0.0 && !M->watch) {
    if (int rc = dalloc(M, &M->watch, size_t(2 + dgdf::kMaxSolverBlocks))) return rc;
  }
  M->watch_tol = rel_tol;
  if (int rc = reset_watch(M)) return rc;
  return finish(M, false);
}

int dg_test_multilevel_apply(dg_mesh* M, const double* r, double* z, int on_device) {
  if (int rc = check_mesh(M)) return rc;
  if (!r || !z) return fail(DG_ERR_INVALID_ARG, "NULL r or z");
  if (!M->use_ml) return fail(DG_ERR_UNSUPPORTED, "the mesh does not use the multilevel preconditioner");
  const size_t n = size_t(M->dm.n_facet) * M->dm.nl;
  double *rd = nullptr, *zd = nullptr;
  if (!on_device) {
    if (int rc = dalloc(M, &rd, n)) return rc;
    if (int rc = dalloc(M, &zd, n)) return rc;
    CK(cudaMemcpyAsync(rd, r, n * sizeof(double), cudaMemcpyHostToDevice, M->stream));
  }
  if (int rc = reset_flags(M)) return rc;
  int rc = launch(M, KC_SOLVE_ML, [&] {
    return dgdf::launch_ml_apply(M->dm, on_device ? r : rd, on_device ? z : zd, M->ml_blocks, M->stream);
  });
  if (rc) return rc;
  if (!on_device) CK(cudaMemcpyAsync(z, zd, n * sizeof(double), cudaMemcpyDeviceToHost, M->stream));
  return finish(M, true);
}

int dg_solver_history(dg_mesh* M, int enable, double* out, int cap, int* n_out) {
  if (int rc = check_mesh(M)) return rc;
  if (!M->use_ml) return fail(DG_ERR_UNSUPPORTED, "the history is recorded by the multilevel solver only");
  if (enable == 1 && !M->dm.ml_hist) {
    if (int rc = dalloc(M, &M->dm.ml_hist, size_t(4) * dgdf::kMLHist)) return rc;
  } else if (enable == 0) {
    M->dm.ml_hist = nullptr;
  }
  if (out && M->dm.ml_hist) {
    if (int rc = finish(M, false)) return rc;
    const int n = std::min(std::max(cap, 0), 4 * dgdf::kMLHist);
    CK(cudaMemcpy(out, M->dm.ml_hist, size_t(n) * sizeof(double), cudaMemcpyDeviceToHost));
  }
  if (n_out) {
    CK(cudaMemcpy(M->host_stats, M->dm.stats, sizeof(dgdf::DevStats), cudaMemcpyDeviceToHost));
    *n_out = M->host_stats->last_iters;
  }
  return DG_OK;
}

int dg_test_barrier_fault(dg_mesh* M, int64_t spin_limit, int skip_block) {
  if (int rc = check_mesh(M)) return rc;
  if (spin_limit < 0) return fail(DG_ERR_INVALID_ARG, "spin_limit must be >= 0");
  if (skip_block < -1) return fail(DG_ERR_INVALID_ARG, "skip_block must be >= -1");
  const unsigned long long lim = (unsigned long long)spin_limit;
  const int skip = skip_block + 1;
  CK(cudaMemcpyAsync(&M->dm.stats->spin_limit, &lim, sizeof(lim), cudaMemcpyHostToDevice, M->stream));
  CK(cudaMemcpyAsync(&M->dm.stats->skip_block, &skip, sizeof(skip), cudaMemcpyHostToDevice, M->stream));
  return finish(M, false);
}

int dg_profile(dg_mesh* M, int enable, double* out_ms, int64_t* out_launches, int n) {
  if (int rc = check_mesh(M)) return rc;
  CK(cudaStreamSynchronize(M->stream));
  collect_profile(M);
  if (enable == 2) {
    for (int i = 0; i < KC_COUNT; ++i) {
      M->prof_ms[i] = 0.0;
      M->prof_n[i] = 0;
    }
  } else if (enable == 0 || enable == 1) {
    M->prof = enable == 1;
  } else {
    return fail(DG_ERR_INVALID_ARG, "enable must be 0, 1 or 2");
  }
  for (int i = 0; i < n && i < KC_COUNT; ++i) {
    if (out_ms) out_ms[i] = M->prof_ms[i];
    if (out_launches) out_launches[i] = M->prof_n[i];
  }
  return DG_OK;
}

}  // extern "C"
