// Host-only introspection entry points (include/dgdf_host.h): the set-up of
// setup.cpp without any device, for checks on machines without a GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/dgdf.h"
#include "../../include/dgdf_host.h"
#include "multilevel.hpp"
#include "setup.hpp"
#include "setup3.hpp"

extern "C" {

int dg_host_topology(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int64_t* n_facet,
                     int32_t* tri_facet, int8_t* tri_orient, int32_t* facet_tri) {
  if (!n_facet) return DG_ERR_INVALID_ARG;
  dgdf::Topology topo;
  std::string err;
  int rc = dgdf::build_topology(n_tri, tri_vertex_ids, tri_coords, topo, err);
  if (rc) return rc;
  *n_facet = topo.n_facet;
  if (tri_facet) std::memcpy(tri_facet, topo.tri_facet.data(), topo.tri_facet.size() * sizeof(int32_t));
  if (tri_orient) std::memcpy(tri_orient, topo.tri_orient.data(), topo.tri_orient.size() * sizeof(int8_t));
  if (facet_tri) std::memcpy(facet_tri, topo.facet_tri.data(), topo.facet_tri.size() * sizeof(int32_t));
  return DG_OK;
}

int dg_host_reference(int k, int table, double* out, int64_t cap, int64_t* n_out) {
  if (!n_out) return DG_ERR_INVALID_ARG;
  dgdf::RefTables ref;
  std::string err;
  int rc = dgdf::build_reference(k, ref, err);
  if (rc) return rc;
  std::vector<double> v;
  switch (table) {
    case 0:
      for (int q = 0; q < ref.nq; ++q) {
        v.push_back(ref.vxi[2 * q]);
        v.push_back(ref.vxi[2 * q + 1]);
        v.push_back(ref.vw[q]);
      }
      break;
    case 1:
      for (int q = 0; q < ref.nqf; ++q) {
        v.push_back(ref.ft[q]);
        v.push_back(ref.fw[q]);
      }
      break;
    case 2: v = ref.vphi; break;
    case 3: v = ref.vdphi; break;
    case 4: v = ref.lat_phi; break;
    default: return DG_ERR_INVALID_ARG;
  }
  *n_out = int64_t(v.size());
  if (out) {
    if (cap < int64_t(v.size())) return DG_ERR_INVALID_ARG;
    std::memcpy(out, v.data(), v.size() * sizeof(double));
  }
  return DG_OK;
}

int dg_host_facet_operator(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k,
                           double alpha, int64_t* n_facet, int64_t* n_stencil, int32_t* facet_nbr, int32_t* stencil,
                           double* blocks, double* binv, int64_t cap_blocks) {
  if (!n_facet || !n_stencil || !(alpha > 0.0)) return DG_ERR_INVALID_ARG;
  dgdf::HostMesh hm;
  std::string err;
  int rc = dgdf::build_host_mesh(n_tri, tri_vertex_ids, tri_coords, k, alpha, hm, err);
  if (rc) return rc;
  *n_facet = hm.topo.n_facet;
  *n_stencil = hm.n_stencil;
  if ((blocks || binv) && cap_blocks < hm.n_stencil) return DG_ERR_INVALID_ARG;
  if (facet_nbr) std::memcpy(facet_nbr, hm.facet_nbr.data(), hm.facet_nbr.size() * sizeof(int32_t));
  if (stencil) std::memcpy(stencil, hm.facet_stencil.data(), hm.facet_stencil.size() * sizeof(int32_t));
  if (blocks) std::memcpy(blocks, hm.stencil_blocks.data(), hm.stencil_blocks.size() * sizeof(double));
  if (binv) std::memcpy(binv, hm.stencil_binv.data(), hm.stencil_binv.size() * sizeof(double));
  return DG_OK;
}

int dg_host_lattice(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k, double alpha,
                    int64_t* N, int32_t* facet_of, double* sinv, int64_t cap) {
  if (!N || !(alpha > 0.0)) return DG_ERR_INVALID_ARG;
  dgdf::HostMesh hm;
  std::string err;
  int rc = dgdf::build_host_mesh(n_tri, tri_vertex_ids, tri_coords, k, alpha, hm, err);
  if (rc) return rc;
  dgdf::Lattice lat;
  dgdf::build_lattice(hm, tri_coords, lat);
  if (!lat.ok) return DG_ERR_UNSUPPORTED;
  *N = lat.N;
  if (facet_of) std::memcpy(facet_of, lat.facet_of.data(), lat.facet_of.size() * sizeof(int32_t));
  if (sinv) {
    if (cap < int64_t(lat.sinv.size())) return DG_ERR_INVALID_ARG;
    std::memcpy(sinv, lat.sinv.data(), lat.sinv.size() * sizeof(double));
  }
  return DG_OK;
}

int dg_host_multilevel(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k, double alpha,
                       int64_t info[34], int nr, const double* r, double* z, const double* g, double* lam, double rtol,
                       int64_t* iters) {
  if (!info || !(alpha > 0.0) || nr < 0 || (nr > 0 && (!r || !z))) return DG_ERR_INVALID_ARG;
  dgdf::HostMesh hm;
  std::string err;
  int rc = dgdf::build_host_mesh(n_tri, tri_vertex_ids, tri_coords, k, alpha, hm, err);
  if (rc) return rc;
  dgdf::MLHost ml;
  if ((rc = dgdf::build_multilevel(hm, ml, err))) return rc;
  for (int i = 0; i < 34; ++i) info[i] = 0;
  info[0] = int64_t(ml.lv.size());
  info[1] = ml.nc;
  for (size_t l = 0; l < ml.lv.size() && l < 16; ++l) {
    info[2 + 2 * l] = ml.lv[l].n;
    info[3 + 2 * l] = ml.lv[l].bs;
  }
  const size_t n = size_t(hm.topo.n_facet) * hm.nl;
  for (int i = 0; i < nr; ++i) dgdf::multilevel_apply_host(hm, ml, r + i * n, z + i * n);
  if (g && lam) {
    // PCG from zero, the constant multiplier left out of g and of the residual norm
    const int nl = hm.nl;
    const size_t nf = size_t(hm.topo.n_facet);
    std::vector<double> b(g, g + n), rr(n), zz(n), p(n), q(n);
    double c0 = 0.0;
    for (size_t f = 0; f < nf; ++f) c0 += b[f * nl];
    c0 /= double(nf);
    for (size_t f = 0; f < nf; ++f) b[f * nl] -= c0;
    auto norm_r = [&](const std::vector<double>& v) {
      double s = 0.0, m = 0.0;
      for (size_t i = 0; i < n; ++i) s += v[i] * v[i];
      for (size_t f = 0; f < nf; ++f) m += v[f * nl];
      return std::sqrt(std::max(s - m * m / double(nf), 0.0));
    };
    auto applyS = [&](const double* x, double* y) {
      for (size_t f = 0; f < nf; ++f) {
        const double* blk = &hm.stencil_blocks[size_t(hm.facet_stencil[f]) * 5 * nl * nl];
        size_t nb[5] = {f, size_t(hm.facet_nbr[f * 4]), size_t(hm.facet_nbr[f * 4 + 1]), size_t(hm.facet_nbr[f * 4 + 2]),
                        size_t(hm.facet_nbr[f * 4 + 3])};
        for (int i = 0; i < nl; ++i) {
          double v = 0.0;
          for (int bb = 0; bb < 5; ++bb)
            for (int j = 0; j < nl; ++j) v += blk[(size_t(bb) * nl + i) * nl + j] * x[nb[bb] * nl + j];
          y[f * nl + i] = v;
        }
      }
    };
    for (size_t i = 0; i < n; ++i) lam[i] = 0.0;
    rr = b;
    const double stop = rtol * norm_r(b);
    dgdf::multilevel_apply_host(hm, ml, rr.data(), zz.data());
    p = zz;
    double rz = 0.0;
    for (size_t i = 0; i < n; ++i) rz += rr[i] * zz[i];
    int64_t it = 0;
    for (; it < 10000 && norm_r(rr) > stop; ++it) {
      applyS(p.data(), q.data());
      double pq = 0.0;
      for (size_t i = 0; i < n; ++i) pq += p[i] * q[i];
      const double a = rz / pq;
      for (size_t i = 0; i < n; ++i) {
        lam[i] += a * p[i];
        rr[i] -= a * q[i];
      }
      dgdf::multilevel_apply_host(hm, ml, rr.data(), zz.data());
      double rz2 = 0.0;
      for (size_t i = 0; i < n; ++i) rz2 += rr[i] * zz[i];
      for (size_t i = 0; i < n; ++i) p[i] = zz[i] + rz2 / rz * p[i];
      rz = rz2;
    }
    if (iters) *iters = it;
  }
  return DG_OK;
}

int dg3_host_faces(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords, int64_t* n_face_out,
                   int64_t* face_tet, int8_t* face_loc, int64_t* face_vid) {
  if (!tet_vertex_ids || !tet_coords) return DG_ERR_INVALID_ARG;
  dgdf::HostMesh3 hm;
  std::string err;
  int rc = dgdf::build_host_mesh3(n_tet, tet_vertex_ids, tet_coords, 1, 2.0, hm, err);
  if (rc) return rc;
  if (n_face_out) *n_face_out = hm.n_face;
  for (int64_t f = 0; f < hm.n_face; ++f) {
    for (int s = 0; s < 2; ++s) {
      if (face_tet) face_tet[f * 2 + s] = hm.face_tet[size_t(f) * 2 + s];
      if (face_loc) face_loc[f * 2 + s] = hm.face_loc[size_t(f) * 2 + s];
    }
    if (face_vid) {
      // the three vertices of the first side's local face (all but its vertex e), sorted by id
      const int64_t t = hm.face_tet[size_t(f) * 2];
      const int e = hm.face_loc[size_t(f) * 2];
      int64_t id[3];
      int n = 0;
      for (int v = 0; v < 4; ++v)
        if (v != e) id[n++] = tet_vertex_ids[t * 4 + v];
      std::sort(id, id + 3);
      for (int c = 0; c < 3; ++c) face_vid[f * 3 + c] = id[c];
    }
  }
  return DG_OK;
}

int dg3_host_project(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords, int k, double alpha,
                     const double* vals, double* out, int64_t* iters) {
  if (!vals || !out || !(alpha > 0.0)) return DG_ERR_INVALID_ARG;
  dgdf::HostMesh3 hm;
  std::string err;
  int rc = dgdf::build_host_mesh3(n_tet, tet_vertex_ids, tet_coords, k, alpha, hm, err);
  if (rc) return rc;
  const int ns = hm.ns, nd = hm.nd, nl = hm.nl, L4 = 4 * nl;
  const size_t nT = size_t(hm.n_tet), nF = size_t(hm.n_face), n = nF * nl;
  // coefficients of the interpolant (M = I in the orthonormal basis), then g = sum of G f
  std::vector<double> f(nT * nd), g(n, 0.0);
  for (size_t t = 0; t < nT; ++t) {
    const dgdf::Class3& co = hm.classes[hm.tet_class[t]];
    const double sq = std::sqrt(co.det);
    for (int c = 0; c < 3; ++c)
      for (int j = 0; j < ns; ++j) {
        double v = 0.0;
        for (int p = 0; p < ns; ++p) v += hm.ref.lat_inv[size_t(j) * ns + p] * vals[(t * ns + p) * 3 + c];
        f[t * nd + c * ns + j] = sq * v;
      }
    for (int e = 0; e < 4; ++e) {
      const size_t fc = size_t(hm.tet_face[t * 4 + e]);
      for (int m = 0; m < nl; ++m) {
        double v = 0.0;
        for (int j = 0; j < nd; ++j) v += co.G[size_t(e * nl + m) * nd + j] * f[t * nd + j];
        g[fc * nl + m] += v;
      }
    }
  }
  // S lam = g by PCG with one host V-cycle of the assembled hierarchy (point-Jacobi smoothing on
  // every level), the constant multiplier left out of g and of the residual
  dgdf::CsrHost A = dgdf::stencil_csr(int(nF), nl, 6, hm.face_stencil.data(), hm.face_nbr.data(),
                                      hm.stencil_blocks.data());
  dgdf::MLHost ml;
  if ((rc = dgdf::build_multilevel_csr(A, nl, nullptr, nullptr, ml, err))) return rc;
  auto centre = [&](std::vector<double>& v) {
    double c0 = 0.0;
    for (size_t fc = 0; fc < nF; ++fc) c0 += v[fc * nl];
    c0 /= double(nF);
    for (size_t fc = 0; fc < nF; ++fc) v[fc * nl] -= c0;
  };
  auto apply = [&](const std::vector<double>& x, std::vector<double>& y) {
    for (size_t i = 0; i < n; ++i) {
      double v = 0.0;
      for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) v += A.v[p] * x[A.ci[p]];
      y[i] = v;
    }
  };
  auto dot = [&](const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
  };
  const dgdf::HostMesh none;
  centre(g);
  std::vector<double> lam(n, 0.0), r(g), z(n), p(n), q(n);
  const double gn = std::sqrt(dot(g, g));
  int64_t it = 0;
  if (gn > 0.0) {
    dgdf::multilevel_apply_host(none, ml, r.data(), z.data());
    p = z;
    double rho = dot(r, z);
    for (; it < 2000 && std::sqrt(dot(r, r)) > 1e-13 * gn; ++it) {
      apply(p, q);
      const double al = rho / dot(p, q);
      for (size_t i = 0; i < n; ++i) {
        lam[i] += al * p[i];
        r[i] -= al * q[i];
      }
      centre(r);
      dgdf::multilevel_apply_host(none, ml, r.data(), z.data());
      const double rn = dot(r, z), be = rn / rho;
      rho = rn;
      for (size_t i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
    }
  }
  if (iters) *iters = it;
  // u = P f - G^T lam, as lattice values
  for (size_t t = 0; t < nT; ++t) {
    const dgdf::Class3& co = hm.classes[hm.tet_class[t]];
    std::vector<double> u(nd), lt(L4);
    for (int e = 0; e < 4; ++e)
      for (int m = 0; m < nl; ++m) lt[e * nl + m] = lam[size_t(hm.tet_face[t * 4 + e]) * nl + m];
    for (int i = 0; i < nd; ++i) {
      double v = 0.0;
      for (int j = 0; j < nd; ++j) v += co.P[size_t(i) * nd + j] * f[t * nd + j];
      for (int l = 0; l < L4; ++l) v -= co.G[size_t(l) * nd + i] * lt[l];
      u[i] = v;
    }
    const double s = 1.0 / std::sqrt(co.det);
    for (int pt = 0; pt < ns; ++pt)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int j = 0; j < ns; ++j) v += hm.ref.lat_phi[size_t(pt) * ns + j] * u[c * ns + j];
        out[(t * ns + pt) * 3 + c] = s * v;
      }
  }
  return DG_OK;
}

}  // extern "C"
