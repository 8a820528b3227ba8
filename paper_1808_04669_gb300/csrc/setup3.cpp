// Host-side FP64 set-up of the three-dimensional path (see setup3.hpp).
#include "setup3.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "../../include/dgdf.h"
#include "setup.hpp"

namespace dgdf {
namespace {

// the six orderings of a face's three local vertices (the perm index)
constexpr int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
constexpr double kRefV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// ascending local vertices of local face e
void face_verts(int e, int out[3]) {
  int n = 0;
  for (int v = 0; v < 4; ++v)
    if (v != e) out[n++] = v;
}

// Gauss rules mapped to [0, 1]: weight 1 (a = 0) or (1 - x)^a
void rule01(int n, double a, std::vector<double>& x, std::vector<double>& w) {
  host_gauss_jacobi(n, a, 0.0, x, w);
  const double scale = std::pow(0.5, a + 1.0);
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (x[i] + 1.0);
    w[i] *= scale;
  }
}

// Collapsed rule on the reference tetrahedron, n points per direction (exact to degree 2n - 1).
void tet_rule(int n, std::vector<double>& xi, std::vector<double>& w) {
  std::vector<double> a, wa, b, wb, c, wc;
  rule01(n, 0.0, a, wa);
  rule01(n, 1.0, b, wb);
  rule01(n, 2.0, c, wc);
  xi.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < n; ++l) {
        xi.push_back(a[i] * (1.0 - b[j]) * (1.0 - c[l]));
        xi.push_back(b[j] * (1.0 - c[l]));
        xi.push_back(c[l]);
        w.push_back(wa[i] * wb[j] * wc[l]);
      }
}

// Monomial exponents of total degree <= k on the tetrahedron, ordered by degree.
std::vector<std::array<int, 3>> monomials3(int k) {
  std::vector<std::array<int, 3>> m;
  for (int d = 0; d <= k; ++d)
    for (int c = 0; c <= d; ++c)
      for (int b = 0; b <= d - c; ++b) m.push_back({d - b - c, b, c});
  return m;
}

struct Basis3 {
  std::vector<std::array<int, 3>> mono;
  std::vector<double> B;   // [ns][ns]: function j = sum_m B[j][m] mono_m
  int ns = 0;
  void eval(const double* x, double* v, double* g) const {
    std::vector<double> mv(ns), mg(size_t(ns) * 3);
    for (int m = 0; m < ns; ++m) {
      const auto& e = mono[m];
      auto pw = [&](double y, int p) { return p == 0 ? 1.0 : std::pow(y, p); };
      mv[m] = pw(x[0], e[0]) * pw(x[1], e[1]) * pw(x[2], e[2]);
      for (int d = 0; d < 3; ++d) {
        if (e[d] == 0) {
          mg[m * 3 + d] = 0.0;
          continue;
        }
        double t = e[d] * pw(x[d], e[d] - 1);
        for (int o = 0; o < 3; ++o)
          if (o != d) t *= pw(x[o], e[o]);
        mg[m * 3 + d] = t;
      }
    }
    for (int j = 0; j < ns; ++j) {
      double s = 0, g0 = 0, g1 = 0, g2 = 0;
      for (int m = 0; m < ns; ++m) {
        const double c = B[size_t(j) * ns + m];
        s += c * mv[m];
        g0 += c * mg[m * 3];
        g1 += c * mg[m * 3 + 1];
        g2 += c * mg[m * 3 + 2];
      }
      v[j] = s;
      if (g) {
        g[j * 3] = g0;
        g[j * 3 + 1] = g1;
        g[j * 3 + 2] = g2;
      }
    }
  }
};

// Gram-Schmidt (modified, twice) of the columns of V [nq][n] in the inner product sum_q w_q;
// returns the coefficient matrix B [n][n] of the orthonormal functions in the original ones.
std::vector<double> gram_schmidt(const std::vector<double>& V, const std::vector<double>& w, int nq, int n) {
  std::vector<double> B(size_t(n) * n, 0.0), F(V);   // F: current function values [nq][n]
  for (int j = 0; j < n; ++j) B[size_t(j) * n + j] = 1.0;
  auto dot = [&](int a, int b) {
    double s = 0;
    for (int q = 0; q < nq; ++q) s += w[q] * F[size_t(q) * n + a] * F[size_t(q) * n + b];
    return s;
  };
  for (int j = 0; j < n; ++j) {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < j; ++i) {
        const double c = dot(i, j);
        for (int q = 0; q < nq; ++q) F[size_t(q) * n + j] -= c * F[size_t(q) * n + i];
        for (int m = 0; m < n; ++m) B[size_t(j) * n + m] -= c * B[size_t(i) * n + m];
      }
    const double nrm = std::sqrt(dot(j, j));
    for (int q = 0; q < nq; ++q) F[size_t(q) * n + j] /= nrm;
    for (int m = 0; m < n; ++m) B[size_t(j) * n + m] /= nrm;
  }
  return B;
}

int build_ref3(int k, Ref3& r, std::string& err) {
  r.k = k;
  r.ns = n_lat3(k);
  r.nw = n_lat3(k - 1);
  r.nl = (k + 1) * (k + 2) / 2;
  const int ns = r.ns;
  // orthonormal basis of P^k on the reference tetrahedron (exact rule of degree 2k + 1)
  Basis3 B;
  B.mono = monomials3(k);
  B.ns = ns;
  {
    std::vector<double> xi, w;
    tet_rule(k + 1, xi, w);
    const int nq = int(w.size());
    std::vector<double> V(size_t(nq) * ns);
    B.B.assign(size_t(ns) * ns, 0.0);
    for (int j = 0; j < ns; ++j) B.B[size_t(j) * ns + j] = 1.0;
    for (int q = 0; q < nq; ++q) B.eval(&xi[q * 3], &V[size_t(q) * ns], nullptr);
    B.B = gram_schmidt(V, w, nq, ns);
  }
  // volume rule of degree 3k - 1
  tet_rule((3 * k + 1) / 2, r.vxi, r.vw);
  r.nq = int(r.vw.size());
  r.vphi.resize(size_t(r.nq) * ns);
  r.vdphi.resize(size_t(r.nq) * ns * 3);
  for (int q = 0; q < r.nq; ++q) B.eval(&r.vxi[q * 3], &r.vphi[size_t(q) * ns], &r.vdphi[size_t(q) * ns * 3]);
  // face rule (shared convention, setup3.hpp)
  {
    const int q1 = (3 * k + 2) / 2;
    std::vector<double> a, wa, b, wb;
    rule01(q1, 0.0, a, wa);
    rule01(q1, 1.0, b, wb);
    r.fst.clear();
    r.fw.clear();
    for (int i = 0; i < q1; ++i)
      for (int j = 0; j < q1; ++j) {
        r.fst.push_back(a[i] * (1.0 - b[j]));
        r.fst.push_back(b[j]);
        r.fw.push_back(wa[i] * wb[j]);
      }
    r.nqf = int(r.fw.size());
  }
  r.fphi.resize(size_t(4) * 6 * r.nqf * ns);
  r.fdphi.resize(size_t(4) * 6 * r.nqf * ns * 3);
  for (int e = 0; e < 4; ++e) {
    int fv[3];
    face_verts(e, fv);
    for (int p = 0; p < 6; ++p) {
      const double* P0 = kRefV[fv[kPerm3[p][0]]];
      const double* P1 = kRefV[fv[kPerm3[p][1]]];
      const double* P2 = kRefV[fv[kPerm3[p][2]]];
      for (int q = 0; q < r.nqf; ++q) {
        const double s = r.fst[q * 2], t = r.fst[q * 2 + 1];
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = P0[d] + s * (P1[d] - P0[d]) + t * (P2[d] - P0[d]);
        const size_t o = (size_t(e * 6 + p) * r.nqf + q) * ns;
        B.eval(x, &r.fphi[o], &r.fdphi[o * 3]);
      }
    }
  }
  // multiplier basis: monomials s^a t^b (a + b <= k) orthonormalised with the face rule (exact to 3k)
  {
    const int nl = r.nl, nqf = r.nqf;
    std::vector<double> V(size_t(nqf) * nl);
    for (int q = 0; q < nqf; ++q) {
      int m = 0;
      for (int d = 0; d <= k; ++d)
        for (int bb = 0; bb <= d; ++bb, ++m)
          V[size_t(q) * nl + m] = std::pow(r.fst[q * 2], d - bb) * std::pow(r.fst[q * 2 + 1], bb);
    }
    std::vector<double> C = gram_schmidt(V, r.fw, nqf, nl);
    r.mu.assign(size_t(nqf) * nl, 0.0);
    for (int q = 0; q < nqf; ++q)
      for (int j = 0; j < nl; ++j) {
        double s = 0;
        for (int m = 0; m < nl; ++m) s += C[size_t(j) * nl + m] * V[size_t(q) * nl + m];
        r.mu[size_t(q) * nl + j] = s;
      }
    // the same basis at the face's k-lattice points
    r.mu_lat.assign(size_t(nl) * nl, 0.0);
    int p = 0;
    for (int jj = 0; jj <= k; ++jj)
      for (int ii = 0; ii <= k - jj; ++ii, ++p) {
        const double sp = double(ii) / k, tp = double(jj) / k;
        std::vector<double> mono(nl);
        int m = 0;
        for (int d = 0; d <= k; ++d)
          for (int bb = 0; bb <= d; ++bb, ++m) mono[m] = std::pow(sp, d - bb) * std::pow(tp, bb);
        for (int j = 0; j < nl; ++j) {
          double s = 0;
          for (int mm = 0; mm < nl; ++mm) s += C[size_t(j) * nl + mm] * mono[mm];
          r.mu_lat[size_t(p) * nl + j] = s;
        }
      }
  }
  // lattice (l outer, j, i inner; i/k, j/k, l/k)
  r.lat_phi.resize(size_t(ns) * ns);
  {
    int p = 0;
    for (int l = 0; l <= k; ++l)
      for (int j = 0; j <= k - l; ++j)
        for (int i = 0; i <= k - l - j; ++i, ++p) {
          const double x[3] = {double(i) / k, double(j) / k, double(l) / k};
          B.eval(x, &r.lat_phi[size_t(p) * ns], nullptr);
        }
  }
  // the first nw functions (a basis of P^(k-1)) at the (k-1)-lattice, or at the centroid
  {
    const int km = k - 1, nw = r.nw;
    r.plat_phi.assign(size_t(nw) * nw, 0.0);
    std::vector<double> all(ns);
    int p = 0;
    for (int l = 0; l <= km; ++l)
      for (int j = 0; j <= km - l; ++j)
        for (int i = 0; i <= km - l - j; ++i, ++p) {
          const double x[3] = {km ? double(i) / km : 0.25, km ? double(j) / km : 0.25, km ? double(l) / km : 0.25};
          B.eval(x, all.data(), nullptr);
          for (int m = 0; m < nw; ++m) r.plat_phi[size_t(p) * nw + m] = all[m];
        }
  }
  r.lat_inv = r.lat_phi;
  if (!host_invert(r.lat_inv, ns)) {
    err = "3-D set-up: singular lattice interpolation";
    return DG_ERR_MESH;
  }
  return DG_OK;
}

void inverse3(const double* J, double* Ji, double& det) {
  det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
}

// Element operators of one class: D, C, then P, G = C P, S = G C^T (M = I in the orthonormal basis).
void class_ops3(const Ref3& r, Class3& co) {
  const int ns = r.ns, nd = 3 * ns, nw = r.nw, nl = r.nl;
  std::vector<double> D(size_t(nw) * nd, 0.0), C(size_t(4 * nl) * nd, 0.0);
  for (int q = 0; q < r.nq; ++q)
    for (int m = 0; m < nw; ++m) {
      const double z = r.vw[q] * r.vphi[size_t(q) * ns + m];
      for (int j = 0; j < ns; ++j) {
        const double* g = &r.vdphi[(size_t(q) * ns + j) * 3];
        for (int c = 0; c < 3; ++c)
          D[size_t(m) * nd + c * ns + j] += z * (g[0] * co.Jinv[0 * 3 + c] + g[1] * co.Jinv[1 * 3 + c] +
                                                 g[2] * co.Jinv[2 * 3 + c]);
      }
    }
  const double s = 1.0 / std::sqrt(co.det);
  for (int e = 0; e < 4; ++e)
    for (int q = 0; q < r.nqf; ++q) {
      const double w = 2.0 * co.area[e] * r.fw[q] * s;
      const double* ph = &r.fphi[(size_t(e * 6 + co.perm[e]) * r.nqf + q) * ns];
      for (int m = 0; m < nl; ++m) {
        const double mu = r.mu[size_t(q) * nl + m];
        for (int j = 0; j < ns; ++j)
          for (int c = 0; c < 3; ++c) C[size_t(e * nl + m) * nd + c * ns + j] += w * mu * ph[j] * co.normal[e][c];
      }
    }
  // P = I - D^T (D D^T)^-1 D
  std::vector<double> DDt(size_t(nw) * nw, 0.0);
  for (int a = 0; a < nw; ++a)
    for (int b = 0; b < nw; ++b) {
      double v = 0;
      for (int j = 0; j < nd; ++j) v += D[size_t(a) * nd + j] * D[size_t(b) * nd + j];
      DDt[size_t(a) * nw + b] = v;
    }
  host_invert(DDt, nw);
  std::vector<double> Wm(size_t(nw) * nd, 0.0);   // (D D^T)^-1 D
  for (int a = 0; a < nw; ++a)
    for (int j = 0; j < nd; ++j) {
      double v = 0;
      for (int b = 0; b < nw; ++b) v += DDt[size_t(a) * nw + b] * D[size_t(b) * nd + j];
      Wm[size_t(a) * nd + j] = v;
    }
  co.P.assign(size_t(nd) * nd, 0.0);
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < nd; ++j) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int a = 0; a < nw; ++a) v -= D[size_t(a) * nd + i] * Wm[size_t(a) * nd + j];
      co.P[size_t(i) * nd + j] = v;
    }
  // pressure rows: u - D^T w = r and D u = 0 give w = -(D D^T)^-1 D r, r = f - C^T lam
  co.W.assign(size_t(nw) * nd, 0.0);
  for (size_t i = 0; i < co.W.size(); ++i) co.W[i] = -Wm[i];
  co.WC.assign(size_t(nw) * 4 * nl, 0.0);
  for (int a = 0; a < nw; ++a)
    for (int l = 0; l < 4 * nl; ++l) {
      double v = 0;
      for (int j = 0; j < nd; ++j) v += co.W[size_t(a) * nd + j] * C[size_t(l) * nd + j];
      co.WC[size_t(a) * 4 * nl + l] = v;
    }
  for (int i = 0; i < nd; ++i)
    for (int j = i + 1; j < nd; ++j) {
      const double a = 0.5 * (co.P[size_t(i) * nd + j] + co.P[size_t(j) * nd + i]);
      co.P[size_t(i) * nd + j] = co.P[size_t(j) * nd + i] = a;
    }
  const int L4 = 4 * nl;
  co.G.assign(size_t(L4) * nd, 0.0);
  for (int i = 0; i < L4; ++i)
    for (int j = 0; j < nd; ++j) {
      double v = 0;
      for (int m = 0; m < nd; ++m) v += C[size_t(i) * nd + m] * co.P[size_t(m) * nd + j];
      co.G[size_t(i) * nd + j] = v;
    }
  co.S.assign(size_t(L4) * L4, 0.0);
  for (int i = 0; i < L4; ++i)
    for (int j = 0; j < L4; ++j) {
      double v = 0;
      for (int m = 0; m < nd; ++m) v += co.G[size_t(i) * nd + m] * C[size_t(j) * nd + m];
      co.S[size_t(i) * L4 + j] = v;
    }
  for (int i = 0; i < L4; ++i)
    for (int j = i + 1; j < L4; ++j) {
      const double a = 0.5 * (co.S[size_t(i) * L4 + j] + co.S[size_t(j) * L4 + i]);
      co.S[size_t(i) * L4 + j] = co.S[size_t(j) * L4 + i] = a;
    }
}

}  // namespace

int build_host_mesh3(int64_t n_tet, const int64_t* vid, const double* X, int k, double alpha, HostMesh3& hm,
                     std::string& err) {
  if (n_tet < 1 || !vid || !X) {
    err = "3-D mesh: empty or NULL arrays";
    return DG_ERR_INVALID_ARG;
  }
  if (k < 1 || k > kMaxDegree3) {
    err = "3-D path: k must be 1.." + std::to_string(kMaxDegree3);
    return DG_ERR_UNSUPPORTED;
  }
  hm = HostMesh3();
  int rc = build_ref3(k, hm.ref, err);
  if (rc) return rc;
  hm.k = k;
  hm.alpha = alpha;
  hm.ns = hm.ref.ns;
  hm.nd = 3 * hm.ns;
  hm.nw = hm.ref.nw;
  hm.nl = hm.ref.nl;
  hm.n_tet = n_tet;
  double scale = 1.0;
  for (int64_t i = 0; i < n_tet * 12; ++i) scale = std::max(scale, std::fabs(X[i]) + 1.0);
  const double tol = 1e-9 * scale;
  auto rnd = [&](double v) { return (long long)std::llround(v / tol); };
  // faces: canonical order by periodic id, matched by ids and edge vectors
  using Key = std::tuple<int64_t, int64_t, int64_t, long long, long long, long long, long long, long long, long long>;
  std::map<Key, int32_t> faces;
  std::vector<std::array<int32_t, 2>> ftet;
  std::vector<std::array<int8_t, 2>> floc;
  std::vector<int> nside;
  std::vector<int> tet_perm(size_t(n_tet) * 4);
  hm.tet_face.resize(size_t(n_tet) * 4);
  hm.diam.resize(n_tet);
  // geometry classes: J rounded and the four perm indices
  std::map<std::array<long long, 13>, int32_t> cls;
  hm.tet_class.resize(n_tet);
  for (int64_t t = 0; t < n_tet; ++t) {
    const double* x = X + t * 12;
    const int64_t* id = vid + t * 4;
    double J[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) J[r * 3 + c] = x[(c + 1) * 3 + r] - x[r];
    double Ji[9], det;
    inverse3(J, Ji, det);
    if (!(det > 0.0)) {
      err = "3-D mesh: tetrahedron " + std::to_string(t) + " is not positively oriented";
      return DG_ERR_MESH;
    }
    double dm = 0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double s = 0;
        for (int d = 0; d < 3; ++d) s += (x[a * 3 + d] - x[b * 3 + d]) * (x[a * 3 + d] - x[b * 3 + d]);
        dm = std::max(dm, std::sqrt(s));
      }
    hm.diam[t] = dm;
    std::array<long long, 13> ck{};
    for (int e = 0; e < 4; ++e) {
      int fv[3];
      face_verts(e, fv);
      const int64_t a = id[fv[0]], b = id[fv[1]], c = id[fv[2]];
      if (a == b || b == c || a == c) {
        err = "3-D mesh: a face needs three distinct periodic vertex ids";
        return DG_ERR_MESH;
      }
      // ordering of the local vertices by id
      int p = 0;
      for (; p < 6; ++p) {
        const int64_t i0 = id[fv[kPerm3[p][0]]], i1 = id[fv[kPerm3[p][1]]], i2 = id[fv[kPerm3[p][2]]];
        if (i0 < i1 && i1 < i2) break;
      }
      tet_perm[size_t(t) * 4 + e] = p;
      const int v0 = fv[kPerm3[p][0]], v1 = fv[kPerm3[p][1]], v2 = fv[kPerm3[p][2]];
      Key key{id[v0], id[v1], id[v2], rnd(x[v1 * 3] - x[v0 * 3]), rnd(x[v1 * 3 + 1] - x[v0 * 3 + 1]),
              rnd(x[v1 * 3 + 2] - x[v0 * 3 + 2]), rnd(x[v2 * 3] - x[v0 * 3]), rnd(x[v2 * 3 + 1] - x[v0 * 3 + 1]),
              rnd(x[v2 * 3 + 2] - x[v0 * 3 + 2])};
      auto it = faces.find(key);
      int32_t f;
      if (it == faces.end()) {
        f = int32_t(ftet.size());
        faces.emplace(key, f);
        ftet.push_back({int32_t(t), -1});
        floc.push_back({int8_t(e), -1});
        nside.push_back(1);
      } else {
        f = it->second;
        if (nside[f] >= 2) {
          err = "3-D mesh: a face has more than two sides";
          return DG_ERR_MESH;
        }
        ftet[f][1] = int32_t(t);
        floc[f][1] = int8_t(e);
        nside[f] = 2;
      }
      hm.tet_face[size_t(t) * 4 + e] = f;
      ck[9 + e] = p;
    }
    for (int i = 0; i < 9; ++i) ck[i] = rnd(J[i]);
    auto cit = cls.find(ck);
    if (cit == cls.end()) {
      Class3 co{};
      std::copy(J, J + 9, co.J);
      std::copy(Ji, Ji + 9, co.Jinv);
      co.det = det;
      for (int e = 0; e < 4; ++e) {
        int fv[3];
        face_verts(e, fv);
        double u[3], w[3], n[3];
        for (int d = 0; d < 3; ++d) {
          u[d] = x[fv[1] * 3 + d] - x[fv[0] * 3 + d];
          w[d] = x[fv[2] * 3 + d] - x[fv[0] * 3 + d];
        }
        n[0] = u[1] * w[2] - u[2] * w[1];
        n[1] = u[2] * w[0] - u[0] * w[2];
        n[2] = u[0] * w[1] - u[1] * w[0];
        const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        double away = 0;
        for (int d = 0; d < 3; ++d) away += n[d] * (x[fv[0] * 3 + d] - x[e * 3 + d]);
        for (int d = 0; d < 3; ++d) co.normal[e][d] = (away > 0 ? 1.0 : -1.0) * n[d] / nn;
        co.area[e] = 0.5 * nn;
        co.perm[e] = tet_perm[size_t(t) * 4 + e];
      }
      class_ops3(hm.ref, co);
      const int32_t cid = int32_t(hm.classes.size());
      hm.classes.push_back(std::move(co));
      cls.emplace(ck, cid);
      hm.tet_class[t] = cid;
    } else {
      hm.tet_class[t] = cit->second;
    }
  }
  hm.n_face = int64_t(ftet.size());
  for (int64_t f = 0; f < hm.n_face; ++f)
    if (nside[f] != 2) {
      err = "3-D mesh: closed meshes only (face " + std::to_string(f) + " has one side)";
      return DG_ERR_UNSUPPORTED;
    }
  hm.face_tet.resize(size_t(hm.n_face) * 2);
  hm.face_loc.resize(size_t(hm.n_face) * 2);
  hm.tet_nbr.resize(size_t(n_tet) * 4);
  hm.tet_nbr_loc.resize(size_t(n_tet) * 4);
  hm.face_sigma.resize(hm.n_face);
  for (int64_t f = 0; f < hm.n_face; ++f) {
    for (int s = 0; s < 2; ++s) {
      hm.face_tet[f * 2 + s] = ftet[f][s];
      hm.face_loc[f * 2 + s] = floc[f][s];
    }
    const int32_t t0 = ftet[f][0], t1 = ftet[f][1];
    hm.tet_nbr[size_t(t0) * 4 + floc[f][0]] = t1;
    hm.tet_nbr_loc[size_t(t0) * 4 + floc[f][0]] = floc[f][1];
    hm.tet_nbr[size_t(t1) * 4 + floc[f][1]] = t0;
    hm.tet_nbr_loc[size_t(t1) * 4 + floc[f][1]] = floc[f][0];
    hm.face_sigma[f] = alpha * k * k / std::max(hm.diam[t0], hm.diam[t1]);
  }
  // face stencil of S: own block (both sides) and the three other faces of each side
  const int nl = hm.nl, L4 = 4 * nl;
  hm.face_nbr.resize(size_t(hm.n_face) * 6);
  hm.face_stencil.resize(hm.n_face);
  std::map<std::array<int, 4>, int32_t> st;
  for (int64_t f = 0; f < hm.n_face; ++f) {
    std::array<int, 4> key{};
    for (int s = 0; s < 2; ++s) {
      const int32_t t = ftet[f][s];
      const int e = floc[f][s];
      int n = 0;
      for (int o = 0; o < 4; ++o)
        if (o != e) hm.face_nbr[size_t(f) * 6 + s * 3 + n++] = hm.tet_face[size_t(t) * 4 + o];
      key[s * 2] = hm.tet_class[t];
      key[s * 2 + 1] = e;
    }
    auto it = st.find(key);
    if (it != st.end()) {
      hm.face_stencil[f] = it->second;
      continue;
    }
    const int32_t id = int32_t(st.size());
    st.emplace(key, id);
    hm.face_stencil[f] = id;
    std::vector<double> blk(size_t(7) * nl * nl, 0.0);
    for (int s = 0; s < 2; ++s) {
      const Class3& co = hm.classes[key[s * 2]];
      const int e = key[s * 2 + 1];
      for (int m = 0; m < nl; ++m)
        for (int mm = 0; mm < nl; ++mm) blk[size_t(m) * nl + mm] += co.S[size_t(e * nl + m) * L4 + e * nl + mm];
      int n = 0;
      for (int o = 0; o < 4; ++o) {
        if (o == e) continue;
        for (int m = 0; m < nl; ++m)
          for (int mm = 0; mm < nl; ++mm)
            blk[size_t(1 + s * 3 + n) * nl * nl + m * nl + mm] = co.S[size_t(e * nl + m) * L4 + o * nl + mm];
        ++n;
      }
    }
    std::vector<double> inv(blk.begin(), blk.begin() + nl * nl);
    if (!host_invert(inv, nl)) {
      err = "3-D set-up: singular face block";
      return DG_ERR_MESH;
    }
    hm.stencil_blocks.insert(hm.stencil_blocks.end(), blk.begin(), blk.end());
    hm.stencil_binv.insert(hm.stencil_binv.end(), inv.begin(), inv.end());
  }
  hm.n_stencil = int(st.size());
  return DG_OK;
}

}  // namespace dgdf
