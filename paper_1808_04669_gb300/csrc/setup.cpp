// Host-side FP64 set-up of libdgdf (see setup.hpp).
#include "setup.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <tuple>

#include "../../include/dgdf.h"

namespace dgdf {
namespace {

// ---------------------------------------------------------------- small dense LA
// In-place inverse of an n x n row-major matrix by Gauss-Jordan with partial pivoting.
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) I[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[size_t(r) * n + c]) > std::fabs(A[size_t(piv) * n + c])) piv = r;
    if (A[size_t(piv) * n + c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(A[size_t(c) * n + j], A[size_t(piv) * n + j]);
        std::swap(I[size_t(c) * n + j], I[size_t(piv) * n + j]);
      }
    double d = 1.0 / A[size_t(c) * n + c];
    for (int j = 0; j < n; ++j) {
      A[size_t(c) * n + j] *= d;
      I[size_t(c) * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[size_t(r) * n + j] -= f * A[size_t(c) * n + j];
        I[size_t(r) * n + j] -= f * I[size_t(c) * n + j];
      }
    }
  }
  A.swap(I);
  return true;
}

// C[m x n] = A[m x p] B[p x n]
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m, int p, int n) {
  std::vector<double> C(size_t(m) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < p; ++l) {
      double a = A[size_t(i) * p + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[size_t(i) * n + j] += a * B[size_t(l) * n + j];
    }
  return C;
}

std::vector<double> transpose(const std::vector<double>& A, int m, int n) {
  std::vector<double> T(size_t(m) * n);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) T[size_t(j) * m + i] = A[size_t(i) * n + j];
  return T;
}

// Eigen-decomposition of a small symmetric matrix by cyclic Jacobi rotations.
void sym_eig(std::vector<double> A, int n, std::vector<double>& evals, std::vector<double>& evecs) {
  evecs.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) evecs[size_t(i) * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[size_t(i) * n + j] * A[size_t(i) * n + j];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[size_t(p) * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[size_t(p) * n + p], aqq = A[size_t(q) * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[size_t(k) * n + p], akq = A[size_t(k) * n + q];
          A[size_t(k) * n + p] = c * akp - s * akq;
          A[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[size_t(p) * n + k], aqk = A[size_t(q) * n + k];
          A[size_t(p) * n + k] = c * apk - s * aqk;
          A[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = evecs[size_t(k) * n + p], vkq = evecs[size_t(k) * n + q];
          evecs[size_t(k) * n + p] = c * vkp - s * vkq;
          evecs[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  evals.resize(n);
  for (int i = 0; i < n; ++i) evals[i] = A[size_t(i) * n + i];
}

// ------------------------------------------------------------- orthogonal polys
// Jacobi polynomial P_n^{(a,b)}(x) by its three-term recurrence (Abramowitz-Stegun 22.7.1).
double jacobi(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  for (int m = 1; m < n; ++m) {
    double c = 2.0 * m + a + b;
    double a1 = 2.0 * (m + 1) * (m + a + b + 1) * c;
    double a2 = (c + 1) * (a * a - b * b);
    double a3 = c * (c + 1) * (c + 2);
    double a4 = 2.0 * (m + a) * (m + b) * (c + 2);
    double p2 = ((a2 + a3 * x) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)} (Abramowitz-Stegun 22.8.1 in derivative form).
double djacobi(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x);
}

double legendre(int n, double x) { return jacobi(n, 0.0, 0.0, x); }

// Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b on [-1,1] by Golub-Welsch.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> T(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double c = 2.0 * i + a + b;
    T[size_t(i) * n + i] = (i == 0 && std::fabs(a + b) < 1e-300) ? (b - a) / (a + b + 2.0)
                                                                  : (b * b - a * a) / (c * (c + 2.0));
    if (i + 1 < n) {
      double m = i + 1.0;
      double cm = 2.0 * m + a + b;
      double off = std::sqrt(4.0 * m * (m + a) * (m + b) * (m + a + b) / (cm * cm * (cm + 1.0) * (cm - 1.0)));
      T[size_t(i) * n + i + 1] = off;
      T[size_t(i + 1) * n + i] = off;
    }
  }
  std::vector<double> ev, V;
  sym_eig(T, n, ev, V);
  double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 2.0);
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return ev[i] < ev[j]; });
  x.resize(n);
  w.resize(n);
  for (int r = 0; r < n; ++r) {
    int i = idx[r];
    double xi = ev[i];
    // Newton polish on P_n^{(a,b)}
    for (int it = 0; it < 3; ++it) {
      double d = djacobi(n, a, b, xi);
      if (d != 0.0) xi -= jacobi(n, a, b, xi) / d;
    }
    x[r] = xi;
    w[r] = mu0 * V[size_t(0) * n + i] * V[size_t(0) * n + i];
  }
}

// Dubiner basis psi_{pq}(xi) = Q_p(xi) P_q^{(2p+1,0)}(2 xi2 - 1), where
// Q_p = (1-xi2)^p P_p((2 xi1 - 1 + xi2)/(1 - xi2)) is evaluated through the
// homogenised Legendre recurrence (no division by 1 - xi2).
struct Dubiner {
  int k, ns;
  std::vector<int> pp, qq;
  std::vector<double> norm;
  explicit Dubiner(int k_) : k(k_) {
    for (int d = 0; d <= k; ++d)
      for (int q = 0; q <= d; ++q) {
        pp.push_back(d - q);
        qq.push_back(q);
      }
    ns = int(pp.size());
    norm.assign(ns, 1.0);
  }
  // values [ns], gradients [ns][2] at one reference point
  void eval(double x1, double x2, double* v, double* g) const {
    double s = 2.0 * x1 - 1.0 + x2, t = 1.0 - x2;
    const double ds[2] = {2.0, 1.0}, dt[2] = {0.0, -1.0};
    std::vector<double> Q(k + 1), Qx(k + 1), Qy(k + 1);
    Q[0] = 1.0;
    Qx[0] = Qy[0] = 0.0;
    if (k >= 1) {
      Q[1] = s;
      Qx[1] = ds[0];
      Qy[1] = ds[1];
    }
    for (int n = 1; n < k; ++n) {
      double a = (2.0 * n + 1.0), b = double(n);
      Q[n + 1] = (a * s * Q[n] - b * t * t * Q[n - 1]) / (n + 1.0);
      Qx[n + 1] = (a * (ds[0] * Q[n] + s * Qx[n]) - b * (2.0 * t * dt[0] * Q[n - 1] + t * t * Qx[n - 1])) / (n + 1.0);
      Qy[n + 1] = (a * (ds[1] * Q[n] + s * Qy[n]) - b * (2.0 * t * dt[1] * Q[n - 1] + t * t * Qy[n - 1])) / (n + 1.0);
    }
    for (int j = 0; j < ns; ++j) {
      int p = pp[j], q = qq[j];
      double y = 2.0 * x2 - 1.0;
      double R = jacobi(q, 2.0 * p + 1.0, 0.0, y);
      double dR = 2.0 * djacobi(q, 2.0 * p + 1.0, 0.0, y);
      double c = norm[j];
      if (v) v[j] = c * Q[p] * R;
      if (g) {
        g[2 * j + 0] = c * Qx[p] * R;
        g[2 * j + 1] = c * (Qy[p] * R + Q[p] * dR);
      }
    }
  }
};

// Collapsed rule on the reference triangle: Gauss-Legendre in a, Gauss-Jacobi(1,0) in b,
// xi1 = (1+a)(1-b)/4, xi2 = (1+b)/2, d xi = (1-b)/8 da db.
void triangle_rule(int n, std::vector<double>& xi, std::vector<double>& w) {
  std::vector<double> xa, wa, xb, wb;
  gauss_jacobi(n, 0.0, 0.0, xa, wa);
  gauss_jacobi(n, 1.0, 0.0, xb, wb);
  xi.clear();
  w.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      xi.push_back(0.25 * (1.0 + xa[i]) * (1.0 - xb[j]));
      xi.push_back(0.5 * (1.0 + xb[j]));
      w.push_back(wa[i] * wb[j] / 8.0);
    }
}

// Fully symmetric volume rules exact to degree 3k - 1 (positive weights, interior points),
// written as orbits in barycentric coordinates: the centroid, orbits (a, a, 1-2a) of 3
// points, and orbits (a, b, 1-a-b) of 6 points. k = 1: one 3-point orbit (degree 2);
// k = 2: Radon's 7-point rule (degree 5, closed form); k = 3: a 16-point rule of degree 8
// with Dunavant's orbit structure (centroid, three 3-point orbits, one 6-point orbit),
// solved here by Gauss-Newton on the moment equations from approximate starting values.
// Weights sum to 1 here and are scaled to the reference area 1/2.
struct SymRule {
  using real = long double;
  real w0 = 0.0;                          // centroid weight (0: no centroid)
  std::vector<real> a3, w3;               // 3-point orbits
  std::vector<real> a6, b6, w6;           // 6-point orbits
  template <typename T>
  void points(std::vector<T>& xi, std::vector<T>& w) const {
    xi.clear();
    w.clear();
    auto add = [&](real l2, real l3, real wt) {
      xi.push_back(T(l2));
      xi.push_back(T(l3));
      w.push_back(T(0.5L * wt));
    };
    if (w0 != 0.0L) add(1.0L / 3.0L, 1.0L / 3.0L, w0);
    for (size_t o = 0; o < a3.size(); ++o) {
      const real a = a3[o], c = 1.0L - 2.0L * a;
      add(a, a, w3[o]);
      add(a, c, w3[o]);
      add(c, a, w3[o]);
    }
    for (size_t o = 0; o < a6.size(); ++o) {
      const real a = a6[o], b = b6[o], c = 1.0L - a - b;
      add(a, b, w6[o]);
      add(b, a, w6[o]);
      add(a, c, w6[o]);
      add(c, a, w6[o]);
      add(b, c, w6[o]);
      add(c, b, w6[o]);
    }
  }
  void get(std::vector<real>& p) const {
    p.clear();
    if (w0 != 0.0L) p.push_back(w0);
    for (size_t o = 0; o < a3.size(); ++o) { p.push_back(a3[o]); p.push_back(w3[o]); }
    for (size_t o = 0; o < a6.size(); ++o) { p.push_back(a6[o]); p.push_back(b6[o]); p.push_back(w6[o]); }
  }
  void set(const std::vector<real>& p) {
    size_t i = 0;
    if (w0 != 0.0L) w0 = p[i++];
    for (size_t o = 0; o < a3.size(); ++o) { a3[o] = p[i++]; w3[o] = p[i++]; }
    for (size_t o = 0; o < a6.size(); ++o) { a6[o] = p[i++]; b6[o] = p[i++]; w6[o] = p[i++]; }
  }
};

// Relative moment residuals of the rule with points xi and weights w: for i + j <= deg,
// (rule(xi1^i xi2^j) - exact) / exact, exact = i! j! / (i+j+2)! on the reference triangle.
template <typename T>
void moment_residual(const std::vector<T>& xi, const std::vector<T>& w, int deg, std::vector<T>& res) {
  res.clear();
  for (int i = 0; i <= deg; ++i)
    for (int j = 0; i + j <= deg; ++j) {
      T exact = 1;
      for (int t = 2; t <= i; ++t) exact *= t;
      for (int t = 2; t <= j; ++t) exact *= t;
      for (int t = 2; t <= i + j + 2; ++t) exact /= t;
      T q = 0;
      for (size_t p = 0; p < w.size(); ++p) {
        T v = w[p];
        for (int t = 0; t < i; ++t) v *= xi[2 * p];
        for (int t = 0; t < j; ++t) v *= xi[2 * p + 1];
        q += v;
      }
      res.push_back((q - exact) / exact);
    }
}

// Gauss-Newton with a finite-difference Jacobian on the relative moment equations (a
// consistent system), in extended precision so that the rule rounds to double correctly.
void refine_rule(SymRule& R, int deg) {
  using real = SymRule::real;
  std::vector<real> p, r, rp, rm, xi, w;
  R.get(p);
  const int np = int(p.size());
  for (int it = 0; it < 40; ++it) {
    R.points(xi, w);
    moment_residual(xi, w, deg, r);
    real mx = 0;
    for (real v : r) mx = std::max(mx, std::fabs(v));
    if (mx < 1e-18L) break;
    const int ne = int(r.size());
    std::vector<real> J(size_t(ne) * np);
    for (int c = 0; c < np; ++c) {
      const real h = 1e-9L * std::max(real(1e-3L), std::fabs(p[c]));
      std::vector<real> q = p;
      q[c] = p[c] + h;
      R.set(q);
      R.points(xi, w);
      moment_residual(xi, w, deg, rp);
      q[c] = p[c] - h;
      R.set(q);
      R.points(xi, w);
      moment_residual(xi, w, deg, rm);
      for (int e = 0; e < ne; ++e) J[size_t(e) * np + c] = (rp[e] - rm[e]) / (2 * h);
    }
    R.set(p);
    // normal equations J^T J d = -J^T r, Gaussian elimination with partial pivoting
    std::vector<real> A(size_t(np) * np, 0), b(np, 0);
    for (int e = 0; e < ne; ++e)
      for (int c = 0; c < np; ++c) {
        b[c] -= J[size_t(e) * np + c] * r[e];
        for (int d = 0; d < np; ++d) A[size_t(c) * np + d] += J[size_t(e) * np + c] * J[size_t(e) * np + d];
      }
    for (int c = 0; c < np; ++c) {
      int piv = c;
      for (int d = c + 1; d < np; ++d)
        if (std::fabs(A[size_t(d) * np + c]) > std::fabs(A[size_t(piv) * np + c])) piv = d;
      for (int d = 0; d < np; ++d) std::swap(A[size_t(c) * np + d], A[size_t(piv) * np + d]);
      std::swap(b[c], b[piv]);
      for (int d = c + 1; d < np; ++d) {
        const real f = A[size_t(d) * np + c] / A[size_t(c) * np + c];
        for (int e = c; e < np; ++e) A[size_t(d) * np + e] -= f * A[size_t(c) * np + e];
        b[d] -= f * b[c];
      }
    }
    std::vector<real> dlt(np);
    for (int c = np - 1; c >= 0; --c) {
      real v = b[c];
      for (int d = c + 1; d < np; ++d) v -= A[size_t(c) * np + d] * dlt[d];
      dlt[c] = v / A[size_t(c) * np + c];
    }
    for (int c = 0; c < np; ++c) p[c] += dlt[c];
    R.set(p);
  }
}

// The rule of degree 3k - 1 with kVolumePoints(k) points; false if it cannot be built.
bool build_symmetric_rule(int k, std::vector<double>& xi, std::vector<double>& w) {
  using real = SymRule::real;
  SymRule R;
  if (k == 1) {
    R.a3 = {1.0L / 6.0L};
    R.w3 = {1.0L / 3.0L};
  } else if (k == 2) {
    const real s15 = std::sqrt(15.0L);
    R.w0 = 9.0L / 40.0L;
    R.a3 = {(6.0L - s15) / 21.0L, (6.0L + s15) / 21.0L};
    R.w3 = {(155.0L - s15) / 1200.0L, (155.0L + s15) / 1200.0L};
  } else if (k == 3) {
    R.w0 = 0.1443L;
    R.a3 = {0.4593L, 0.1706L, 0.0505L};
    R.w3 = {0.0951L, 0.1032L, 0.0325L};
    R.a6 = {0.2631L};
    R.b6 = {0.0084L};
    R.w6 = {0.0272L};
    refine_rule(R, 3 * k - 1);
  } else {
    return false;
  }
  R.points(xi, w);
  // the rounded rule must be exact to rounding on every monomial up to the degree
  std::vector<double> r;
  moment_residual(xi, w, 3 * k - 1, r);
  for (double v : r)
    if (!(std::fabs(v) < 1e-14)) return false;
  for (size_t q = 0; q < w.size(); ++q)
    if (!(w[q] > 0.0) || !(xi[2 * q] > 0.0) || !(xi[2 * q + 1] > 0.0) || !(xi[2 * q] + xi[2 * q + 1] < 1.0))
      return false;
  return int(w.size()) == kVolumePoints(k);
}

// The rules are built once per process (the k = 3 refinement runs in extended precision).
bool symmetric_triangle_rule(int k, std::vector<double>& xi, std::vector<double>& w) {
  static std::once_flag once[4];
  static std::vector<double> rx[4], rw[4];
  static bool ok[4] = {false, false, false, false};
  if (k < 1 || k > 3) return false;
  std::call_once(once[k], [k] { ok[k] = build_symmetric_rule(k, rx[k], rw[k]); });
  xi = rx[k];
  w = rw[k];
  return ok[k];
}

const double kRefV[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};

}  // namespace

// ------------------------------------------------------------------- topology
int build_topology(int64_t n_tri, const int64_t* vid, const double* X, Topology& topo, std::string& err) {
  if (n_tri < 1 || !vid || !X) {
    err = "mesh: need n_tri >= 1 and non-NULL arrays";
    return DG_ERR_INVALID_ARG;
  }
  double scale = 1.0;
  for (int64_t i = 0; i < n_tri * 6; ++i) {
    if (!std::isfinite(X[i])) {
      err = "mesh: non-finite coordinate";
      return DG_ERR_INVALID_ARG;
    }
    scale = std::max(scale, std::fabs(X[i]) + 1.0);
  }
  const double tol = 1e-9 * scale;
  for (int64_t t = 0; t < n_tri; ++t) {
    const double* x = X + t * 6;
    double det = (x[2] - x[0]) * (x[5] - x[1]) - (x[4] - x[0]) * (x[3] - x[1]);
    if (!(det > 0.0)) {
      err = "mesh: triangle " + std::to_string(t) + " is degenerate or clockwise";
      return DG_ERR_MESH;
    }
  }
  struct Key {
    int64_t a, b, qx, qy;
    int64_t slot;  // 3 t + e
    int8_t orient;
  };
  std::vector<Key> keys(size_t(n_tri) * 3);
  for (int64_t t = 0; t < n_tri; ++t)
    for (int e = 0; e < 3; ++e) {
      int ia = (e + 1) % 3, ib = (e + 2) % 3;
      double dx = X[t * 6 + ib * 2] - X[t * 6 + ia * 2];
      double dy = X[t * 6 + ib * 2 + 1] - X[t * 6 + ia * 2 + 1];
      bool pos = dx > tol || (std::fabs(dx) <= tol && dy > 0.0);
      Key k;
      if (pos) {
        k.a = vid[t * 3 + ia];
        k.b = vid[t * 3 + ib];
        k.orient = 1;
      } else {
        k.a = vid[t * 3 + ib];
        k.b = vid[t * 3 + ia];
        k.orient = -1;
        dx = -dx;
        dy = -dy;
      }
      k.qx = std::llround(dx / tol);
      k.qy = std::llround(dy / tol);
      k.slot = t * 3 + e;
      keys[size_t(t) * 3 + e] = k;
    }
  std::vector<int64_t> order(keys.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t i, int64_t j) {
    const Key &p = keys[i], &q = keys[j];
    return std::tie(p.a, p.b, p.qx, p.qy, p.slot) < std::tie(q.a, q.b, q.qx, q.qy, q.slot);
  });
  // groups of equal keys; each must hold exactly two slots with opposite orientation
  struct Group {
    int64_t s0, s1;
  };
  std::vector<Group> groups;
  groups.reserve(keys.size() / 2);
  for (size_t i = 0; i < order.size();) {
    size_t j = i + 1;
    const Key& p = keys[order[i]];
    while (j < order.size()) {
      const Key& q = keys[order[j]];
      if (q.a != p.a || q.b != p.b || q.qx != p.qx || q.qy != p.qy) break;
      ++j;
    }
    size_t cnt = j - i;
    if (cnt == 1) {   // a wall: the facet has one side
      groups.push_back({keys[order[i]].slot, -1});
      i = j;
      continue;
    }
    if (cnt != 2) {
      err = "mesh: an edge is shared by " + std::to_string(cnt) + " triangles";
      return DG_ERR_MESH;
    }
    if (keys[order[i]].orient == keys[order[i + 1]].orient) {
      err = "mesh: a facet is traversed in the same direction by both triangles";
      return DG_ERR_MESH;
    }
    groups.push_back({keys[order[i]].slot, keys[order[i + 1]].slot});  // slot order: first appearance first
    i = j;
  }
  std::sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.s0 < b.s0; });
  topo.n_tri = n_tri;
  topo.n_facet = int64_t(groups.size());
  if (topo.n_facet > INT32_MAX / 4 || n_tri > INT32_MAX / 4) {
    err = "mesh too large for 32-bit indices";
    return DG_ERR_INVALID_ARG;
  }
  topo.tri_facet.assign(size_t(n_tri) * 3, -1);
  topo.tri_orient.assign(size_t(n_tri) * 3, 0);
  topo.facet_tri.assign(size_t(topo.n_facet) * 2, -1);
  topo.facet_loc.assign(size_t(topo.n_facet) * 2, -1);
  topo.n_boundary = 0;
  for (int64_t f = 0; f < topo.n_facet; ++f) {
    int64_t sl[2] = {groups[f].s0, groups[f].s1};
    if (sl[1] < 0) ++topo.n_boundary;
    for (int s = 0; s < (sl[1] < 0 ? 1 : 2); ++s) {
      topo.facet_tri[f * 2 + s] = int32_t(sl[s] / 3);
      topo.facet_loc[f * 2 + s] = int8_t(sl[s] % 3);
      topo.tri_facet[sl[s]] = int32_t(f);
      topo.tri_orient[sl[s]] = keys[sl[s]].orient;
    }
  }
  return DG_OK;
}

// ------------------------------------------------------------ reference tables
int build_reference(int k, RefTables& ref, std::string& err) {
  if (k < 1 || k > kMaxDegree) {
    err = "degree k must be 1.." + std::to_string(kMaxDegree);
    return DG_ERR_UNSUPPORTED;
  }
  ref.k = k;
  ref.ns = n_lat(k);
  ref.nw = n_lat(k - 1);
  ref.nl = k + 1;
  Dubiner B(k);
  // normalise on the reference triangle with a rule exact to degree 2k
  {
    std::vector<double> xi, w;
    triangle_rule(k + 2, xi, w);
    std::vector<double> v(B.ns);
    std::vector<double> nrm(B.ns, 0.0);
    for (size_t q = 0; q < w.size(); ++q) {
      B.eval(xi[2 * q], xi[2 * q + 1], v.data(), nullptr);
      for (int j = 0; j < B.ns; ++j) nrm[j] += w[q] * v[j] * v[j];
    }
    for (int j = 0; j < B.ns; ++j) B.norm[j] = 1.0 / std::sqrt(nrm[j]);
  }
  const int ns = ref.ns;
  // volume rule exact to degree 3k - 1: the fully symmetric rule (3, 7, 16 points)
  if (!symmetric_triangle_rule(k, ref.vxi, ref.vw)) {
    err = "reference set-up: the symmetric volume rule for k = " + std::to_string(k) + " is not exact";
    return DG_ERR_MESH;
  }
  ref.nq = int(ref.vw.size());
  ref.vphi.resize(size_t(ref.nq) * ns);
  ref.vdphi.resize(size_t(ref.nq) * ns * 2);
  for (int q = 0; q < ref.nq; ++q)
    B.eval(ref.vxi[2 * q], ref.vxi[2 * q + 1], &ref.vphi[size_t(q) * ns], &ref.vdphi[size_t(q) * ns * 2]);
  // facet rule: ceil((3k+1)/2) Gauss-Legendre points on [0,1]
  ref.nqf = (3 * k + 2) / 2;
  {
    std::vector<double> x, w;
    gauss_jacobi(ref.nqf, 0.0, 0.0, x, w);
    ref.ft.resize(ref.nqf);
    ref.fw.resize(ref.nqf);
    for (int q = 0; q < ref.nqf; ++q) {
      ref.ft[q] = 0.5 * (x[q] + 1.0);
      ref.fw[q] = 0.5 * w[q];
    }
  }
  ref.fphi.resize(size_t(3) * ref.nqf * ns);
  ref.fdphi.resize(size_t(3) * ref.nqf * ns * 2);
  for (int e = 0; e < 3; ++e) {
    const double* a = kRefV[(e + 1) % 3];
    const double* b = kRefV[(e + 2) % 3];
    for (int q = 0; q < ref.nqf; ++q) {
      double t = ref.ft[q];
      double x1 = a[0] + t * (b[0] - a[0]), x2 = a[1] + t * (b[1] - a[1]);
      B.eval(x1, x2, &ref.fphi[(size_t(e) * ref.nqf + q) * ns], &ref.fdphi[(size_t(e) * ref.nqf + q) * ns * 2]);
    }
  }
  // lattice tables
  ref.lat_phi.resize(size_t(ns) * ns);
  {
    int p = 0;
    for (int j = 0; j <= k; ++j)
      for (int i = 0; i <= k - j; ++i, ++p) B.eval(double(i) / k, double(j) / k, &ref.lat_phi[size_t(p) * ns], nullptr);
  }
  ref.lat_inv = ref.lat_phi;
  if (!invert(ref.lat_inv, ns)) {
    err = "lattice Vandermonde singular";
    return DG_ERR_UNSUPPORTED;
  }
  const int nw = ref.nw;
  ref.plat_phi.resize(size_t(nw) * nw);
  {
    std::vector<double> v(ns);
    int m = k - 1, p = 0;
    if (m == 0) {
      B.eval(1.0 / 3.0, 1.0 / 3.0, v.data(), nullptr);
      for (int j = 0; j < nw; ++j) ref.plat_phi[j] = v[j];
    } else {
      for (int jj = 0; jj <= m; ++jj)
        for (int ii = 0; ii <= m - jj; ++ii, ++p) {
          B.eval(double(ii) / m, double(jj) / m, v.data(), nullptr);
          for (int j = 0; j < nw; ++j) ref.plat_phi[size_t(p) * nw + j] = v[j];
        }
    }
  }
  ref.mu_lat.resize(size_t(k + 1) * ref.nl);
  for (int i = 0; i <= k; ++i)
    for (int m = 0; m < ref.nl; ++m)
      ref.mu_lat[size_t(i) * ref.nl + m] = std::sqrt(2.0 * m + 1.0) * legendre(m, 2.0 * (double(i) / k) - 1.0);
  return DG_OK;
}

// ------------------------------------------------------------ element classes
namespace {

// Operators of eq. (12) for one triangle with orthonormal bases (so M_T = I):
// D_T[m][(c,j)] = (z_m, d_c psi_j)_T, C_T[(e,m)][(c,j)] = <mu_m, psi_j n_{e,c}>_{F_e}
// with mu_m(s) = sqrt(2m+1) P_m(2s-1) in the element's counter-clockwise parameter s.
void class_ops(const RefTables& ref, const double* x, ClassOps& co) {
  const int ns = ref.ns, nd = 2 * ns, nw = ref.nw, nl = ref.nl;
  co.J[0] = x[2] - x[0];
  co.J[1] = x[4] - x[0];
  co.J[2] = x[3] - x[1];
  co.J[3] = x[5] - x[1];
  co.det = co.J[0] * co.J[3] - co.J[1] * co.J[2];
  co.Jinv[0] = co.J[3] / co.det;
  co.Jinv[1] = -co.J[1] / co.det;
  co.Jinv[2] = -co.J[2] / co.det;
  co.Jinv[3] = co.J[0] / co.det;
  for (int e = 0; e < 3; ++e) {
    int a = (e + 1) % 3, b = (e + 2) % 3;
    double dx = x[2 * b] - x[2 * a], dy = x[2 * b + 1] - x[2 * a + 1];
    double l = std::sqrt(dx * dx + dy * dy);
    co.flen[e] = l;
    co.normal[e][0] = dy / l;
    co.normal[e][1] = -dx / l;
  }
  const double s = 1.0 / std::sqrt(co.det);
  // D (volume rule is exact to 3k-1 >= 2k-2); 2|T| s^2 = 1
  std::vector<double> D(size_t(nw) * nd, 0.0);
  for (int q = 0; q < ref.nq; ++q) {
    double w = ref.vw[q];
    for (int m = 0; m < nw; ++m) {
      double z = ref.vphi[size_t(q) * ns + m];
      for (int j = 0; j < ns; ++j) {
        double g0 = ref.vdphi[(size_t(q) * ns + j) * 2], g1 = ref.vdphi[(size_t(q) * ns + j) * 2 + 1];
        for (int c = 0; c < 2; ++c) {
          double dc = g0 * co.Jinv[0 * 2 + c] + g1 * co.Jinv[1 * 2 + c];
          D[size_t(m) * nd + c * ns + j] += w * z * dc;
        }
      }
    }
  }
  std::vector<double> C(size_t(3 * nl) * nd, 0.0);
  for (int e = 0; e < 3; ++e)
    for (int q = 0; q < ref.nqf; ++q) {
      double w = ref.fw[q] * co.flen[e] * s;
      for (int m = 0; m < nl; ++m) {
        double mu = std::sqrt(2.0 * m + 1.0) * legendre(m, 2.0 * ref.ft[q] - 1.0);
        for (int j = 0; j < ns; ++j) {
          double v = ref.fphi[(size_t(e) * ref.nqf + q) * ns + j];
          for (int c = 0; c < 2; ++c) C[size_t(e * nl + m) * nd + c * ns + j] += w * mu * v * co.normal[e][c];
        }
      }
    }
  // P = I - D^T (D D^T)^-1 D, W = -(D D^T)^-1 D
  std::vector<double> Dt = transpose(D, nw, nd);
  std::vector<double> DDt = matmul(D, Dt, nw, nd, nw);
  invert(DDt, nw);
  std::vector<double> Wm = matmul(DDt, D, nw, nw, nd);
  for (double& v : Wm) v = -v;
  std::vector<double> P = matmul(Dt, Wm, nd, nw, nd);  // -D^T (DD^T)^-1 D
  for (int i = 0; i < nd; ++i) P[size_t(i) * nd + i] += 1.0;
  // symmetrise (exact in exact arithmetic)
  for (int i = 0; i < nd; ++i)
    for (int j = i + 1; j < nd; ++j) {
      double a = 0.5 * (P[size_t(i) * nd + j] + P[size_t(j) * nd + i]);
      P[size_t(i) * nd + j] = P[size_t(j) * nd + i] = a;
    }
  co.P = P;
  co.W = Wm;
  co.G = matmul(C, P, 3 * nl, nd, nd);
  std::vector<double> Ct = transpose(C, 3 * nl, nd);
  co.S = matmul(co.G, Ct, 3 * nl, nd, 3 * nl);
  for (int i = 0; i < 3 * nl; ++i)
    for (int j = i + 1; j < 3 * nl; ++j) {
      double a = 0.5 * (co.S[size_t(i) * 3 * nl + j] + co.S[size_t(j) * 3 * nl + i]);
      co.S[size_t(i) * 3 * nl + j] = co.S[size_t(j) * 3 * nl + i] = a;
    }
  co.WCt = matmul(Wm, Ct, nw, nd, 3 * nl);
}

}  // namespace

int build_host_mesh(int64_t n_tri, const int64_t* vid, const double* X, int k, double alpha, HostMesh& hm,
                    std::string& err, const int8_t* edge_kind) {
  int rc = build_reference(k, hm.ref, err);
  if (rc) return rc;
  rc = build_topology(n_tri, vid, X, hm.topo, err);
  if (rc) return rc;
  // kinds of the boundary facets (Sec. 2.5, eq. (be)): wall, inflow or outflow, from the kind of
  // the single triangle edge of each boundary facet; interior facets are kWall (not used)
  hm.facet_kind.assign(hm.topo.n_facet, kWall);
  hm.has_outflow = false;
  hm.has_inflow = false;
  if (edge_kind) {
    for (int64_t f = 0; f < hm.topo.n_facet; ++f) {
      if (hm.topo.facet_tri[f * 2 + 1] >= 0) continue;
      const int8_t kd = edge_kind[size_t(hm.topo.facet_tri[f * 2]) * 3 + hm.topo.facet_loc[f * 2]];
      if (kd < kWall || kd > kOutflow) {
        err = "edge kinds are 0 (wall), 1 (inflow) or 2 (outflow)";
        return DG_ERR_INVALID_ARG;
      }
      hm.facet_kind[f] = kd;
      hm.has_outflow = hm.has_outflow || kd == kOutflow;
      hm.has_inflow = hm.has_inflow || kd == kInflow;
    }
  }
  const RefTables& ref = hm.ref;
  hm.k = k;
  hm.ns = ref.ns;
  hm.nd = 2 * ref.ns;
  hm.nw = ref.nw;
  hm.nl = ref.nl;
  hm.alpha = alpha;
  const int nl = hm.nl;
  const Topology& T = hm.topo;
  // geometry classes: Jacobians equal to 1e-11 of the largest entry share one set of operators
  double jmax = 0.0;
  for (int64_t t = 0; t < n_tri; ++t) {
    const double* x = X + t * 6;
    for (int c = 1; c < 3; ++c)
      for (int d = 0; d < 2; ++d) jmax = std::max(jmax, std::fabs(x[2 * c + d] - x[d]));
  }
  const double jtol = 1e-11 * jmax;
  std::map<std::array<int64_t, 4>, int32_t> cls;
  hm.tri_class.resize(n_tri);
  std::vector<int64_t> rep;
  for (int64_t t = 0; t < n_tri; ++t) {
    const double* x = X + t * 6;
    std::array<int64_t, 4> key = {std::llround((x[2] - x[0]) / jtol), std::llround((x[4] - x[0]) / jtol),
                                  std::llround((x[3] - x[1]) / jtol), std::llround((x[5] - x[1]) / jtol)};
    auto it = cls.find(key);
    if (it == cls.end()) {
      it = cls.emplace(key, int32_t(rep.size())).first;
      rep.push_back(t);
    }
    hm.tri_class[t] = it->second;
  }
  hm.classes.resize(rep.size());
  for (size_t c = 0; c < rep.size(); ++c) class_ops(ref, X + rep[c] * 6, hm.classes[c]);
  hm.area_total = 0.0;
  for (int64_t t = 0; t < n_tri; ++t) hm.area_total += 0.5 * hm.classes[hm.tri_class[t]].det;
  // neighbours and penalties
  hm.tri_nbr.resize(size_t(n_tri) * 3);
  hm.tri_nbr_loc.resize(size_t(n_tri) * 3);
  // (a wall side has no neighbour: -1, -1)
  for (int64_t f = 0; f < T.n_facet; ++f)
    for (int s = 0; s < 2; ++s) {
      int32_t t = T.facet_tri[f * 2 + s], o = T.facet_tri[f * 2 + 1 - s];
      if (t < 0) continue;
      int e = T.facet_loc[f * 2 + s];
      hm.tri_nbr[size_t(t) * 3 + e] = o;
      hm.tri_nbr_loc[size_t(t) * 3 + e] = T.facet_loc[f * 2 + 1 - s];
    }
  auto diam = [&](int32_t t) {
    const ClassOps& c = hm.classes[hm.tri_class[t]];
    return std::max(c.flen[0], std::max(c.flen[1], c.flen[2]));
  };
  hm.facet_sigma.resize(T.n_facet);
  for (int64_t f = 0; f < T.n_facet; ++f) {
    const int32_t t0 = T.facet_tri[f * 2], t1 = T.facet_tri[f * 2 + 1];
    hm.facet_sigma[f] = alpha * k * k / std::max(diam(t0), diam(t1 < 0 ? t0 : t1));
  }
  // facet stencils: row F = sum over both sides T of D(sigma_e) S_T[e][e'] D(sigma_e') lam_{F_e'}
  // with D(sigma) = diag(sigma^m) mapping the global (canonical) coefficients to T's own.
  hm.facet_nbr.resize(size_t(T.n_facet) * 4);
  hm.facet_stencil.resize(T.n_facet);
  hm.facet_side0.resize(T.n_facet);
  std::map<std::vector<int64_t>, int32_t> st;
  hm.stencil_blocks.clear();
  hm.stencil_binv.clear();
  const int L3 = 3 * nl;
  // A wall facet has one side: its row couples only to the other two facets of that side
  // (slots 3 and 4 point at the facet itself with zero blocks).
  for (int64_t f = 0; f < T.n_facet; ++f) {
    int side_order[2] = {0, 1};
    const int nside = T.facet_tri[f * 2 + 1] < 0 ? 1 : 2;
    if (nside == 2) {
      int32_t t0 = T.facet_tri[f * 2], t1 = T.facet_tri[f * 2 + 1];
      auto key0 = std::make_pair(hm.tri_class[t0], int(T.facet_loc[f * 2]));
      auto key1 = std::make_pair(hm.tri_class[t1], int(T.facet_loc[f * 2 + 1]));
      if (key1 < key0) std::swap(side_order[0], side_order[1]);
    }
    std::vector<int64_t> key;
    hm.facet_side0[f] = T.facet_tri[f * 2 + side_order[0]];
    if (nside == 1) {
      key.push_back(-1);
      hm.facet_nbr[f * 4 + 2] = int32_t(f);
      hm.facet_nbr[f * 4 + 3] = int32_t(f);
    }
    for (int si = 0; si < nside; ++si) {
      int s = side_order[si];
      int32_t t = T.facet_tri[f * 2 + s];
      int e = T.facet_loc[f * 2 + s];
      key.push_back(hm.tri_class[t]);
      key.push_back(e);
      for (int ee = 0; ee < 3; ++ee) key.push_back(T.tri_orient[size_t(t) * 3 + ee]);
      hm.facet_nbr[f * 4 + si * 2 + 0] = T.tri_facet[size_t(t) * 3 + (e + 1) % 3];
      hm.facet_nbr[f * 4 + si * 2 + 1] = T.tri_facet[size_t(t) * 3 + (e + 2) % 3];
    }
    // outflow (p = 0, eq. (be)): the facet's multipliers are zero, so its row is the identity
    // and the other rows do not couple to it
    const bool own_out = hm.facet_kind[f] == kOutflow;
    key.push_back(own_out ? 1 : 0);
    bool slot_out[4];
    for (int b = 0; b < 4; ++b) {
      slot_out[b] = hm.facet_kind[hm.facet_nbr[f * 4 + b]] == kOutflow && hm.facet_nbr[f * 4 + b] != f;
      key.push_back(slot_out[b] ? 1 : 0);
    }
    auto it = st.find(key);
    if (it == st.end()) {
      int32_t id = int32_t(st.size());
      it = st.emplace(key, id).first;
      std::vector<double> blk(size_t(5) * nl * nl, 0.0);
      for (int si = 0; si < nside; ++si) {
        int s = side_order[si];
        int32_t t = T.facet_tri[f * 2 + s];
        int e = T.facet_loc[f * 2 + s];
        const ClassOps& co = hm.classes[hm.tri_class[t]];
        auto sgn = [&](int ee, int m) { return (T.tri_orient[size_t(t) * 3 + ee] < 0 && (m & 1)) ? -1.0 : 1.0; };
        const int targets[3] = {e, (e + 1) % 3, (e + 2) % 3};
        for (int b = 0; b < 3; ++b) {
          int ee = targets[b];
          int slot = (b == 0) ? 0 : 1 + si * 2 + (b - 1);
          for (int m = 0; m < nl; ++m)
            for (int mm = 0; mm < nl; ++mm)
              blk[(size_t(slot) * nl + m) * nl + mm] +=
                  sgn(e, m) * co.S[size_t(e * nl + m) * L3 + ee * nl + mm] * sgn(ee, mm);
        }
      }
      if (own_out) {
        std::fill(blk.begin(), blk.end(), 0.0);
        for (int m = 0; m < nl; ++m) blk[size_t(m) * nl + m] = 1.0;
      }
      for (int b = 0; b < 4; ++b)
        if (slot_out[b]) std::fill(blk.begin() + size_t(b + 1) * nl * nl, blk.begin() + size_t(b + 2) * nl * nl, 0.0);
      std::vector<double> inv(blk.begin(), blk.begin() + nl * nl);
      if (!invert(inv, nl)) {
        err = "singular facet block";
        return DG_ERR_MESH;
      }
      hm.stencil_blocks.insert(hm.stencil_blocks.end(), blk.begin(), blk.end());
      hm.stencil_binv.insert(hm.stencil_binv.end(), inv.begin(), inv.end());
    }
    hm.facet_stencil[f] = it->second;
  }
  hm.n_stencil = int(st.size());
  return DG_OK;
}

// ----------------------------------------------------------------- lattice
namespace {

// Inverse (or, with pinv, pseudo-inverse) of a Hermitian C x C matrix given as [C][C][2].
bool hermitian_inverse(const double* A, int C, double* out, bool pinv) {
  if (!pinv) {
    // real embedding [[Re, -Im], [Im, Re]] is symmetric; invert it and read the blocks back
    const int n = 2 * C;
    std::vector<double> E(size_t(n) * n);
    for (int i = 0; i < C; ++i)
      for (int j = 0; j < C; ++j) {
        const double re = A[(i * C + j) * 2], im = A[(i * C + j) * 2 + 1];
        E[size_t(i) * n + j] = re;
        E[size_t(i) * n + C + j] = -im;
        E[size_t(C + i) * n + j] = im;
        E[size_t(C + i) * n + C + j] = re;
      }
    if (!invert(E, n)) return false;
    for (int i = 0; i < C; ++i)
      for (int j = 0; j < C; ++j) {
        out[(i * C + j) * 2] = E[size_t(i) * n + j];
        out[(i * C + j) * 2 + 1] = E[size_t(C + i) * n + j];
      }
    return true;
  }
  // kappa = 0: the symbol is real symmetric; invert its eigenvalues above 1e-10 of the largest
  std::vector<double> R(size_t(C) * C), ev, V;
  for (int i = 0; i < C * C; ++i) R[i] = A[2 * i];
  sym_eig(R, C, ev, V);
  double emax = 0.0;
  for (double e : ev) emax = std::max(emax, std::fabs(e));
  for (int i = 0; i < C; ++i)
    for (int j = 0; j < C; ++j) {
      double v = 0.0;
      for (int l = 0; l < C; ++l)
        if (std::fabs(ev[l]) > 1e-10 * emax) v += V[size_t(i) * C + l] * V[size_t(j) * C + l] / ev[l];
      out[(i * C + j) * 2] = v;
      out[(i * C + j) * 2 + 1] = 0.0;
    }
  return true;
}

// Eigen-decomposition of a Hermitian C x C matrix A ([C][C][2]) by cyclic complex Jacobi
// rotations: A = V diag(ev) V^H with V unitary, V[b][i] = component b of eigenvector i
// ([C][C][2]). Each rotation first turns A_pq into |A_pq| by a phase on index q, then
// applies the real rotation that zeros it.
void hermitian_eig(const double* A0, int C, std::vector<double>& ev, std::vector<double>& V) {
  std::vector<double> A(A0, A0 + size_t(C) * C * 2);
  V.assign(size_t(C) * C * 2, 0.0);
  for (int i = 0; i < C; ++i) V[(size_t(i) * C + i) * 2] = 1.0;
  auto re = [&](std::vector<double>& M, int i, int j) -> double& { return M[(size_t(i) * C + j) * 2]; };
  auto im = [&](std::vector<double>& M, int i, int j) -> double& { return M[(size_t(i) * C + j) * 2 + 1]; };
  double scale = 0.0;
  for (int i = 0; i < C; ++i) scale = std::max(scale, std::fabs(re(A, i, i)));
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < C; ++i)
      for (int j = i + 1; j < C; ++j) off += re(A, i, j) * re(A, i, j) + im(A, i, j) * im(A, i, j);
    if (off <= 1e-64 * scale * scale) break;
    for (int p = 0; p < C; ++p)
      for (int q = p + 1; q < C; ++q) {
        const double br = re(A, p, q), bi = im(A, p, q), bm = std::hypot(br, bi);
        if (bm <= 1e-300) continue;
        // phase w = conj(b) / |b| on index q: A_iq *= w, A_qj *= conj(w), V_iq *= w
        const double wr = br / bm, wi = -bi / bm;
        for (int i = 0; i < C; ++i) {
          if (i == q) continue;
          const double xr = re(A, i, q), xi = im(A, i, q);
          re(A, i, q) = xr * wr - xi * wi;
          im(A, i, q) = xr * wi + xi * wr;
          re(A, q, i) = re(A, i, q);
          im(A, q, i) = -im(A, i, q);
        }
        for (int i = 0; i < C; ++i) {
          const double xr = re(V, i, q), xi = im(V, i, q);
          re(V, i, q) = xr * wr - xi * wi;
          im(V, i, q) = xr * wi + xi * wr;
        }
        // real rotation in the (p, q) plane: tan 2t = 2 |b| / (A_qq - A_pp)
        const double app = re(A, p, p), aqq = re(A, q, q);
        const double theta = (aqq - app) / (2.0 * bm);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < C; ++k) {   // columns p, q
          const double pr = re(A, k, p), pi = im(A, k, p), qr = re(A, k, q), qi = im(A, k, q);
          re(A, k, p) = c * pr - sn * qr;
          im(A, k, p) = c * pi - sn * qi;
          re(A, k, q) = sn * pr + c * qr;
          im(A, k, q) = sn * pi + c * qi;
        }
        for (int k = 0; k < C; ++k) {   // rows p, q
          const double pr = re(A, p, k), pi = im(A, p, k), qr = re(A, q, k), qi = im(A, q, k);
          re(A, p, k) = c * pr - sn * qr;
          im(A, p, k) = c * pi - sn * qi;
          re(A, q, k) = sn * pr + c * qr;
          im(A, q, k) = sn * pi + c * qi;
        }
        for (int k = 0; k < C; ++k) {
          const double pr = re(V, k, p), pi = im(V, k, p), qr = re(V, k, q), qi = im(V, k, q);
          re(V, k, p) = c * pr - sn * qr;
          im(V, k, p) = c * pi - sn * qi;
          re(V, k, q) = sn * pr + c * qr;
          im(V, k, q) = sn * pi + c * qi;
        }
        re(A, p, q) = im(A, p, q) = re(A, q, p) = im(A, q, p) = 0.0;
      }
  }
  ev.resize(C);
  for (int i = 0; i < C; ++i) ev[i] = re(A, i, i);
}

}  // namespace

void build_lattice(const HostMesh& hm, const double* X, Lattice& L, bool eig_half) {
  L = Lattice();
  const Topology& T = hm.topo;
  const int64_t n = T.n_tri;
  if (T.n_boundary > 0) {
    L.why = "the mesh has walls (boundary facets)";
    return;
  }
  const int N = int(std::llround(std::sqrt(double(n) / 2.0)));
  if (int64_t(2) * N * N != n) {
    L.why = "triangle count is not 2 N^2";
    return;
  }
  if (hm.classes.size() != 2 || hm.n_stencil != 3) {
    L.why = "not two element classes and three facet stencils";
    return;
  }
  // lower triangles: v1 - v0 = (h, 0), v2 - v0 = (h, h); upper: v1 - v0 = (h, h), v2 - v0 = (0, h)
  int lower = -1;
  double h = 0.0;
  for (int c = 0; c < 2; ++c) {
    const double* J = hm.classes[c].J;   // row-major [v1-v0, v2-v0] as columns
    const double a = J[0];
    if (a > 0 && std::fabs(J[2]) <= 1e-9 * a && std::fabs(J[1] - a) <= 1e-9 * a && std::fabs(J[3] - a) <= 1e-9 * a) {
      lower = c;
      h = a;
    }
  }
  if (lower < 0) {
    L.why = "element classes are not split-square triangles";
    return;
  }
  const ClassOps& up = hm.classes[1 - lower];
  if (!(std::fabs(up.J[0] - h) <= 1e-9 * h && std::fabs(up.J[2] - h) <= 1e-9 * h && std::fabs(up.J[1]) <= 1e-9 * h &&
        std::fabs(up.J[3] - h) <= 1e-9 * h)) {
    L.why = "element classes are not split-square triangles";
    return;
  }
  const double x0 = X[0], y0 = X[1];
  std::vector<int32_t> cell(size_t(n) * 2);
  std::vector<int32_t> seen(size_t(2) * N * N, -1);
  for (int64_t t = 0; t < n; ++t) {
    const double fx = (X[t * 6] - x0) / h, fy = (X[t * 6 + 1] - y0) / h;
    const double rx = std::round(fx), ry = std::round(fy);
    if (std::fabs(fx - rx) > 1e-6 || std::fabs(fy - ry) > 1e-6) {
      L.why = "corner 0 off the lattice";
      return;
    }
    const int ci = int(((long long)rx % N + N) % N), cj = int(((long long)ry % N + N) % N);
    cell[t * 2] = ci;
    cell[t * 2 + 1] = cj;
    const int cls = hm.tri_class[t] == lower ? 0 : 1;
    int32_t& s = seen[(size_t(cls) * N + cj) * N + ci];
    if (s >= 0) {
      L.why = "two triangles in one lattice slot";
      return;
    }
    s = int32_t(t);
  }
  const int nl = hm.nl, ntype = hm.n_stencil, C = ntype * nl;
  L.facet_of.assign(size_t(ntype) * N * N, -1);
  std::vector<int32_t> fcell(size_t(T.n_facet) * 2);
  for (int64_t f = 0; f < T.n_facet; ++f) {
    const int32_t t0 = hm.facet_side0[f];
    const int ty = hm.facet_stencil[f];
    const int ci = cell[size_t(t0) * 2], cj = cell[size_t(t0) * 2 + 1];
    fcell[f * 2] = ci;
    fcell[f * 2 + 1] = cj;
    int32_t& s = L.facet_of[(size_t(ty) * N + cj) * N + ci];
    if (s >= 0) {
      L.why = "two facets in one lattice slot";
      return;
    }
    s = int32_t(f);
  }
  // neighbour offsets (mod N) and types must be the same for every facet of a type
  std::vector<int> off(size_t(ntype) * 4 * 3, -1);   // per type, per neighbour: (type, di, dj)
  for (int64_t f = 0; f < T.n_facet; ++f) {
    const int ty = hm.facet_stencil[f];
    for (int b = 0; b < 4; ++b) {
      const int32_t nb = hm.facet_nbr[f * 4 + b];
      const int tb = hm.facet_stencil[nb];
      const int di = ((fcell[size_t(nb) * 2] - fcell[f * 2]) % N + N) % N;
      const int dj = ((fcell[size_t(nb) * 2 + 1] - fcell[f * 2 + 1]) % N + N) % N;
      int* o = &off[(size_t(ty) * 4 + b) * 3];
      if (o[0] < 0) {
        o[0] = tb;
        o[1] = di;
        o[2] = dj;
      } else if (o[0] != tb || o[1] != di || o[2] != dj) {
        L.why = "facet stencil is not translation invariant";
        return;
      }
    }
  }
  // symbol and its inverse, one wavenumber at a time (threads over k_i)
  L.N = N;
  L.ntype = ntype;
  L.C = C;
  const int NK = N / 2 + 1, NE = C * C + C;
  if (eig_half) L.seig.assign(size_t(NK) * N * NE * 2, 0.0);
  else L.sinv.assign(size_t(N) * N * C * C * 2, 0.0);
  const double two_pi = 6.283185307179586476925286766559;
  const std::vector<double>& B = hm.stencil_blocks;
  bool fail = false;
  auto work = [&](int k0, int k1) {
    std::vector<double> S(size_t(C) * C * 2), ev, V;
    for (int ki = k0; ki < k1; ++ki)
      for (int kj = 0; kj < N; ++kj) {
        std::fill(S.begin(), S.end(), 0.0);
        for (int ty = 0; ty < ntype; ++ty)
          for (int b = 0; b < 5; ++b) {
            int tb = ty, di = 0, dj = 0;
            if (b > 0) {
              const int* o = &off[(size_t(ty) * 4 + (b - 1)) * 3];
              tb = o[0];
              di = o[1];
              dj = o[2];
            }
            const double ang = two_pi * double((long long)ki * di + (long long)kj * dj) / double(N);
            const double cr = std::cos(ang), cim = std::sin(ang);
            const double* blk = &B[(size_t(ty) * 5 + b) * nl * nl];
            for (int m = 0; m < nl; ++m)
              for (int mm = 0; mm < nl; ++mm) {
                const double v = blk[m * nl + mm];
                double* d = &S[((size_t(ty * nl + m) * C) + tb * nl + mm) * 2];
                d[0] += v * cr;
                d[1] += v * cim;
              }
          }
        if (!eig_half) {
          double* out = &L.sinv[(size_t(ki) * N + kj) * C * C * 2];
          if (!hermitian_inverse(S.data(), C, out, ki == 0 && kj == 0)) fail = true;
          continue;
        }
        // eigen form: V (C x C) then the inverse eigenvalues (0 for the kernel at kappa = 0)
        hermitian_eig(S.data(), C, ev, V);
        double emax = 0.0;
        for (double e : ev) emax = std::max(emax, std::fabs(e));
        double* out = &L.seig[(size_t(ki) * N + kj) * NE * 2];
        for (int i = 0; i < C * C * 2; ++i) out[i] = V[i];
        for (int i = 0; i < C; ++i) {
          const bool kernel = ki == 0 && kj == 0 && std::fabs(ev[i]) <= 1e-10 * emax;
          if (!kernel && !(ev[i] > 0.0)) fail = true;
          out[C * C * 2 + 2 * i] = kernel ? 0.0 : 1.0 / ev[i];
        }
      }
  };
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (N < 8) nth = 1;
  std::vector<std::thread> th;
  const int nki = eig_half ? NK : N;
  for (unsigned i = 0; i < nth; ++i) {
    const int a = int(int64_t(nki) * i / nth), b = int(int64_t(nki) * (i + 1) / nth);
    th.emplace_back(work, a, b);
  }
  for (auto& t : th) t.join();
  if (fail) {
    L.why = "singular Fourier symbol";
    L.sinv.clear();
    L.seig.clear();
    return;
  }
  L.twiddle.resize(size_t(N) * 2);
  for (int t = 0; t < N; ++t) {
    L.twiddle[2 * t] = std::cos(two_pi * t / N);
    L.twiddle[2 * t + 1] = -std::sin(two_pi * t / N);
  }
  L.ok = true;
}

void renumber_facets_lattice(HostMesh& hm, Lattice& L) {
  Topology& T = hm.topo;
  const int64_t nF = T.n_facet;
  std::vector<int32_t> nw(nF), old_of_new(nF);
  for (int64_t n = 0; n < nF; ++n) {
    old_of_new[n] = L.facet_of[n];
    nw[L.facet_of[n]] = int32_t(n);
  }
  auto permute = [&](auto& v, int width) {
    auto w = v;
    for (int64_t n = 0; n < nF; ++n)
      for (int c = 0; c < width; ++c) w[n * width + c] = v[size_t(old_of_new[n]) * width + c];
    v.swap(w);
  };
  permute(T.facet_tri, 2);
  permute(T.facet_loc, 2);
  permute(hm.facet_sigma, 1);
  permute(hm.facet_nbr, 4);
  for (auto& x : hm.facet_nbr) x = nw[x];
  permute(hm.facet_stencil, 1);
  permute(hm.facet_side0, 1);
  permute(hm.facet_kind, 1);
  for (auto& x : T.tri_facet) x = nw[x];
  for (int64_t n = 0; n < nF; ++n) L.facet_of[n] = int32_t(n);
  hm.facet_ext = old_of_new;
}

}  // namespace dgdf

namespace dgdf {
void inflow_data(const HostMesh& hm, const double* vals, std::vector<double>& uq, std::vector<double>& dmom) {
  const Topology& T = hm.topo;
  const RefTables& ref = hm.ref;
  const int k = hm.k, nl = hm.nl, nqf = ref.nqf;
  uq.assign(size_t(T.n_facet) * nqf * 2, 0.0);
  dmom.assign(size_t(T.n_facet) * nl, 0.0);
  // Lagrange basis of the k+1 equispaced edge points at the facet rule's points
  std::vector<double> Lq(size_t(k + 1) * nqf);
  for (int i = 0; i <= k; ++i)
    for (int q = 0; q < nqf; ++q) {
      double v = 1.0;
      for (int j = 0; j <= k; ++j)
        if (j != i) v *= (ref.ft[q] - double(j) / k) / (double(i - j) / k);
      Lq[size_t(i) * nqf + q] = v;
    }
  std::vector<double> ue(size_t(nqf) * 2);
  for (int64_t f = 0; f < T.n_facet; ++f) {
    if (hm.facet_kind[f] != kInflow) continue;
    const int64_t t = T.facet_tri[f * 2];
    const int e = T.facet_loc[f * 2];
    const bool canon = T.tri_orient[size_t(t) * 3 + e] > 0;
    const double* v = vals + (size_t(t) * 3 + e) * (k + 1) * 2;
    for (int q = 0; q < nqf; ++q)
      for (int c = 0; c < 2; ++c) {
        double a = 0.0;
        for (int i = 0; i <= k; ++i) a += Lq[size_t(i) * nqf + q] * v[i * 2 + c];
        ue[q * 2 + c] = a;
      }
    const ClassOps& co = hm.classes[hm.tri_class[t]];
    for (int q = 0; q < nqf; ++q) {
      // canonical point q is the triangle's point q, or nqf-1-q when it runs the facet backwards
      const int qe = canon ? q : nqf - 1 - q;
      double* o = &uq[(size_t(f) * nqf + q) * 2];
      o[0] = ue[qe * 2];
      o[1] = ue[qe * 2 + 1];
      const double un = o[0] * co.normal[e][0] + o[1] * co.normal[e][1];
      const double w = ref.fw[q] * co.flen[e];
      for (int m = 0; m < nl; ++m)
        dmom[size_t(f) * nl + m] += w * std::sqrt(2.0 * m + 1.0) * legendre(m, 2.0 * ref.ft[q] - 1.0) * un;
    }
  }
}

void symmetric_eigen(const std::vector<double>& A, int n, std::vector<double>& evals, std::vector<double>& evecs) {
  sym_eig(A, n, evals, evecs);
}

void host_gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  gauss_jacobi(n, a, b, x, w);
}

bool host_invert(std::vector<double>& A, int n) { return invert(A, n); }
}  // namespace dgdf
