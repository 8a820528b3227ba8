// Host set-up of the multilevel preconditioner of the facet system (see multilevel.hpp)
// and its host reference V-cycle. FP64, no CUDA.
#include "multilevel.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/dgdf.h"

namespace dgdf {
namespace {

using Vec = std::vector<double>;

double dot(const Vec& a, const Vec& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// ---- operators of one level on the host

// y = A x on a stencil level: row F, modes i < bs: sum over the five stencil slots of the
// leading bs x bs sub-block of S's (k+1) x (k+1) block times the neighbour's first bs values.
void stencil_apply(const HostMesh& hm, int bs, const double* x, double* y) {
  const int nl = hm.nl;
  const int64_t nf = hm.topo.n_facet;
  for (int64_t f = 0; f < nf; ++f) {
    const double* blk = &hm.stencil_blocks[size_t(hm.facet_stencil[f]) * 5 * nl * nl];
    int64_t nb[5] = {f, hm.facet_nbr[f * 4], hm.facet_nbr[f * 4 + 1], hm.facet_nbr[f * 4 + 2], hm.facet_nbr[f * 4 + 3]};
    for (int i = 0; i < bs; ++i) {
      double v = 0.0;
      for (int b = 0; b < 5; ++b)
        for (int j = 0; j < bs; ++j) v += blk[(size_t(b) * nl + i) * nl + j] * x[nb[b] * bs + j];
      y[f * bs + i] = v;
    }
  }
}

void csr_apply(const CsrHost& A, const double* x, double* y) {
  for (int i = 0; i < A.n_rows; ++i) {
    double v = 0.0;
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) v += A.v[p] * x[A.ci[p]];
    y[i] = v;
  }
}

void level_apply(const HostMesh& hm, const MLHostLevel& L, const double* x, double* y) {
  if (L.stencil) stencil_apply(hm, L.bs, x, y);
  else csr_apply(L.A, x, y);
}

// y = B x: the block-Jacobi inverse of the level
void level_binv(const HostMesh& hm, const MLHostLevel& L, const double* x, double* y) {
  if (!L.stencil) {
    for (int i = 0; i < L.n; ++i) y[i] = L.binv[i] * x[i];
    return;
  }
  const int bs = L.bs;
  for (int f = 0; f < L.n; ++f) {
    const double* B = &L.binv[size_t(hm.facet_stencil[f]) * bs * bs];
    for (int i = 0; i < bs; ++i) {
      double v = 0.0;
      for (int j = 0; j < bs; ++j) v += B[i * bs + j] * x[size_t(f) * bs + j];
      y[size_t(f) * bs + i] = v;
    }
  }
}

// Largest eigenvalue of B A by Lanczos: the coefficients of `its` preconditioned CG steps
// on A x = b (b pseudo-random) form the Lanczos tridiagonal matrix, whose largest
// eigenvalue approaches lambda_max(B A) from below.
template <typename FA, typename FB>
double lanczos_lmax(int n, FA applyA, FB applyB, int its) {
  Vec r(n), z(n), p(n), q(n);
  uint64_t s = 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < n; ++i) {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    r[i] = double(int64_t(s >> 11) % 2000001 - 1000000) * 1e-6;
  }
  applyB(r.data(), z.data());
  p = z;
  double rz = dot(r, z);
  std::vector<double> al, be;
  for (int it = 0; it < its && rz > 0.0; ++it) {
    applyA(p.data(), q.data());
    const double pq = dot(p, q);
    if (!(pq > 0.0)) break;
    const double a = rz / pq;
    for (int i = 0; i < n; ++i) r[i] -= a * q[i];
    applyB(r.data(), z.data());
    const double rz2 = dot(r, z);
    const double b = rz2 / rz;
    al.push_back(a);
    be.push_back(b);
    for (int i = 0; i < n; ++i) p[i] = z[i] + b * p[i];
    rz = rz2;
    if (!(rz > 0.0)) break;
  }
  const int m = int(al.size());
  if (m == 0) return 1.0;
  Vec T(size_t(m) * m, 0.0), ev, V;
  for (int i = 0; i < m; ++i) {
    T[size_t(i) * m + i] = 1.0 / al[i] + (i > 0 ? be[i - 1] / al[i - 1] : 0.0);
    if (i + 1 < m) {
      const double o = std::sqrt(be[i]) / al[i];
      T[size_t(i) * m + i + 1] = o;
      T[size_t(i + 1) * m + i] = o;
    }
  }
  symmetric_eigen(T, m, ev, V);
  return *std::max_element(ev.begin(), ev.end());
}

void set_chebyshev(MLHostLevel& L) {
  const double a = 0.25 * L.lmax, b = 1.1 * L.lmax;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
  const double sigma = theta / delta, rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
  L.cheb[0] = 1.0 / theta;
  L.cheb[1] = rho1 * rho0;
  L.cheb[2] = 2.0 * rho1 / delta;
}

// ---- sparse matrices

CsrHost transpose(const CsrHost& A) {
  CsrHost T;
  T.n_rows = A.n_cols;
  T.n_cols = A.n_rows;
  T.rp.assign(T.n_rows + 1, 0);
  for (int32_t c : A.ci) T.rp[c + 1]++;
  for (int i = 0; i < T.n_rows; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int32_t> pos(T.rp.begin(), T.rp.end() - 1);
  for (int i = 0; i < A.n_rows; ++i)
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int q = pos[A.ci[p]]++;
      T.ci[q] = i;
      T.v[q] = A.v[p];
    }
  return T;
}

// C = A B (Gustavson, row by row, columns in order of first appearance)
CsrHost spgemm(const CsrHost& A, const CsrHost& B) {
  CsrHost C;
  C.n_rows = A.n_rows;
  C.n_cols = B.n_cols;
  C.rp.assign(C.n_rows + 1, 0);
  std::vector<int32_t> mark(B.n_cols, -1);
  Vec acc(B.n_cols, 0.0);
  std::vector<int32_t> cols;
  for (int i = 0; i < A.n_rows; ++i) {
    cols.clear();
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int k = A.ci[p];
      const double a = A.v[p];
      for (int q = B.rp[k]; q < B.rp[k + 1]; ++q) {
        const int j = B.ci[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.v[q];
      }
    }
    for (int j : cols) {
      C.ci.push_back(j);
      C.v.push_back(acc[j]);
    }
    C.rp[i + 1] = int32_t(C.ci.size());
  }
  return C;
}

// The mode-0 (facet-constant) operator as a CSR matrix (duplicate columns merged: wall rows
// point their empty slots at themselves with zero blocks).
CsrHost mode0_matrix(const HostMesh& hm) {
  const int nl = hm.nl;
  const int nf = int(hm.topo.n_facet);
  CsrHost A;
  A.n_rows = A.n_cols = nf;
  A.rp.assign(nf + 1, 0);
  for (int f = 0; f < nf; ++f) {
    const double* blk = &hm.stencil_blocks[size_t(hm.facet_stencil[f]) * 5 * nl * nl];
    int32_t nb[5] = {f, hm.facet_nbr[size_t(f) * 4], hm.facet_nbr[size_t(f) * 4 + 1], hm.facet_nbr[size_t(f) * 4 + 2],
                     hm.facet_nbr[size_t(f) * 4 + 3]};
    const size_t start = A.ci.size();
    for (int b = 0; b < 5; ++b) {
      const double v = blk[size_t(b) * nl * nl];
      size_t q = start;
      while (q < A.ci.size() && A.ci[q] != nb[b]) ++q;
      if (q == A.ci.size()) {
        A.ci.push_back(nb[b]);
        A.v.push_back(v);
      } else {
        A.v[q] += v;
      }
    }
    A.rp[f + 1] = int32_t(A.ci.size());
  }
  return A;
}

// Smoothed-aggregation transfer for a scalar operator A with near-null vector nn: returns P
// (and the next level's near-null vector in nn_next).
CsrHost sa_prolongator(const CsrHost& A, const Vec& nn, Vec& nn_next) {
  const int n = A.n_rows;
  const double theta = 0.08;
  Vec d(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (A.ci[p] == i) d[i] += A.v[p];
  // strong connections
  std::vector<int32_t> srp(n + 1, 0), sci;
  for (int i = 0; i < n; ++i) {
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int j = A.ci[p];
      if (j != i && std::fabs(A.v[p]) >= theta * std::sqrt(std::fabs(d[i] * d[j]))) sci.push_back(j);
    }
    srp[i + 1] = int32_t(sci.size());
  }
  // isolated rows (no nonzero off the diagonal: the identity rows of outflow facets) join no
  // aggregate; their rows of P are empty, the smoother solves them exactly
  std::vector<char> isolated(n, 1);
  for (int i = 0; i < n; ++i)
    for (int p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (A.ci[p] != i && A.v[p] != 0.0) isolated[i] = 0;
  // aggregation: a node whose strong neighbours are all free starts an aggregate with them;
  // then every free node joins the aggregate of a strong neighbour, or starts its own
  std::vector<int32_t> agg(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0 || isolated[i]) continue;
    bool free = true;
    for (int p = srp[i]; p < srp[i + 1] && free; ++p) free = agg[sci[p]] < 0;
    if (!free) continue;
    agg[i] = na;
    for (int p = srp[i]; p < srp[i + 1]; ++p) agg[sci[p]] = na;
    ++na;
  }
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0 || isolated[i]) continue;
    for (int p = srp[i]; p < srp[i + 1]; ++p)
      if (agg[sci[p]] >= 0) {
        agg[i] = agg[sci[p]];
        break;
      }
    if (agg[i] < 0) agg[i] = na++;
  }
  // tentative prolongator: the near-null vector restricted to each aggregate, normalised
  nn_next.assign(na, 0.0);
  for (int i = 0; i < n; ++i)
    if (agg[i] >= 0) nn_next[agg[i]] += nn[i] * nn[i];
  for (double& v : nn_next) v = std::sqrt(v);
  CsrHost P0;
  P0.n_rows = n;
  P0.n_cols = na;
  P0.rp.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) {
      P0.ci.push_back(agg[i]);
      P0.v.push_back(nn_next[agg[i]] > 0.0 ? nn[i] / nn_next[agg[i]] : 0.0);
    }
    P0.rp[i + 1] = int32_t(P0.ci.size());
  }
  // smoothed prolongator P = (I - omega D^-1 A) P0, omega = 4 / (3 rho(D^-1 A))
  auto aA = [&](const double* x, double* y) { csr_apply(A, x, y); };
  auto aD = [&](const double* x, double* y) {
    for (int i = 0; i < n; ++i) y[i] = x[i] / d[i];
  };
  const double rho = 1.1 * lanczos_lmax(n, aA, aD, 20);
  const double omega = 4.0 / (3.0 * rho);
  CsrHost AP = spgemm(A, P0);
  CsrHost P;
  P.n_rows = n;
  P.n_cols = na;
  P.rp.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    // row i of P0 (one entry, none for an isolated row) minus omega / d_i times row i of A P0
    const size_t start = P.ci.size();
    for (int p = P0.rp[i]; p < P0.rp[i + 1]; ++p) {
      P.ci.push_back(P0.ci[p]);
      P.v.push_back(P0.v[p]);
    }
    for (int p = AP.rp[i]; p < AP.rp[i + 1]; ++p) {
      const double v = -omega / d[i] * AP.v[p];
      size_t q = start;
      while (q < P.ci.size() && P.ci[q] != AP.ci[p]) ++q;
      if (q == P.ci.size()) {
        P.ci.push_back(AP.ci[p]);
        P.v.push_back(v);
      } else {
        P.v[q] += v;
      }
    }
    P.rp[i + 1] = int32_t(P.ci.size());
  }
  return P;
}

bool invert_small(std::vector<double>& A, int n) {
  // Gauss-Jordan with partial pivoting on a row-major n x n matrix
  std::vector<double> I(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) I[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[size_t(r) * n + c]) > std::fabs(A[size_t(piv) * n + c])) piv = r;
    if (A[size_t(piv) * n + c] == 0.0) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(A[size_t(c) * n + j], A[size_t(piv) * n + j]);
      std::swap(I[size_t(c) * n + j], I[size_t(piv) * n + j]);
    }
    const double inv = 1.0 / A[size_t(c) * n + c];
    for (int j = 0; j < n; ++j) {
      A[size_t(c) * n + j] *= inv;
      I[size_t(c) * n + j] *= inv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[size_t(r) * n + c];
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

// Chebyshev(2) smoothing of A x = b: from x = 0 (x0 == nullptr) or from x0, result in x.
void smooth(const HostMesh& hm, const MLHostLevel& L, const double* b, const double* x0, double* x) {
  const size_t n = size_t(L.n) * L.bs;
  Vec res(n), d(n), t(n);
  if (x0) {
    level_apply(hm, L, x0, t.data());
    for (size_t i = 0; i < n; ++i) res[i] = b[i] - t[i];
  } else {
    std::copy(b, b + n, res.begin());
  }
  level_binv(hm, L, res.data(), t.data());
  for (size_t i = 0; i < n; ++i) {
    d[i] = L.cheb[0] * t[i];
    x[i] = (x0 ? x0[i] : 0.0) + d[i];
  }
  level_apply(hm, L, d.data(), t.data());
  for (size_t i = 0; i < n; ++i) res[i] -= t[i];
  level_binv(hm, L, res.data(), t.data());
  for (size_t i = 0; i < n; ++i) x[i] += L.cheb[1] * d[i] + L.cheb[2] * t[i];
}

void vcycle(const HostMesh& hm, const MLHost& ml, size_t l, const double* b, double* x) {
  if (l == ml.lv.size()) {
    for (int i = 0; i < ml.nc; ++i) {
      double v = 0.0;
      for (int j = 0; j < ml.nc; ++j) v += ml.cpinv[size_t(i) * ml.nc + j] * b[j];
      x[i] = v;
    }
    return;
  }
  const MLHostLevel& L = ml.lv[l];
  const size_t n = size_t(L.n) * L.bs, nn = size_t(L.n_next) * L.bs_next;
  smooth(hm, L, b, nullptr, x);
  Vec r(n), bn(nn), xn(nn);
  level_apply(hm, L, x, r.data());
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
  if (L.inject) {
    for (int f = 0; f < L.n; ++f)
      for (int j = 0; j < L.bs_next; ++j) bn[size_t(f) * L.bs_next + j] = r[size_t(f) * L.bs + j];
  } else {
    csr_apply(L.R, r.data(), bn.data());
  }
  vcycle(hm, ml, l + 1, bn.data(), xn.data());
  Vec x1(x, x + n);
  if (L.inject) {
    for (int f = 0; f < L.n; ++f)
      for (int j = 0; j < L.bs_next; ++j) x1[size_t(f) * L.bs + j] += xn[size_t(f) * L.bs_next + j];
  } else {
    Vec px(n);
    csr_apply(L.P, xn.data(), px.data());
    for (size_t i = 0; i < n; ++i) x1[i] += px[i];
  }
  smooth(hm, L, b, x1.data(), x);
}

// Pseudo-inverse of the coarsest operator A (symmetric positive semi-definite, nc rows), dense,
// symmetrised. Up to 256 rows: from its eigen-decomposition, the eigenvalues below 1e-10 of the
// largest dropped. Larger (the Jacobi eigensolver's cost grows as nc^3 per sweep): when the
// near-null vector v is in the kernel (|A v| <= 1e-9 |A|_F |v|, a closed mesh), through the
// definite matrix B = A + s u u^T (u = v / |v|, s the mean diagonal entry), whose inverse is
// A^+ + u u^T / s, so that A^+ = B^-1 - u u^T / s; otherwise (A definite) A^-1. Both by
// Gauss-Jordan elimination with partial pivoting. Returns false if the matrix is singular.
bool coarse_pinv(const CsrHost& A, const Vec& v, Vec& out) {
  const int nc = A.n_rows;
  Vec D(size_t(nc) * nc, 0.0);
  for (int r = 0; r < nc; ++r)
    for (int p = A.rp[r]; p < A.rp[r + 1]; ++p) D[size_t(r) * nc + A.ci[p]] += A.v[p];
  for (int r = 0; r < nc; ++r)
    for (int c = r + 1; c < nc; ++c) {
      const double h = 0.5 * (D[size_t(r) * nc + c] + D[size_t(c) * nc + r]);
      D[size_t(r) * nc + c] = D[size_t(c) * nc + r] = h;
    }
  out.assign(size_t(nc) * nc, 0.0);
  if (nc <= 256) {
    Vec ev, V;
    symmetric_eigen(D, nc, ev, V);
    double emax = 0.0;
    for (double e : ev) emax = std::max(emax, std::fabs(e));
    for (int i = 0; i < nc; ++i) {
      if (!(ev[i] > 1e-10 * emax)) continue;
      const double inv = 1.0 / ev[i];
      for (int r = 0; r < nc; ++r)
        for (int c = 0; c < nc; ++c) out[size_t(r) * nc + c] += V[size_t(r) * nc + i] * inv * V[size_t(c) * nc + i];
    }
    return true;
  }
  double fro = 0.0, vv = 0.0, avv = 0.0, tr = 0.0;
  for (double x : D) fro += x * x;
  for (int r = 0; r < nc; ++r) {
    double y = 0.0;
    for (int c = 0; c < nc; ++c) y += D[size_t(r) * nc + c] * v[c];
    avv += y * y;
    vv += v[r] * v[r];
    tr += D[size_t(r) * nc + r];
  }
  const bool kernel = vv > 0.0 && std::sqrt(avv) <= 1e-9 * std::sqrt(fro) * std::sqrt(vv);
  const double s = tr / nc;
  if (kernel)
    for (int r = 0; r < nc; ++r)
      for (int c = 0; c < nc; ++c) D[size_t(r) * nc + c] += s * v[r] * v[c] / vv;
  if (!host_invert(D, nc)) return false;
  for (int r = 0; r < nc; ++r)
    for (int c = 0; c < nc; ++c) {
      double x = 0.5 * (D[size_t(r) * nc + c] + D[size_t(c) * nc + r]);
      if (kernel) x -= v[r] * v[c] / (vv * s);
      out[size_t(r) * nc + c] = x;
    }
  return true;
}

}  // namespace

int build_multilevel(const HostMesh& hm, MLHost& ml, std::string& err) {
  ml = MLHost();
  const int nl = hm.nl, nf = int(hm.topo.n_facet);
  // p-levels: k+1 modes, then 2 (k >= 2), then 1
  std::vector<int> modes = {nl};
  if (nl > 2) modes.push_back(2);
  if (nl > 1) modes.push_back(1);
  CsrHost A0 = mode0_matrix(hm);
  const bool mode0_coarsest = nf <= kMLCoarseMax;
  for (size_t i = 0; i < modes.size(); ++i) {
    const int bs = modes[i];
    if (bs == 1 && mode0_coarsest) break;   // the mode-0 operator is the coarsest level itself
    MLHostLevel L;
    L.stencil = true;
    L.bs = bs;
    L.n = nf;
    L.binv.resize(size_t(hm.n_stencil) * bs * bs);
    for (int s = 0; s < hm.n_stencil; ++s) {
      std::vector<double> B(size_t(bs) * bs);
      for (int a = 0; a < bs; ++a)
        for (int c = 0; c < bs; ++c) B[size_t(a) * bs + c] = hm.stencil_blocks[(size_t(s) * 5 * nl + a) * nl + c];
      if (!invert_small(B, bs)) {
        err = "multilevel: singular facet sub-block";
        return DG_ERR_MESH;
      }
      std::copy(B.begin(), B.end(), L.binv.begin() + size_t(s) * bs * bs);
    }
    L.inject = bs > 1;
    L.n_next = nf;
    L.bs_next = bs > 1 ? modes[i + 1] : 1;
    ml.lv.push_back(std::move(L));
  }
  // h-levels on the mode-0 operator
  CsrHost A = A0;
  Vec nn(nf, 1.0), nn_next;
  if (!mode0_coarsest) {
    while (A.n_rows > kMLCoarseMax && int(ml.lv.size()) < kMLMaxLevels) {
      CsrHost P = sa_prolongator(A, nn, nn_next);
      if (P.n_cols >= A.n_rows) break;   // no coarsening
      CsrHost R = transpose(P);
      CsrHost Ac = spgemm(R, spgemm(A, P));
      MLHostLevel& last = ml.lv.back();
      if (last.stencil && last.bs == 1 && last.P.n_rows == 0) {
        last.P = P;
        last.R = R;
        last.inject = false;
        last.n_next = P.n_cols;
      } else {
        MLHostLevel L;
        L.stencil = false;
        L.bs = 1;
        L.n = A.n_rows;
        L.A = A;
        L.binv.resize(L.n);
        for (int r = 0; r < L.n; ++r) {
          double dd = 0.0;
          for (int p = A.rp[r]; p < A.rp[r + 1]; ++p)
            if (A.ci[p] == r) dd += A.v[p];
          L.binv[r] = 1.0 / dd;
        }
        L.P = P;
        L.R = R;
        L.n_next = P.n_cols;
        ml.lv.push_back(std::move(L));
      }
      A = std::move(Ac);
      nn.swap(nn_next);
    }
  }
  // aggregation made no progress on the mode-0 operator: it is the coarsest level itself
  if (!ml.lv.empty() && ml.lv.back().stencil && ml.lv.back().bs == 1 && ml.lv.back().P.n_rows == 0) ml.lv.pop_back();
  // coarsest: pseudo-inverse of the remaining operator (coarse_pinv)
  const int nc = A.n_rows;
  if (nc > 4 * kMLCoarseMax) {
    err = "multilevel: coarsening stalled";
    return DG_ERR_UNSUPPORTED;
  }
  ml.nc = nc;
  if (!coarse_pinv(A, nn, ml.cpinv)) {
    err = "multilevel: singular coarsest operator";
    return DG_ERR_MESH;
  }
  if (!ml.lv.empty()) {
    ml.lv.back().n_next = nc;
    if (ml.lv.back().inject) ml.lv.back().bs_next = 1;
  }
  // Chebyshev intervals
  for (MLHostLevel& L : ml.lv) {
    const int n = L.n * L.bs;
    auto aA = [&](const double* x, double* y) { level_apply(hm, L, x, y); };
    auto aB = [&](const double* x, double* y) { level_binv(hm, L, x, y); };
    L.lmax = lanczos_lmax(n, aA, aB, 30);
    set_chebyshev(L);
  }
  return DG_OK;
}

CsrHost stencil_csr(int n, int nl, int nb, const int32_t* cls, const int32_t* nbr, const double* blocks) {
  CsrHost A;
  A.n_rows = A.n_cols = n * nl;
  A.rp.assign(size_t(n) * nl + 1, 0);
  std::vector<int32_t> cols;
  std::vector<double> vals;
  for (int f = 0; f < n; ++f) {
    const double* blk = blocks + size_t(cls[f]) * (1 + nb) * nl * nl;
    for (int i = 0; i < nl; ++i) {
      cols.clear();
      vals.clear();
      for (int b = 0; b <= nb; ++b) {
        const int g = b == 0 ? f : nbr[size_t(f) * nb + b - 1];
        for (int j = 0; j < nl; ++j) {
          const int c = g * nl + j;
          const double v = blk[(size_t(b) * nl + i) * nl + j];
          size_t q = 0;
          while (q < cols.size() && cols[q] != c) ++q;
          if (q == cols.size()) {
            cols.push_back(c);
            vals.push_back(v);
          } else {
            vals[q] += v;
          }
        }
      }
      A.ci.insert(A.ci.end(), cols.begin(), cols.end());
      A.v.insert(A.v.end(), vals.begin(), vals.end());
      A.rp[size_t(f) * nl + i + 1] = int32_t(A.ci.size());
    }
  }
  return A;
}

int build_multilevel_csr(const CsrHost& A0, int nl, const int32_t* cls, const std::vector<double>* cls_binv,
                         MLHost& ml, std::string& err) {
  ml = MLHost();
  if (A0.n_rows % nl) {
    err = "multilevel: operator size is not a multiple of the modes per face";
    return DG_ERR_INVALID_ARG;
  }
  const int nf = A0.n_rows / nl;
  auto diag_inv = [](const CsrHost& A) {
    std::vector<double> d(A.n_rows, 0.0);
    for (int r = 0; r < A.n_rows; ++r)
      for (int p = A.rp[r]; p < A.rp[r + 1]; ++p)
        if (A.ci[p] == r) d[r] += A.v[p];
    for (double& v : d) v = 1.0 / v;
    return d;
  };
  // injection of the face-constant multipliers (mode 0 of every face)
  CsrHost Pm;
  Pm.n_rows = A0.n_rows;
  Pm.n_cols = nf;
  Pm.rp.assign(A0.n_rows + 1, 0);
  for (int i = 0; i < A0.n_rows; ++i) {
    if (i % nl == 0) {
      Pm.ci.push_back(i / nl);
      Pm.v.push_back(1.0);
    }
    Pm.rp[i + 1] = int32_t(Pm.ci.size());
  }
  const CsrHost Rm = transpose(Pm);
  CsrHost A = spgemm(Rm, spgemm(A0, Pm));   // the mode-0 operator
  // level 0: all modes; block Jacobi on the face stencil (cls given) or point Jacobi on the CSR rows
  {
    MLHostLevel L0;
    L0.n_next = nf;
    if (cls) {
      L0.stencil = true;
      L0.bs = nl;
      L0.n = nf;
      L0.binv = *cls_binv;
      L0.inject = true;
      L0.bs_next = 1;
    } else {
      L0.stencil = false;
      L0.bs = 1;
      L0.n = A0.n_rows;
      L0.A = A0;
      L0.binv = diag_inv(A0);
      L0.P = Pm;
      L0.R = Rm;
    }
    auto aA = [&](const double* x, double* y) { csr_apply(A0, x, y); };
    auto aB = [&](const double* x, double* y) {
      if (!cls) {
        for (int i = 0; i < A0.n_rows; ++i) y[i] = L0.binv[i] * x[i];
        return;
      }
      for (int f = 0; f < nf; ++f) {
        const double* B = &(*cls_binv)[size_t(cls[f]) * nl * nl];
        for (int a = 0; a < nl; ++a) {
          double v = 0.0;
          for (int c = 0; c < nl; ++c) v += B[a * nl + c] * x[size_t(f) * nl + c];
          y[size_t(f) * nl + a] = v;
        }
      }
    };
    L0.lmax = lanczos_lmax(A0.n_rows, aA, aB, 30);
    set_chebyshev(L0);
    ml.lv.push_back(std::move(L0));
  }
  // h-levels: smoothed aggregation on the mode-0 operator
  Vec nn(nf, 1.0), nn_next;
  while (A.n_rows > kMLCoarseMax && int(ml.lv.size()) < kMLMaxLevels) {
    CsrHost P = sa_prolongator(A, nn, nn_next);
    if (P.n_cols >= A.n_rows) break;
    MLHostLevel L;
    L.stencil = false;
    L.bs = 1;
    L.n = A.n_rows;
    L.binv = diag_inv(A);
    L.R = transpose(P);
    L.n_next = P.n_cols;
    CsrHost Ac = spgemm(L.R, spgemm(A, P));
    L.A = std::move(A);
    L.P = std::move(P);
    const HostMesh none;
    auto aA = [&](const double* x, double* y) { level_apply(none, L, x, y); };
    auto aB = [&](const double* x, double* y) { level_binv(none, L, x, y); };
    L.lmax = lanczos_lmax(L.n, aA, aB, 30);
    set_chebyshev(L);
    ml.lv.push_back(std::move(L));
    A = std::move(Ac);
    nn.swap(nn_next);
  }
  const int nc = A.n_rows;
  if (nc > 4 * kMLCoarseMax) {
    err = "multilevel: coarsening stalled";
    return DG_ERR_UNSUPPORTED;
  }
  ml.nc = nc;
  if (!coarse_pinv(A, nn, ml.cpinv)) {
    err = "multilevel: singular coarsest operator";
    return DG_ERR_MESH;
  }
  ml.lv.back().n_next = nc;
  return DG_OK;
}

void multilevel_apply_host(const HostMesh& hm, const MLHost& ml, const double* r, double* z) {
  vcycle(hm, ml, 0, r, z);
}

}  // namespace dgdf
