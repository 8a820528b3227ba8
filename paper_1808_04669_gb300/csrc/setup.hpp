// Host-side FP64 set-up of libdgdf: topology, reference tables, element operators.
//
// Everything here runs once per mesh on the CPU (the hybrid-mixed matrix does
// not depend on dt, Remark 2, so its element blocks are precomputed) and is
// then uploaded. No CUDA in this translation unit.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dgdf {

constexpr int kMaxDegree = 3;

inline int n_lat(int m) { return (m + 1) * (m + 2) / 2; }

// Reference quadrature rules and the orthonormal (Dubiner) basis of P^k on the
// triangle {xi1, xi2 >= 0, xi1 + xi2 <= 1}, ordered by total degree so that the
// first n_lat(k-1) functions span P^{k-1}.
struct RefTables {
  int k = 0, ns = 0, nw = 0, nl = 0, nq = 0, nqf = 0;
  std::vector<double> vxi, vw;        // volume rule: [nq][2], [nq] (weights sum to 1/2)
  std::vector<double> vphi, vdphi;    // [nq][ns], [nq][ns][2]
  std::vector<double> ft, fw;         // facet rule on [0,1]: [nqf]
  std::vector<double> fphi, fdphi;    // local facet e, element-CCW point order: [3][nqf][ns], [3][nqf][ns][2]
  std::vector<double> lat_phi;        // basis at the k-lattice, [ns][ns] (row = point)
  std::vector<double> lat_inv;        // its inverse [ns][ns]
  std::vector<double> plat_phi;       // first nw functions at the (k-1)-lattice, [nw][nw]
  std::vector<double> mu_lat;         // facet basis mu_m at t = i/k, [k+1][nl]
};

// Operators of one element geometry class (elements equal up to translation).
struct ClassOps {
  double J[4];      // [v1-v0, v2-v0] as columns, row-major
  double Jinv[4];   // row-major, (J^-1)_{r d} = d xi_r / d x_d
  double det;       // 2 |T|
  double normal[3][2];
  double flen[3];
  std::vector<double> P;    // [nd][nd]    (A_T^-1)_uu: M-orthogonal projector onto ker D_T
  std::vector<double> G;    // [3nl][nd]   C_T P_T
  std::vector<double> S;    // [3nl][3nl]  C_T P_T C_T^T
  std::vector<double> W;    // [nw][nd]    (A_T^-1)_wu
  std::vector<double> WCt;  // [nw][3nl]   W_T C_T^T
};

struct Topology {
  int64_t n_tri = 0, n_facet = 0;
  std::vector<int32_t> tri_facet;   // [n_tri][3]
  std::vector<int8_t> tri_orient;   // [n_tri][3] +1 along canonical direction, -1 against
  std::vector<int32_t> facet_tri;   // [n_facet][2] first appearance first; -1: a wall's missing side
  std::vector<int8_t> facet_loc;    // [n_facet][2] (-1 likewise)
  int64_t n_boundary = 0;           // wall facets (one side)
};

// Split-square lattice structure of a translation-invariant periodic mesh: facets
// are (type, cell) with type = stencil class and cell in an N x N grid, and row
// (type, c) of the facet system couples to (type_b, c + delta_b) with offsets that
// do not depend on c, so S is block circulant. Its Fourier symbol S^(kappa) is a
// (3(k+1)) x (3(k+1)) Hermitian block per wavenumber; sinv holds its inverse
// (pseudo-inverse at kappa = 0, where the constant multiplier is the kernel).
struct Lattice {
  bool ok = false;
  std::string why;             // reason when not ok
  int N = 0, ntype = 0, C = 0; // cells per direction, facet types, components C = ntype * (k+1)
  std::vector<int32_t> facet_of;   // [ntype][N(j)][N(i)] -> facet id
  std::vector<double> sinv;        // [N(ki)][N(kj)][C][C][2] (re, im)
  // eigen form of the half spectrum (FP32 preconditioner): [N/2+1 (ki)][N (kj)][C*C + C][2]:
  // V[b][i] (component b of eigenvector i, unitary), then 1/eigenvalue i in the real slots
  std::vector<double> seig;
  std::vector<double> twiddle;     // [N][2] exp(-2 pi i t / N)
};

// kinds of boundary facets (Sec. 2.5, eq. (be)); interior facets are kWall
enum : int8_t { kWall = 0, kInflow = 1, kOutflow = 2 };

struct HostMesh {
  int k = 0, ns = 0, nd = 0, nw = 0, nl = 0;
  std::vector<int8_t> facet_kind;   // [n_facet]
  bool has_inflow = false, has_outflow = false;
  double alpha = 2.0;
  Topology topo;
  RefTables ref;
  std::vector<int32_t> tri_class;   // [n_tri]
  std::vector<ClassOps> classes;
  std::vector<int32_t> tri_nbr;     // [n_tri][3] neighbour across local facet e (-1: wall)
  std::vector<int8_t> tri_nbr_loc;  // [n_tri][3] the neighbour's local index of that facet (-1: wall)
  std::vector<double> facet_sigma;  // [n_facet] alpha k^2 / h_F, h_F = max diameter of the two triangles
  // Facet-system stencil: row F couples to itself and to the other two facets of
  // each adjacent triangle. Rows with equal blocks share a stencil class.
  std::vector<int32_t> facet_nbr;   // [n_facet][4]
  std::vector<int32_t> facet_stencil;   // [n_facet]
  std::vector<double> stencil_blocks;   // [n_stencil][5][nl][nl] (own, then the 4 neighbours)
  std::vector<double> stencil_binv;     // [n_stencil][nl][nl] inverse of the own block (block Jacobi)
  int n_stencil = 0;
  std::vector<int32_t> facet_side0;     // [n_facet] triangle on the stencil's first (canonical) side
  std::vector<int32_t> facet_ext;       // internal -> external (first-appearance) facet id; empty = identity
  double area_total = 0.0;
};

// Returns 0 or a dg_status code; message in err.
int build_topology(int64_t n_tri, const int64_t* vid, const double* X, Topology& topo, std::string& err);
// Points of the volume rule of degree 3k - 1 (fully symmetric rules; Dims<K>::NQ on the device).
constexpr int kVolumePoints(int k) { return k == 1 ? 3 : (k == 2 ? 7 : 16); }

int build_reference(int k, RefTables& ref, std::string& err);
// Inflow data of Sec. 2.5 from u_in at the k+1 equispaced points of every triangle edge
// (vals [n_tri][3][k+1][2], the triangle's counter-clockwise direction; read on inflow edges):
// uq [n_facet][nqf][2] = u_in at the facet rule's points in canonical order, dmom [n_facet][nl]
// = int_F mu_m (u_in.n) ds with the multiplier basis mu_m in the canonical parameter and n the
// outward normal. Zero on every other facet.
void inflow_data(const HostMesh& hm, const double* vals, std::vector<double>& uq, std::vector<double>& dmom);
// edge_kind: kind of every triangle edge [n_tri][3] (read on boundary edges) or NULL (walls)
int build_host_mesh(int64_t n_tri, const int64_t* vid, const double* X, int k, double alpha,
                    HostMesh& hm, std::string& err, const int8_t* edge_kind = nullptr);
// Detects the split-square lattice structure and computes the inverse Fourier symbol.
// eig_half: the eigen form of the half spectrum (seig) instead of the full inverse (sinv).
void build_lattice(const HostMesh& hm, const double* X, Lattice& lat, bool eig_half = false);
// Eigen-decomposition of a small dense symmetric matrix (row-major [n][n]) by cyclic Jacobi
// rotations: evals[i] and column i of evecs ([n][n], row-major).
void symmetric_eigen(const std::vector<double>& A, int n, std::vector<double>& evals, std::vector<double>& evecs);
// Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b on [-1,1] (n points, Golub-Welsch).
void host_gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
// In-place inverse of an n x n row-major matrix (partial pivoting); false if singular.
bool host_invert(std::vector<double>& A, int n);
// Renumbers the facets of a lattice mesh internally in (type, j, i) order, so that the
// facet-major vectors are the Fourier passes' row order; records the external ids.
void renumber_facets_lattice(HostMesh& hm, Lattice& lat);

}  // namespace dgdf
