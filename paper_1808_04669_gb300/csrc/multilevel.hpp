// Multilevel preconditioner for the condensed facet system S lam = g of eq. (12)
// (Sec. 2.4) on meshes without the lattice structure (walls, perturbed or
// unstructured meshes), built once per mesh on the host. The paper factorises
// this system directly (Sec. 4); here it is solved by PCG, and block Jacobi
// alone needs O(1/h) iterations.
//
// Levels (finest first):
//   p-levels on the facet space: all k+1 Legendre modes of each facet, then modes
//   {0, 1} (k >= 2), then mode 0 (the facet-constant multipliers). Each is the
//   facet stencil of S restricted to its leading modes (the Galerkin operator of
//   the injection), applied matrix-free; transfers keep or add the leading modes.
//   h-levels: smoothed aggregation on the mode-0 operator (a zero-row-sum M-matrix:
//   its kernel is the constant multiplier). Aggregates from strong connections,
//   tentative prolongator from the near-null vector carried down the levels (so
//   the kernel stays exact on every level), one Jacobi smoothing step of the
//   prolongator, Galerkin coarse operators R A P with R = P^T.
//   The coarsest operator (<= kMLCoarseMax rows) is applied through its dense
//   pseudo-inverse (one grid-wide phase, where every further level would take
//   four or five).
// Smoothing: Chebyshev polynomials of degree 2 in B A with B the block-Jacobi
// inverse, on [lmax / 4, 1.1 lmax], lmax estimated by Lanczos (from CG
// coefficients). Pre- and post-smoothing use the same polynomial, so one V-cycle
// is a symmetric positive semi-definite preconditioner.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "setup.hpp"

namespace dgdf {

constexpr int kMLMaxLevels = 16;
constexpr int kMLCoarseMax = 1024;

struct CsrHost {
  int n_rows = 0, n_cols = 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> v;
};

struct MLHostLevel {
  bool stencil = false;       // operator: the facet stencil on the first bs modes (else the CSR matrix A)
  int bs = 1;                 // values per row
  int n = 0;                  // rows (facets on stencil levels)
  std::vector<double> binv;   // stencil: [n_stencil][bs][bs] inverses of the own sub-blocks; CSR: [n] 1 / a_ii
  CsrHost A;                  // CSR levels
  bool inject = false;        // transfer to the next level keeps its leading modes (facet rows on both)
  CsrHost P, R;               // otherwise: prolongation [n x n_next] and restriction R = P^T
  int n_next = 0, bs_next = 1;
  double lmax = 0.0;          // estimate of the largest eigenvalue of B A
  double cheb[3] = {0, 0, 0}; // Chebyshev(2) coefficients c0 = 1 / theta, c1 = rho1 rho0, c2 = 2 rho1 / delta
};

struct MLHost {
  std::vector<MLHostLevel> lv;   // smoothing levels, finest first
  int nc = 0;                    // rows of the coarsest level
  std::vector<double> cpinv;     // [nc][nc] pseudo-inverse of the coarsest operator
};

// Builds the hierarchy from hm's facet stencil. Returns 0 or a dg_status code.
int build_multilevel(const HostMesh& hm, MLHost& ml, std::string& err);

// The same hierarchy from an assembled operator A0 (CSR, nl values per face, face-major): level 0
// keeps all modes and transfers to the face-constant multipliers (mode 0) by injection, then
// smoothed aggregation as above with point-Jacobi smoothing. Level 0 smooths with block Jacobi
// on its face stencil when cls (stencil class per face) and cls_binv ([class][nl][nl] inverses of
// the own blocks) are given (a stencil level, applied by the device through the level's own
// stencil pointers; the host V-cycle does not take it), else with point Jacobi on the CSR rows.
// Used for the face system of the three-dimensional path.
int build_multilevel_csr(const CsrHost& A0, int nl, const int32_t* cls, const std::vector<double>* cls_binv,
                         MLHost& ml, std::string& err);

// A block stencil operator as CSR: row block f couples to itself and to nbr[f][0..nb) through
// blocks[cls[f]][1 + nb][nl][nl] (slot 0 its own block); duplicate columns are merged.
CsrHost stencil_csr(int n, int nl, int nb, const int32_t* cls, const int32_t* nbr, const double* blocks);

// z = M r for one V-cycle, on the host (the reference of the device kernel);
// r and z hold n_facet (k+1) values.
void multilevel_apply_host(const HostMesh& hm, const MLHost& ml, const double* r, double* z);

}  // namespace dgdf
