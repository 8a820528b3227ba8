// Device-side data of one closed tetrahedral mesh (the three-dimensional path, FP64) and the
// launch interface between api3.cu and k_tet.cu. Conventions: setup3.hpp.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "device.cuh"

namespace dgdf {

// Per-class geometry record (doubles): Jinv[9] row-major (d xi_r / d x_d), det = 6|T|,
// s = 1/sqrt(det), outward normals [4][3], face areas [4], face perm indices [4]; padded to 32.
constexpr int kGeo3 = 32;
enum Geo3Slot { G3_JINV = 0, G3_DET = 9, G3_S = 10, G3_NRM = 11, G3_AREA = 23, G3_PERM = 27 };

struct DevMesh3 {
  int k, ns, nd, nw, nl, nq, nqf;
  int n_tet, n_face, n_class, n_stencil;
  double nu;
  // reference tables: volume rule and basis [nq], [nq][ns], [nq][ns][3]; face rule [nqf];
  // basis at the face points per (local face, perm) [4][6][nqf][ns] and [4][6][nqf][ns][3];
  // lattice interpolation [ns][ns] and its inverse
  const double *vw, *vphi, *vdphi, *fw, *fphi, *fdphi, *lat_phi, *lat_inv;
  const double* geo;                  // [n_class][kGeo3]
  const double *P, *G;                // [n_class][nd][nd], [n_class][4 nl][nd]
  const double *W, *WC;               // pressure rows [n_class][nw][nd], [n_class][nw][4 nl]
  const double *plat_phi, *mu_lat;    // P^(k-1) basis at the (k-1)-lattice [nw][nw]; face basis
                                      // at the face's k-lattice [nl][nl]
  const int32_t *tet_class, *tet_nbr, *tet_face;
  const int8_t* tet_nbr_loc;
  const double* face_sigma;           // [n_face]
  const int32_t *face_tet, *face_nbr, *face_stencil;   // [n_face][2], [n_face][6], [n_face]
  const int8_t* face_loc;             // [n_face][2]
  const double *st_blk, *st_binv;     // [n_stencil][7][nl][nl], [n_stencil][nl][nl]
  double *u, *ustage, *h, *gl;        // [n_tet][nd] x3, [n_tet][4 nl]
  double *lam, *g, *r, *z, *pa, *pb, *q;   // [n_face][nl]
  double* red;                        // reduction scratch [kRedSlots][kMaxSolverBlocks]
  GridBar* bar;
  DevStats* stats;
  double* diag;                       // [4] energy, enstrophy, max |div u|, max |[u.n]|
};

bool tet_tables_match(int k, int nq, int nqf);   // host rule sizes equal the kernels' constants
cudaError_t launch_stage3(const DevMesh3& m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_recover3(const DevMesh3& m, double* out, cudaStream_t s);
cudaError_t launch_solve3(const DevMesh3& m, const SolveArgs& a, int nblocks, cudaStream_t s);
int solver3_blocks(const DevMesh3& m);
cudaError_t launch_lattice_to_coef3(const DevMesh3& m, const double* vals, double* coef, cudaStream_t s);
cudaError_t launch_coef_to_lattice3(const DevMesh3& m, const double* coef, double* vals, cudaStream_t s);
cudaError_t launch_diagnostics3(const DevMesh3& m, const double* coef, cudaStream_t s);
// Pressure from h = f (MODE_PRESSURE) and lam: pe [n_tet][nw] lattice values and pf [n_face][nl]
// (NULL: not written), shifted to a zero mean over the domain of volume vol; part holds
// pressure3_parts(m) doubles of scratch.
int pressure3_parts(const DevMesh3& m);
cudaError_t launch_pressure3(const DevMesh3& m, double* pe, double* pf, double* part, double vol, cudaStream_t s);
// FP64 PCG with the multilevel preconditioner of an assembled hierarchy (k_multilevel.cu): mv
// holds the hierarchy (ml_*), the PCG vectors r and z, red, bar and stats
int solver3_ml_blocks(const DevMesh3& m, bool fp32);   // fp32: the V-cycle in FP32 (mv.ml_lv_f)
cudaError_t launch_solve3_ml(const DevMesh3& m, const DevMesh& mv, const SolveArgs& a, int nblocks, cudaStream_t s);

}  // namespace dgdf
