// Device-side data of one mesh and the launch interface between api.cu and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace dgdf {

// Error bits the kernels set in DevStats::flags.
enum : int {
  kFlagNotConverged = 1,
  kFlagNonFinite = 2,
  kFlagBarrierTimeout = 4,
  kFlagEnergyGrowth = 8,
};

// Kinds of boundary facets (Sec. 2.5, eq. (be)); interior facets read as walls.
enum : int { kFacetWall = 0, kFacetInflow = 1, kFacetOutflow = 2 };

// Per-class geometry record (doubles): Jinv[4] row-major (d xi_r / d x_d),
// det = 2|T|, s = 1/sqrt(det), normal[3][2], flen[3], zint0 = integral of the
// constant basis function, cinv0 = coefficient of the constant 1 in the first
// basis function's scale; padded to 20.
constexpr int kGeo = 20;
enum GeoSlot { G_JINV = 0, G_DET = 4, G_S = 5, G_NRM = 6, G_FLEN = 12, G_ZINT0 = 15, G_CINV0 = 16 };

struct DevStats {
  int flags;
  int last_iters;
  long long total_iters;
  long long solves;
  double last_relres;
  int last_sweeps;
  int pad;
  long long total_sweeps;
  // failure-detection test hooks (dg_test_barrier_fault); zero = off
  unsigned long long spin_limit;   // polls before a grid barrier gives up (0: kBarrierSpinLimit)
  int skip_block;                  // 1 + the block that leaves at its first grid barrier without arriving
  int pad2;
};

// Grid-barrier state for the persistent solver kernel.
struct GridBar {
  unsigned int count;
  unsigned int gen;
};

// One smoothing level of the multilevel preconditioner (multilevel.hpp), in device memory, with
// its operators and vectors in the precision R of the V-cycle (FP64, or FP32 in the mixed form).
template <typename R>
struct MLLevelT {
  int stencil;        // 1: the facet stencil of S on the first bs modes; 0: the CSR matrix a_*
  int bs, n;          // values per row, rows
  int inject;         // 1: transfer to the next level keeps the leading bs_next modes (same facet rows)
  int n_next, bs_next;
  int modes;          // CSR level 0 of an assembled hierarchy: values per face (row i is mode i % modes);
                      // 0 or 1 otherwise
  const R* binv;      // stencil: [n_stencil][bs][bs]; CSR: [n] 1 / a_ii
  const int32_t *a_rp, *a_ci;
  const R* a_v;
  const int32_t *p_rp, *p_ci;   // prolongation [n x n_next] (CSR transfer)
  const R* p_v;
  const int32_t *r_rp, *r_ci;   // restriction [n_next x n]
  const R* r_v;
  R c0, c1, c2;       // Chebyshev(2) coefficients
  R *x, *b, *r, *d;   // work vectors [n * bs]
  // a stencil level with a stencil of its own (NULL st_nbr: the facet stencil of the mesh):
  // row i couples to itself and to st_nbr[i][0..st_nnb) through st_blk[st_cls[i]][1 + st_nnb][bs][bs]
  const int32_t *st_cls, *st_nbr;
  int st_nnb;
  const R* st_blk;
};
using MLLevelDev = MLLevelT<double>;

struct DevMesh {
  int k, ns, nd, nw, nl, nq, nqf;
  int n_tri, n_facet, n_class, n_stencil;
  double nu;
  double area_total;
  int elem_df;     // 1: element kernels in double-float (mixed form), 0: FP64
  // reference tables
  const double *vw, *vphi, *vdphi, *fw, *fphi, *fdphi;
  const double *lat_inv, *lat_phi, *plat_phi, *mu_lat;
  // element classes
  const double *geo;     // [n_class][kGeo]
  const double *P, *G, *W, *WCt;     // [n_class][...]
  const float2 *Pdf, *Gdf;           // P and G as double-float (hi, lo) pairs
  const int32_t *tri_class, *tri_nbr, *tri_facet;
  const int8_t *tri_nbr_loc, *tri_orient;
  const double *facet_sigma;
  // double-float images (mixed form): reference tables in SmemTables order, class
  // geometry [n_class][kGeo], penalty per facet
  const float2 *tab_df, *geo_df, *sigma_df;
  // meshes with at most kDnClasses geometry classes (NULL otherwise), for the paired
  // (FP32x2) stage kernel: ptab = reference tables and the normal derivatives of the basis
  // at the facet points per class, fdphi . (Jinv n_e), in the layout of PairTables<K>;
  // P2 [n_class][nd][nd/2] and G2 [n_class][3(k+1)][nd/2] (pairs of consecutive columns:
  // both leading words, then both trailing words)
  const float4 *ptab, *P2, *G2;
  int ptab_words;   // float4 words of ptab
  // facet-system stencil
  const int32_t *facet_nbr, *facet_stencil, *facet_tri;
  const int32_t *facet_ext;           // internal -> external facet id (NULL: identity)
  const int8_t *facet_loc;
  const double *st_blk, *st_binv;     // [n_stencil][5][nl][nl], [n_stencil][nl][nl]
  const float *st_blk_f, *st_binv_f;
  const float2* st_blk_df;            // stencil blocks in double-float (mixed lattice solver)
  // state and work arrays
  double *u, *ustage, *h, *gl;        // [n_tri][nd] x3, [n_tri][3 nl]
  // mixed form: double-float twins of u and u' (written with them by the recovery),
  // and the condensation outputs h = P f, gl = G f in double-float
  float2 *u_df, *ustage_df, *h_df, *gl_df;
  double *lam, *g, *r, *z, *pa, *pb, *q;   // [n_facet][nl]
  float *rf, *zf, *paf, *pbf, *qf, *xf;    // FP32 inner-solve vectors
  float2* lam_df;                     // mixed lattice solver: the multipliers in double-float,
                                      // facet stride lat_vs
  float2 *lv_g, *lv_r, *lv_q, *lv_p;  // mixed lattice solver vectors [n_facet][lat_vs]
  float* lv_z;
  int lat_vs;                         // facet stride of those vectors (k = 2: padded to 4)
  int lam_is_df;                      // 1: the last solve left lam in lam_df (recovery reads it)
  double *red;                        // reduction scratch [kRedSlots][max_blocks]
  // lattice (translation-invariant split-square) solver data
  int lat_N, lat_logn;              // cells per direction, log2 N
  int lat_bufsz;                    // complex elements of the shared-memory transform buffer
  int lat_grp;                      // rows per transform group (scratch of lat_grp rows)
  const int32_t* lat_facet_of;        // [3][N][N]
  const void* lat_sinv;               // [N/2+1][C(C+1)/2 (FP32) or C*C (FP64)][N] complex
  const double* lat_tw;               // [N][2]
  void* lat_x;                        // [C][N/2+1][N] complex work array
  void* lat_x2;                       // the same size: inverse halves of the split column pass
  int lat_split;                      // column pass split into even / odd wavenumbers
  int lat_tw2_off;                    // complex elements before the N/2 twiddles in shared memory
  // tensor-core recovery (k_recover_tc.cu; mixed form, at most two geometry classes): tiles
  // of 128 triangles of one class, the class operators [P, -G^T] as bf16 digit slices
  int tc_rec;                         // 1: the stage kernel writes f into h_df, the recovery is k_recover_tc
  int tc_tiles;
  const int32_t* tc_rows;             // [tc_tiles][128] triangle ids, -1 padding
  const int32_t* tc_tile_cls;         // [tc_tiles]
  const uint16_t* tc_b;               // [n_class][kTcSlices][NP][KP] bf16 bits, tile layout
  const int32_t* tc_ec;               // [n_class][NP] column exponents
  // multilevel preconditioner (NULL ml_lv and ml_lv_f: none). The V-cycle runs in FP64 (ml_lv,
  // ml_cpinv, ml_xc, ml_bc) or, in the mixed form, in FP32 (the _f twins; level 0 then has
  // vectors of its own, filled from and written back to the PCG vectors r and z)
  const MLLevelDev* ml_lv;            // [ml_nlev] in device memory
  const MLLevelT<float>* ml_lv_f;
  int ml_nlev, ml_nc;                 // smoothing levels, rows of the coarsest level
  const double* ml_cpinv;             // [ml_nc][ml_nc] pseudo-inverse of the coarsest operator
  double *ml_xc, *ml_bc;              // coarsest vectors
  const float* ml_cpinv_f;
  float *ml_xc_f, *ml_bc_f;
  double* ml_hist;                    // NULL, or [kMLHist][4] per-iteration history of the last
                                      // multilevel solve: relres, r.z, p.S p, alpha
  // inflow / outflow boundaries (Sec. 2.5, eq. (be)); facet_kind NULL: every boundary facet
  // is a wall
  const int8_t* facet_kind;           // [n_facet] kFacetWall / kFacetInflow / kFacetOutflow
  const double* inflow_q;             // [n_facet][nqf][2] u_in at the facet points, canonical order
  const double* inflow_d;             // [n_facet][nl] moments of u_in.n (outward) against the
                                      // multiplier basis, canonical orientation
  int has_kernel;                     // 1: S is singular by the constant multiplier (no outflow
                                      // facet); 0: outflow rows are identities and S is definite
  GridBar *bar;
  DevStats *stats;
  double *diag;                       // [8] diagnostics output
};

constexpr int kRedSlots = 8;
constexpr int kMLHist = 512;
constexpr int kDnClasses = 4;
constexpr int kMaxSolverBlocks = 2048;

// Stage kernel modes.
enum StageMode : int {
  MODE_STAGE = 0,      // f = a u^n + b u' + c L(u'), h = P f, gl = G f
  MODE_RESIDUAL = 1,   // h = L(u') (Riesz representer, no solve)
  MODE_PRESSURE = 2,   // h = f = L(u'), gl = G f
  MODE_PROJECT = 3,    // f = u', h = P f, gl = G f
};

struct StageArgs {
  int mode;
  double a, b, c;      // MODE_STAGE: f = a M u^n + b M u' + c L(u') (c carries the step size)
  const double* un;    // u^n
  const double* up;    // u'
  const float2* un_df;   // their double-float twins (mixed form)
  const float2* up_df;
};

struct SolveArgs {
  double warm_scale;   // lam0 = warm_scale * lam (0: cold start)
  double rtol;
  int maxit;
  int mixed;           // 1: FP32 PCG inside FP64 refinement
  double inner_rtol;   // relative tolerance of each inner FP32 solve
  int max_sweeps;
  int inner_maxit;     // iteration cap of each inner FP32 solve
  double floor_rtol;   // accepted relative residual once refinement stagnates at its rounding floor
  int homog;           // 1: u.n = 0 on inflow facets (no data moments subtracted from g)
  // lattice solver, warm start from the same stage of earlier steps (overrides warm_scale):
  // lam0 = c1 hist1 + c2 hist2 + c3 hist3 (hist2 read only if c2 != 0, hist3 only if
  // c3 != 0); the kernel then moves hist2 into hist3 (if hist3 is set) and hist1 into
  // hist2, and the caller stores the new lam in hist1. Layout of lam.
  void* hist1;
  void* hist2;
  void* hist3;
  double c1, c2, c3;
};

// Launchers (k dispatched at run time). Return the launch error.
cudaError_t launch_lattice_to_coef(const DevMesh& m, const double* vals, double* coef, cudaStream_t s);
cudaError_t launch_coef_to_lattice(const DevMesh& m, const double* coef, double* vals, cudaStream_t s);
cudaError_t launch_stage(const DevMesh& m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_stage_df(const DevMesh& m, const StageArgs& a, cudaStream_t s);
cudaError_t launch_recover_df(const DevMesh& m, double* out, float2* out_df, cudaStream_t s);
// out may be NULL in the mixed form (only the double-float twin is written)
cudaError_t launch_recover(const DevMesh& m, double* out, float2* out_df, cudaStream_t s);
// tensor-core recovery (tc_rec): u = [P, -G^T] [f; lam] per class tile
cudaError_t launch_recover_tc(const DevMesh& m, double* out, float2* out_df, cudaStream_t s);
int tc_dims(int k, int* kp, int* np);   // padded K and N of the tensor-core recovery for degree k
// z = alpha x + beta y over n entries: double-float (mixed form) or FP64; z may alias x
cudaError_t launch_axpby_df(const float2* x, const float2* y, float2* z, double alpha, double beta, long long n,
                            cudaStream_t s);
cudaError_t launch_axpby64(const double* x, const double* y, double* z, double alpha, double beta, long long n,
                           cudaStream_t s);
cudaError_t launch_to_dfl(const double* x, float2* y, long long n, cudaStream_t s);
cudaError_t launch_to_double(const float2* x, int sx, double* y, int ny, long long nrow, cudaStream_t s);
cudaError_t launch_pressure(const DevMesh& m, double* w, cudaStream_t s);
cudaError_t launch_pressure_lattice(const DevMesh& m, const double* w, double* pe, double* pf, cudaStream_t s);
cudaError_t launch_diagnostics(const DevMesh& m, const double* coef, cudaStream_t s);
cudaError_t launch_adjoint(const DevMesh& m, const double* u, const double* w, double* out, double cw, double cj,
                           int accumulate, double nu_coef, double* nu_acc, cudaStream_t s);
cudaError_t launch_check_finite(const double* v, long long n, int* flag, cudaStream_t s);
// Energy watchdog: E = sum of squares of the n coefficients (the L2 norm squared in the
// orthonormal basis); sets kFlagEnergyGrowth in st->flags when E > watch[0] (1 + tol) with
// watch[0] >= 0, then stores E in watch[0] and E / previous in watch[1]. watch holds
// 2 + kMaxSolverBlocks doubles (the tail takes the block partials).
cudaError_t launch_energy_watch(const double* u, long long n, double* watch, double tol, DevStats* st,
                                cudaStream_t s);
cudaError_t launch_solve(const DevMesh& m, const SolveArgs& a, int nblocks, cudaStream_t s);
// FP64 PCG with the multilevel preconditioner (k_multilevel.cu)
cudaError_t launch_solve_ml(const DevMesh& m, const SolveArgs& a, int nblocks, cudaStream_t s);
int solver_ml_blocks(const DevMesh& m);
cudaError_t launch_ml_apply(const DevMesh& m, const double* r, double* z, int nblocks, cudaStream_t s);
int solver_max_blocks(const DevMesh& m, int mixed);
size_t lattice_smem_bytes(int k, int N, int fp32, int grp);
bool lattice_split(int N);
size_t lattice_tw2_offset(int k, int N, int fp32, int grp);
int lattice_group_rows(int k, int N, int fp32);          // rows per transform group (0: no fit)
size_t lattice_symbol_elems(int k, int N, int fp32);   // complex entries of the stored inverse symbol
size_t lattice_spectrum_elems(int k, int N);   // complex entries of the spectrum work array
size_t lattice_buffer_elems(int k, int N, int fp32);
int lattice_blocks(int k, int N, int fp32);
cudaError_t launch_solve_lattice(const DevMesh& m, const SolveArgs& a, int nblocks, int fp32, cudaStream_t s);
long long noalloc_max_dofs();
cudaError_t solve_noalloc(int k, int n_facet, const int32_t* facet_nbr, const int32_t* stencil, const double* blocks,
                          const double* binv, const double* g, double* lam, double rtol, int maxit, cudaStream_t s,
                          DevStats* host_stats);

}  // namespace dgdf
