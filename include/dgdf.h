/*
 * dgdf.h - C ABI of the GB300 explicit divergence-free DG library (libdgdf).
 *
 * The library advances the incompressible Euler / Navier-Stokes equations with
 * the explicit divergence-free DG method of G. Fu, "An explicit divergence-free
 * DG method for incompressible flow" (arXiv:1808.04669):
 *   - velocity in the globally divergence-free subspace V_h^{k,-1} of the broken
 *     space [P^k(T)]^2 on a triangulation (Sec. 2.1, eq. (4d));
 *   - spatial operator L(u)(v) = -C_h(u;u,v) - B_h(u,v), the upwind convection
 *     form (Sec. 2.2, eq. (7)) plus the symmetric interior-penalty viscous form
 *     (Sec. 3, eq. (18));
 *   - SSP-RK3 in time (Sec. 2.3, eq. (8)); every stage inverts the mass matrix
 *     of V_h^{k,-1} as the hybrid-mixed Poisson solve of Sec. 2.4, eq. (12)
 *     (Theorem 2): element static condensation, a preconditioned CG solve of
 *     the SPD facet-multiplier system, element-local recovery.
 *
 * All compute runs in CUDA kernels on the current device (sm_103a). The host
 * does set-up only (topology, reference tables, element operators, once per
 * mesh, in FP64).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Mesh: n_tri counter-clockwise triangles. tri_vertex_ids[t][c] (int64) is the
 *   id of corner c after periodic identification; tri_coords[t][c][0..1]
 *   (double) are the unwrapped corner coordinates, so every triangle keeps its
 *   true shape next to a periodic seam. An edge shared by two triangles is an
 *   interior (or periodic) facet; an edge with one triangle is a wall, a
 *   free-slip boundary facet (the wall conditions of the Navier-Stokes system
 *   of Sec. 3: u.n = 0 and zero tangential stress). There the facet multiplier
 *   enforces u.n = 0 and L(u) has no term: the convective flux vanishes with
 *   u.n, and the SIPG form of eq. (18) sums over interior facets only. An edge
 *   with three or more triangles is DG_ERR_MESH. Inflow and outflow boundaries
 *   are not supported.
 * Local facet e of a triangle is the edge opposite corner e. Two edges are the
 *   same facet when they join the same identified vertices in the same
 *   canonical order and have equal edge vectors; the canonical direction of a
 *   facet is its edge vector d with d_x > 0, or d_x = 0 and d_y > 0. Facets
 *   are numbered in order of first appearance over (triangle, local facet).
 * Lattice values (the basis-free exchange format): a field of degree m on a
 *   triangle is given by its values at v0 + (i/m)(v1-v0) + (j/m)(v2-v0),
 *   j = 0..m, i = 0..m-j (j outer), n_lat(m) = (m+1)(m+2)/2 points; for m = 0
 *   the point is the centroid. Velocity: double [n_tri][n_lat(k)][2];
 *   element pressure: double [n_tri][n_lat(k-1)]; facet pressure: double
 *   [n_facet][k+1] at the equispaced points t = i/k, i = 0..k, along the
 *   canonical direction.
 * Memory: the library owns every device buffer inside a dg_mesh. Inputs are
 *   copied; outputs go to caller-allocated buffers. "on_device" = 1 means the
 *   pointer is device memory on the mesh's device, 0 host memory.
 * Streams: all work is enqueued on dg_params.cuda_stream (NULL = legacy
 *   default stream). Every call returns a dg_status and has finished its
 *   device work (the stream is synchronised) before returning, except where
 *   stated.
 * Errors: a negative dg_status; dg_last_error() gives a message (per thread).
 *   After DG_ERR_CUDA the mesh should be destroyed.
 */
#ifndef DGDF_H
#define DGDF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh;
typedef struct dg_batch dg_batch;

typedef enum {
  DG_OK = 0,
  DG_ERR_INVALID_ARG = -1,   /* bad pointer, size or parameter */
  DG_ERR_MESH = -2,          /* degenerate / clockwise triangle, inconsistent facet */
  DG_ERR_UNSUPPORTED = -3,   /* degree out of range, lattice structure absent where required */
  DG_ERR_CUDA = -4,          /* a CUDA runtime call failed */
  DG_ERR_NOT_CONVERGED = -5, /* a facet-system solve hit cg_maxit (state is still updated) */
  DG_ERR_NONFINITE = -6,     /* NaN/Inf in an input or in a solver residual */
  DG_ERR_OOM = -7,           /* device allocation failed */
  DG_ERR_UNSTABLE = -8       /* the energy watchdog saw ||u||^2 grow in a step (dg_set_energy_watchdog) */
} dg_status;

enum { DG_PRECISION_FP64 = 0, DG_PRECISION_MIXED = 1 };
enum { DG_PRECOND_AUTO = 0, DG_PRECOND_BLOCK_JACOBI = 1, DG_PRECOND_MULTILEVEL = 2 };
/* explicit time-stepping schemes of dg_step */
enum { DG_SCHEME_SSPRK3 = 0, DG_SCHEME_EULER = 1, DG_SCHEME_RK4 = 2 };

typedef struct {
  int k;              /* polynomial degree, 1 <= k <= 3 */
  double nu;          /* kinematic viscosity >= 0 (nu = 0: Euler) */
  double alpha;       /* SIPG penalty alpha of eq. (18); the paper uses 2 (Sec. 4) */
  int precision;      /* DG_PRECISION_FP64 or DG_PRECISION_MIXED (FP32 PCG inside FP64 refinement) */
  double cg_rtol;     /* facet solve stops at ||g - S lam||_2 <= cg_rtol ||g||_2 (<= 0: 1e-13) */
  int cg_maxit;       /* iteration cap per solve (<= 0: 20000) */
  void* cuda_stream;  /* cudaStream_t to enqueue on (NULL: default stream) */
  int precond;        /* DG_PRECOND_AUTO: on a translation-invariant split-square mesh (a torus,
                         no walls), precondition with the exact Fourier-space inverse of the
                         block-circulant facet operator (FP32 in the mixed form, FP64 in the FP64
                         form), else with the multilevel preconditioner;
                         DG_PRECOND_BLOCK_JACOBI: always block Jacobi (FP64 PCG, or FP32 PCG
                         inside FP64 refinement in the mixed form);
                         DG_PRECOND_MULTILEVEL: always the multilevel preconditioner: FP64 PCG
                         with one V-cycle per iteration over p-levels of the facet space (k+1,
                         2, 1 Legendre modes per facet) and smoothed aggregation on the
                         facet-constant multipliers, Chebyshev(2) block-Jacobi smoothing, set up
                         on the host at creation (dgdf_host.h, dg_host_multilevel) */
} dg_params;

/* Build a mesh: topology, reference tables and the per-element operators of
 * eq. (12) on the host in FP64 (Remark 2: the matrix does not depend on dt, so
 * it is set up once), then uploaded. State starts at zero.
 * n_tri >= 1; tri_vertex_ids int64 [n_tri][3]; tri_coords double [n_tri][3][2]
 * (both host memory). On success *out owns the mesh.
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_MESH, DG_ERR_UNSUPPORTED, DG_ERR_CUDA, DG_ERR_OOM. */
int dg_mesh_create(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords,
                   const dg_params* params, dg_mesh** out);

/* dg_mesh_create with the kinds of the boundary facets of Sec. 2.5, eq. (be).
 * edge_kind int8 [n_tri][3] (host memory; edge e of a triangle is the one opposite its
 * vertex e), read on boundary edges only: 0 wall (u.n = 0, the default of dg_mesh_create),
 * 1 inflow (u.n = u_in.n with the data of dg_set_inflow, zero until it is called), 2 outflow
 * (p = 0: the facet's multipliers are zero and u.n is free). On inflow and outflow facets the
 * convective flux of eq. (7) takes u.n as the average of the interior trace and the exterior
 * state (u_in on inflow, the interior trace on outflow) and the upwind value from the side
 * u.n leaves; the viscous form has no boundary terms (natural conditions on every boundary
 * facet). With an outflow facet the facet system is definite and the pressure is not shifted
 * to mean zero. NULL edge_kind: every boundary facet is a wall.
 * Errors: those of dg_mesh_create; DG_ERR_INVALID_ARG for a kind outside 0..2. */
int dg_mesh_create_ex(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords,
                      const int8_t* edge_kind, const dg_params* params, dg_mesh** out);

/* Inflow data u_in of Sec. 2.5 (eq. (be)) for a mesh with inflow facets: vals double
 * [n_tri][3][k+1][2] (host memory), the velocity at the k+1 equispaced points of every
 * triangle edge, from vertex (e+1) mod 3 to vertex (e+2) mod 3 of the triangle (its
 * counter-clockwise direction); read on inflow edges only, interpolated to the facet
 * quadrature points. Steps, projections and stage solves then impose u.n = u_in.n (as the
 * moments against the multiplier basis) and take u_in as the exterior state of the
 * convective flux. Synchronises the mesh's stream. Errors: DG_ERR_INVALID_ARG (NULL, no
 * inflow facets, non-finite values), DG_ERR_CUDA. */
int dg_set_inflow(dg_mesh* mesh, const double* vals);

/* Release every device buffer of the mesh. NULL is allowed. */
int dg_mesh_destroy(dg_mesh* mesh);

/* Sizes: out[0] = n_tri, out[1] = n_facet, out[2] = k, out[3] = n_lat(k),
 * out[4] = element geometry classes, out[5] = facet stencil classes,
 * out[6] = broken velocity DOFs n_tri (k+1)(k+2), out[7] = multiplier DOFs n_facet (k+1). */
int dg_mesh_info(const dg_mesh* mesh, int64_t out[8]);

/* Set the state from lattice values vals [n_tri][n_lat(k)][2] (the broken P^k
 * field interpolating them). No projection is applied: call
 * dg_project_divfree to move it into V_h^{k,-1}. The facet solver keeps its multipliers of
 * the last stages and steps: they set only the initial guess of the next solves, whose results
 * meet cg_rtol from any guess, and a state that continues the trajectory (a host round trip per
 * step) keeps the short warm-started solves; dg_project_divfree drops them.
 * Errors: DG_ERR_INVALID_ARG (NULL), DG_ERR_NONFINITE (NaN/Inf in vals). */
int dg_set_velocity(dg_mesh* mesh, const double* vals, int on_device);

/* Read the state as lattice values [n_tri][n_lat(k)][2]. */
int dg_get_velocity(dg_mesh* mesh, double* vals, int on_device);

/* State <- L2 projection onto V_h^{k,-1}: the hybrid-mixed solve of eq. (12)
 * with the functional F(v) = (u, v) (Theorem 2). */
int dg_project_divfree(dg_mesh* mesh);

/* nsteps >= 0 steps of SSP-RK3 (eq. (8)) with the fixed step dt > 0. Each stage
 * forms F = a M u^n + b [M u' + dt L(u')] and solves eq. (12) for the next
 * stage velocity. With DG_PRECISION_MIXED the facet system of each stage is
 * solved with FP32 preconditioning: FP32 PCG inside FP64 iterative refinement
 * (block Jacobi), or PCG on double-float vectors with the FP32 Fourier-space
 * preconditioner (lattice meshes), to the same cg_rtol; the element residual,
 * condensation and recovery run in double-float arithmetic (FP32 pairs, about
 * 48 significant bits) in the mixed form and in FP64 in the FP64 form.
 * Each stage's solve starts from an extrapolation of the same stage's multipliers in
 * the last steps (linear on lattice meshes, quadratic otherwise, once the steps had the
 * same dt; an initial guess only: every solve meets cg_rtol).
 * Returns DG_ERR_NOT_CONVERGED if any solve hit cg_maxit, DG_ERR_NONFINITE if
 * a residual norm became NaN/Inf (the state is then undefined).
 * Same as dg_step(mesh, DG_SCHEME_SSPRK3, dt, nsteps). */
int dg_rk3_step(dg_mesh* mesh, double dt, int64_t nsteps);

/* nsteps >= 0 steps of an explicit scheme with the fixed step dt > 0, each stage a
 * hybrid-mixed solve of eq. (12) with F = a M x + b M u' + c dt L(u'):
 *   DG_SCHEME_SSPRK3  SSP-RK3 of eq. (8) (three stages);
 *   DG_SCHEME_EULER   forward Euler, eq. (FE) of Sec. 3.1 with the full L (one stage);
 *   DG_SCHEME_RK4     classical four-stage RK4 of Example 1b (Table 2): stages
 *                     u_i = u^n + (dt/2, dt/2, dt) Q L(u_(i-1)), then
 *                     u^(n+1) = W + u_3 / 3 + dt/6 Q L(u_3), W = (-u^n + u_1 + 2 u_2) / 3,
 *                     Q the hybrid-mixed solve; the first RK4 step allocates W (one state).
 * Errors: DG_ERR_INVALID_ARG (unknown scheme, dt, nsteps), otherwise as dg_rk3_step. */
int dg_step(dg_mesh* mesh, int scheme, double dt, int64_t nsteps);

/* State as coefficients in the library's orthonormal basis (per triangle: 2 x n_lat(k)
 * scalar Dubiner polynomials scaled to unit L2 norm on the triangle; component-major,
 * double [n_tri][2 n_lat(k)]). The Euclidean inner product of coefficient arrays is
 * the L2 inner product of the fields, so gradients in this representation are L2
 * Riesz representers. Setting keeps the solver's warm-start multipliers, as dg_set_velocity. */
int dg_set_coefficients(dg_mesh* mesh, const double* coef, int on_device);
int dg_get_coefficients(dg_mesh* mesh, double* coef, int on_device);

/* Change the viscosity nu >= 0 of an existing mesh (nothing else depends on it). */
int dg_set_viscosity(dg_mesh* mesh, double nu);

/* Vector-Jacobian product of nsteps SSP-RK3 steps (the hand-written adjoint of eq. (8)).
 * With the current state u_0, it advances the state to u_K (K = nsteps, as dg_rk3_step
 * would) and returns, for the output cotangent ubar (coefficients, [n_tri][2 n_lat(k)]),
 * u0bar = (du_K/du_0)^T ubar in the same representation and *nubar = ubar . du_K/dnu.
 * Each stage u_s = Q(a M u^n + b [M u' + dt L(u')]) is reversed with the symmetric
 * hybrid-mixed solve Q (F-bar = Q u_s-bar), then u'-bar += b (F-bar + dt J_L(u')^T F-bar)
 * and u^n-bar += a F-bar, with J_L^T the transposed Jacobian of the upwind/SIPG residual
 * (d|s|/ds = sign(s), sign(0) = 0). u0bar is the gradient with respect to u_0 in the
 * broken space; pair it with divergence-free directions (or project it) for the
 * gradient on V_h^{k,-1}. States are kept every checkpoint_every steps and each segment
 * is recomputed during the reverse sweep (device memory: (K/checkpoint_every +
 * 3 checkpoint_every + 5) states, allocated for the call). Meshes with inflow or outflow
 * facets (dg_mesh_create_ex) give DG_ERR_UNSUPPORTED. */
int dg_rk3_vjp(dg_mesh* mesh, double dt, int64_t nsteps, int64_t checkpoint_every, const double* ubar,
               double* u0bar, double* nubar, int on_device);

/* Ensembles: advance several independent meshes (any sizes, degrees, viscosities,
 * precision forms) together. dg_batch_create records the members (the batch does
 * not own them; destroy the batch before its members). A batch call runs after the
 * work already on cuda_stream, on a stream the batch owns, and returns when it is done. dg_batch_rk3_step advances member i by nsteps
 * SSP-RK3 steps of size dt[i] (host array of n). One step of all members is
 * captured once as a CUDA graph and replayed per step; the first step after
 * creation, a projection or a change of any dt runs eagerly (it warms the
 * solver and fixes the step sizes the graph holds), and the graph is re-captured
 * when the step sizes change. Results equal those of dg_rk3_step on each member.
 * Returns the first member's non-OK status (all members are still advanced). */
int dg_batch_create(int n, dg_mesh* const* meshes, void* cuda_stream, dg_batch** out);
int dg_batch_destroy(dg_batch* batch);
int dg_batch_rk3_step(dg_batch* batch, const double* dt, int64_t nsteps);

/* Parallel branches of the captured ensemble step (no counterpart in the paper).
 * The members are dealt out, largest first to the least loaded, to `lanes` branches
 * of the graph that run concurrently; each member's persistent solver grid is then
 * divided by the lanes, so that every solver grid that can run at the same time fits
 * on the device together (no grid barrier can wait for another grid's blocks).
 * lanes = 0 (the default) makes the next dg_batch_rk3_step tune it: it captures the
 * step for 1, 2, 4, 8 and 16 lanes, times one replay of each (these are real steps of
 * the run, two per candidate) and keeps the fastest. lanes 1, 2, 4, 8 or 16 fixes it.
 * Member results do not depend on the lanes beyond the rounding of the solvers'
 * block-wise reductions. Errors: DG_ERR_INVALID_ARG. */
int dg_batch_set_lanes(dg_batch* batch, int lanes);
/* The lanes in use (0 before tuning) and the step times measured by the tuner for
 * 1, 2, 4, 8, 16 lanes in ms (-1 where not measured); either pointer may be NULL. */
int dg_batch_get_tuning(dg_batch* batch, int* lanes, double ms[5]);

/* Pressure of the current state: the (w, lam) of eq. (12) with the functional
 * L(u) alone, so w ~ p in the elements and lam ~ p on the skeleton (Theorem 2,
 * Remark 2), shifted by one constant so that the integral of w is zero
 * (L^2_0, eq. (4e)); with outflow facets p = 0 there fixes the constant and no shift is
 * applied (eq. (be)), and u.n = 0 is imposed on inflow facets (the functional L(u) is the
 * time derivative of a state that keeps its inflow data).
 * p_elem [n_tri][n_lat(k-1)]; p_facet [n_facet][k+1] or NULL. */
int dg_get_pressure(dg_mesh* mesh, double* p_elem, double* p_facet, int on_device);

/* Riesz representer of L(u) for the current state u (no projection): the
 * broken P^k field r with (r, v) = L(u)(v) for every broken v, as lattice
 * values [n_tri][n_lat(k)][2]. Exposes the residual kernels on their own. */
int dg_eval_residual(dg_mesh* mesh, double* vals, int on_device);

/* Diagnostics of the current state, computed on the device in FP64:
 * out[0] energy ||u||^2, out[1] enstrophy ||curl_h u||^2 (Example 2),
 * out[2] max |div u| at volume quadrature points, out[3] max |[u.n]| at facet
 * quadrature points, out[4] CG iterations of the last solve, out[5] CG
 * iterations summed since creation, out[6] solves since creation,
 * out[7] relative residual of the last solve. */
int dg_get_diagnostics(dg_mesh* mesh, double out[8]);

/* Facet-solver counters: out[0] CG iterations of the last solve (inner FP32
 * iterations summed over refinement sweeps in the mixed form), out[1] total
 * iterations, out[2] solves, out[3] final relative residual of the last solve,
 * out[4] refinement sweeps of the last solve, out[5] total sweeps, out[6] 1 if
 * the Fourier-space (lattice) preconditioner is in use, 2 for the multilevel
 * one, 0 for block Jacobi, out[7] persistent-kernel blocks of the solver in use. */
int dg_get_solver_stats(dg_mesh* mesh, double out[8]);

/* FP64 facet-system solve that allocates nothing, for callers that cannot call
 * cudaMalloc at all (for example code that must run inside someone else's
 * memory budget or pool, or in a context where allocation is forbidden), and
 * so cannot create a dg_mesh. The paper has no counterpart: it is the same
 * block-Jacobi PCG as the mesh solver (stop at ||g - S lam|| <= rtol ||g||
 * with the constant-multiplier component left out), on an operator the caller
 * holds. All pointers are device memory on the current device, owned by the
 * caller: facet_nbr int32 [n_facet][4], stencil int32 [n_facet], blocks double
 * [n_stencil][5][k+1][k+1], binv double [n_stencil][k+1][k+1] (the layout of
 * dg_host_facet_operator), g double [n_facet][k+1], lam double [n_facet][k+1]
 * (in: initial guess; out: solution, defined up to the constant multiplier).
 * Every facet_nbr entry must lie in [0, n_facet) and every stencil entry in
 * [0, n_stencil) for the blocks and binv passed: the call cannot check them
 * (it does not know n_stencil and reads no device data on the host), and an
 * index out of range makes the kernel read outside the caller's arrays.
 * Work vectors, reductions, the grid barrier and counters live in one static
 * device array sized for n_facet*(k+1) <= 262144 multiplier DOFs (about 12.7 MB,
 * held by every GPU that loads the library until exit); larger sizes return
 * DG_ERR_INVALID_ARG with a message and launch nothing. The first call on a
 * device looks up that array's address (cudaGetSymbolAddress), so make the
 * first call on each device before any stream capture. Every call shares the
 * array: calls that overlap on the GPU (other streams, other threads) race.
 * The call synchronises cuda_stream before it returns (it copies its counters
 * from the scratch array to the host). *iterations and *relres (may be NULL)
 * receive the CG iterations and final relative residual.
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED, DG_ERR_CUDA, DG_ERR_NOT_CONVERGED, DG_ERR_NONFINITE. */
int dg_facet_solve_noalloc(int k, int64_t n_facet, const int32_t* facet_nbr, const int32_t* stencil,
                           const double* blocks, const double* binv, const double* g, double* lam, double rtol,
                           int maxit, void* cuda_stream, int* iterations, double* relres);

/* Tensor-core recovery (mixed form, meshes with at most two geometry classes; off by
 * default: on GB300 it measured slower than the double-float recovery, whose work is
 * bound by memory latency, not by arithmetic). The recovery u_T = P_T f_T - G_T^T lam_T of eq. (12) runs
 * as one product [P_T, -G_T^T] [f_T; lam_T] per tile of 128 triangles of one class on
 * the tcgen05 tensor cores: bf16 operands split into seven signed 8-bit digits with
 * power-of-two scales, so that every FP32 accumulation is exact, and the digit levels
 * combined in double-float (relative error about 4e-15). enable = 0 (the default)
 * uses the double-float recovery on the FP32 units. Errors: DG_ERR_INVALID_ARG,
 * DG_ERR_UNSUPPORTED (enable = 1 where it is not set up). */
int dg_set_tensor_cores(dg_mesh* mesh, int enable);

/* Energy watchdog (failure detection; the paper has no counterpart, it rests on
 * the energy stability of Sec. 2.2 and Sec. 3): the kinetic energy ||u||^2 of
 * the scheme never grows for nu = 0 with upwinding (Sec. 2.2), nor with the
 * coercive viscous form, under a stable step size. With rel_tol > 0, every step
 * of dg_step / dg_rk3_step / dg_batch_rk3_step ends with a device reduction of
 * ||u||^2 (orthonormal basis: the sum of squared coefficients) compared with the
 * previous step's; growth by more than rel_tol (relative) makes the call return
 * DG_ERR_UNSTABLE (the state is still advanced), the usual sign of a step size
 * above the stability (CFL) limit. Setting a new state restarts the comparison.
 * rel_tol = 0 turns it off (the default). The first call with rel_tol > 0
 * allocates 16 KB of device memory. */
int dg_set_energy_watchdog(dg_mesh* mesh, double rel_tol);

/* Convergence history of the multilevel facet solver (no counterpart in the paper).
 * enable = 1 starts recording (allocates 16 KB of device memory once), 0 stops;
 * any other value only reads. out (cap doubles, may be NULL) receives, for every
 * PCG iteration i < 512 of the last solve, 4 values: the relative residual before
 * the iteration, r.z, p.S p and the step length alpha (-1 where p.S p <= 0 ended
 * the solve); *n_out (may be NULL) the iterations of the last solve.
 * Errors: DG_ERR_UNSUPPORTED (the mesh uses another preconditioner). */
int dg_solver_history(dg_mesh* mesh, int enable, double* out, int cap, int* n_out);

/* Test hook of the multilevel preconditioner (no counterpart in the paper): z = M r
 * for one V-cycle on the device, r and z [n_facet][k+1] in the coefficient layout of
 * dg_host_facet_operator (host memory for on_device = 0, which allocates two device
 * vectors for the mesh). Compares with dg_host_multilevel's host V-cycle.
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_UNSUPPORTED (the mesh uses another preconditioner). */
int dg_test_multilevel_apply(dg_mesh* mesh, const double* r, double* z, int on_device);

/* Test hook of the failure detection of the facet solvers (no counterpart in the
 * paper). Every grid barrier of the persistent solver kernels waits a bounded
 * number of polls (default 2^26); when the wait runs out the kernel sets an error
 * flag, every block leaves at its next barrier, and the call returns DG_ERR_CUDA
 * ("solver grid barrier timed out") with the device context intact.
 * spin_limit > 0 replaces the default limit for this mesh's solves (0: default);
 * skip_block >= 0 makes that block of the solver kernel leave at its first grid
 * barrier without arriving, so that the other blocks' wait runs out (-1: off).
 * The state after such a solve is undefined; (0, -1) restores normal operation. */
int dg_test_barrier_fault(dg_mesh* mesh, int64_t spin_limit, int skip_block);

/* Per-kernel-class device timing. enable = 1 makes the library record CUDA events
 * on its stream around every kernel launch from then on and add the elapsed times
 * up at the end of each call; inside a time step, a launch that directly follows
 * another starts at that launch's end event (one event per kernel boundary; the
 * launch gap counts in the following kernel). enable = 0 stops recording,
 * enable = 2 resets the totals. out_ms / out_launches (each n entries, or NULL)
 * receive the totals per class in the order of dg_kernel_name(0..). */
int dg_profile(dg_mesh* mesh, int enable, double* out_ms, int64_t* out_launches, int n);

/* Name of kernel class i, or NULL past the last class. */
const char* dg_kernel_name(int i);

/* Message of the last failing call on this thread ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DGDF_H */
