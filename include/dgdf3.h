/* libdgdf, three-dimensional path: the explicit divergence-free DG method on closed tetrahedral
 * meshes (Sec. 2.1 with d = 3: BDM_k velocities, broken P^{k-1} pressures, P^k multipliers on the
 * triangular faces; the hybrid-mixed solve of eq. (12) after static condensation; the upwind
 * convection form eq. (7) and the SIPG viscous form eq. (18); SSP-RK3, eq. (8)). FP64 form,
 * multilevel (or block-Jacobi) PCG on the face system, k = 1 or 2.
 *
 * Conventions:
 * - local face e of a tetrahedron is the one opposite its vertex e; every face must be shared by
 *   two tetrahedra (periodic or interior), with three distinct periodic vertex ids (so a periodic
 *   cube needs at least 2 cells per direction);
 * - velocity values are given at the equispaced lattice points of each tetrahedron,
 *   v0 + (i/k)(v1-v0) + (j/k)(v2-v0) + (l/k)(v3-v0) for l = 0..k, j = 0..k-l, i = 0..k-l-j
 *   (i fastest), n_lat3(k) = (k+1)(k+2)(k+3)/6 points, three components each;
 * - a face is parametrised by its vertices in increasing periodic vertex id, and both sides
 *   evaluate at the same points of the face rule (q = ceil((3k+1)/2) Gauss-Legendre points times
 *   q Gauss-Jacobi points for the weight (1 - b), collapsed).
 * Ownership, status codes (dgdf.h), streams and the thread-local dg_last_error are as in dgdf.h.
 */
#ifndef DGDF3_H
#define DGDF3_H

#include <stdint.h>

#include "dgdf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh3 dg_mesh3;

/* Build a mesh: n_tet >= 1; tet_vertex_ids int64 [n_tet][4] (ids of the identified periodic
 * vertices), tet_coords double [n_tet][4][3] (unwrapped corners, positively oriented); host memory.
 * params as for dg_mesh_create: k in 1..2, nu >= 0, alpha > 0 (eq. (18)), precision must be
 * DG_PRECISION_FP64, cg_rtol / cg_maxit / cuda_stream as there. precond: DG_PRECOND_BLOCK_JACOBI
 * gives block-Jacobi PCG; otherwise (the default) PCG with one V-cycle of a multilevel
 * preconditioner per iteration: block-Jacobi Chebyshev(2) smoothing on the face system, injection
 * to the face-constant multipliers, smoothed aggregation on their operator with point-Jacobi
 * smoothing, a pseudo-inverse on the coarsest level (set up on the host at creation; the V-cycle
 * runs in FP32, the PCG vectors, S and the stopping test in FP64).
 * State starts at zero. Errors: DG_ERR_INVALID_ARG, DG_ERR_MESH, DG_ERR_UNSUPPORTED (k, precision,
 * a face with one side), DG_ERR_CUDA, DG_ERR_OOM. */
int dg3_mesh_create(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords,
                    const dg_params* params, dg_mesh3** out);
int dg3_mesh_destroy(dg_mesh3* mesh);

/* out[0] = n_tet, out[1] = n_face, out[2] = k, out[3] = n_lat3(k), out[4] = geometry classes,
 * out[5] = face stencil classes, out[6] = velocity DOFs, out[7] = multiplier DOFs. */
int dg3_mesh_info(const dg_mesh3* mesh, int64_t out[8]);

/* State from / to lattice values [n_tet][n_lat3(k)][3] (host or device memory). Setting applies
 * no projection. Errors: DG_ERR_INVALID_ARG (NULL), DG_ERR_NONFINITE (host input). */
int dg3_set_velocity(dg_mesh3* mesh, const double* vals, int on_device);
int dg3_get_velocity(dg_mesh3* mesh, double* vals, int on_device);

/* State <- L2 projection onto the divergence-free broken space (the hybrid-mixed solve with
 * F(v) = (u, v)). Errors: DG_ERR_NOT_CONVERGED, DG_ERR_NONFINITE, DG_ERR_CUDA. */
int dg3_project_divfree(dg_mesh3* mesh);

/* nsteps >= 0 SSP-RK3 steps of size dt > 0, each stage M u_s = a M u^n + b [M u' + dt L(u')]
 * solved by the hybrid-mixed system (eq. (8), eq. (12)). Each stage's face solve starts from
 * the quadratic extrapolation of the same stage's multipliers in the last three steps (once
 * they had this dt; fewer entries: linear, or the last one rescaled); dg3_set_velocity keeps
 * that history, dg3_project_divfree drops it. Errors as dg3_project_divfree. */
int dg3_rk3_step(dg_mesh3* mesh, double dt, int64_t nsteps);

/* Pressure of the current state: the (w, lam) of eq. (12) with the functional L(u) alone, so
 * w ~ p in the tetrahedra and lam ~ p on the faces (Theorem 2, Remark 2), shifted by one constant
 * so that the integral of w over the domain is zero (L^2_0, eq. (4e)).
 * p_elem [n_tet][n_lat3(k-1)]: w at the degree-(k-1) lattice points of each tetrahedron (the
 * order of the velocity lattice with k - 1 for k; the centroid for k = 1).
 * p_face [n_face][(k+1)(k+2)/2] or NULL: lam at the points p0 + (i/k)(p1 - p0) + (j/k)(p2 - p0),
 * j = 0..k, i = 0..k-j (i fastest), p0, p1, p2 the face's vertices in increasing periodic vertex
 * id; faces are numbered in order of first appearance over the tetrahedra t = 0, 1, ... and
 * their local faces e = 0..3 (dg3_host_faces in dgdf_host.h lists them).
 * Host or device memory. Errors as dg3_project_divfree. */
int dg3_get_pressure(dg_mesh3* mesh, double* p_elem, double* p_face, int on_device);

/* The Riesz representer of L(u) (eq. (6)) of the current state, as lattice values. */
int dg3_eval_residual(dg_mesh3* mesh, double* vals, int on_device);

/* out[0] energy ||u||^2, out[1] enstrophy ||curl_h u||^2, out[2] max |div u| at the volume
 * points, out[3] max |[u.n]| at the face points, out[4] PCG iterations of the last solve,
 * out[5] its relative residual, out[6] total iterations, out[7] solves. */
int dg3_get_diagnostics(dg_mesh3* mesh, double out[8]);

#ifdef __cplusplus
}
#endif

#endif /* DGDF3_H */
