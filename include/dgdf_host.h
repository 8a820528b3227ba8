/*
 * dgdf_host.h - host-only introspection of libdgdf's set-up (no GPU needed).
 *
 * These calls expose the FP64 set-up that dg_mesh_create performs on the host
 * before anything reaches the device, so that it can be checked on a machine
 * without a GPU: the facet topology of Sec. 2.1 and the reference quadrature
 * rules and orthonormal basis behind the element and facet kernels. They
 * allocate host memory only and never touch CUDA.
 */
#ifndef DGDF_HOST_H
#define DGDF_HOST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Facet topology with the conventions of dgdf.h. Inputs as dg_mesh_create.
 * *n_facet receives the facet count. If tri_facet (int32 [n_tri][3]) is not
 * NULL it receives the facet of each local facet; tri_orient (int8 [n_tri][3])
 * +1 / -1 when the triangle traverses it along / against its canonical
 * direction; facet_tri (int32 [n_facet][2]) its two triangles, first
 * appearance first, -1 as the second on a wall (an edge with one triangle);
 * all three must then hold the sizes above (call once with NULLs to get
 * n_facet). Errors: DG_ERR_INVALID_ARG, DG_ERR_MESH. */
int dg_host_topology(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords,
                     int64_t* n_facet, int32_t* tri_facet, int8_t* tri_orient, int32_t* facet_tri);

/* Reference tables for degree k (1..3) on the triangle {xi1, xi2 >= 0, xi1 + xi2 <= 1}:
 *   table 0: volume rule, [nq][3] = (xi1, xi2, weight), exact to degree 3k-1 (weights sum to 1/2)
 *   table 1: facet rule on [0,1], [nqf][2] = (t, weight), nqf = ceil((3k+1)/2)
 *   table 2: orthonormal basis at the volume points, [nq][ns]
 *   table 3: reference gradients at the volume points, [nq][ns][2]
 *   table 4: basis at the k-lattice points, [ns][ns] (row = point)
 * ns = (k+1)(k+2)/2. *n_out receives the number of doubles; out (capacity cap
 * doubles) may be NULL to query the size. */
int dg_host_reference(int k, int table, double* out, int64_t cap, int64_t* n_out);

/* The condensed facet system of eq. (12) as the library stores it. Inputs as
 * dg_mesh_create (k 1..3, alpha > 0). Its row F is
 *   (S x)_F = sum_b blocks[stencil[F]][b] x_{nbr_b}, nbr_0 = F, nbr_1..4 = facet_nbr[F][0..3],
 * with coefficients in the facet basis sqrt(2m+1) P_m(2t-1) of the canonical parameter t.
 * *n_facet and *n_stencil receive the counts. facet_nbr (int32 [n_facet][4]),
 * stencil (int32 [n_facet]), blocks (double [n_stencil][5][k+1][k+1]) and binv
 * (double [n_stencil][k+1][k+1], inverse of the own block) may be NULL; when
 * given, cap_blocks must be >= n_stencil (call once with NULLs for the sizes). */
int dg_host_facet_operator(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k,
                           double alpha, int64_t* n_facet, int64_t* n_stencil, int32_t* facet_nbr,
                           int32_t* stencil, double* blocks, double* binv, int64_t cap_blocks);

/* Lattice structure used by DG_PRECOND_AUTO: returns DG_ERR_UNSUPPORTED when the
 * mesh is not a translation-invariant split-square mesh with N a power of two.
 * *N receives the cells per direction; facet_of (int32 [3][N][N], row j, column
 * i) the facet of each (type, cell); sinv (double [N][N][C][C][2], C = 3(k+1))
 * the inverse of the Fourier symbol of the facet operator at (k_i, k_j), as
 * (re, im), pseudo-inverse at (0, 0); cap is the capacity of sinv in doubles.
 * Pass NULL arrays to query N. */
int dg_host_lattice(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k, double alpha,
                    int64_t* N, int32_t* facet_of, double* sinv, int64_t cap);

/* The multilevel preconditioner of the facet system (DG_PRECOND_MULTILEVEL; no
 * counterpart in the paper, which factorises the system directly, Sec. 4), built
 * on the host as dg_mesh_create builds it. Inputs as dg_host_facet_operator.
 * info[0] = smoothing levels L, info[1] = rows of the coarsest level, then for
 * level l < L: info[2 + 2l] = rows, info[3 + 2l] = values per row (p-levels on the
 * facets: k+1, 2, 1 modes; aggregation levels: 1). With nr > 0, z[i] = M r[i] for
 * nr vectors of n_facet (k+1) values (one V-cycle each, FP64, in the coefficient
 * layout of dg_host_facet_operator). With g and lam given, PCG with M from lam = 0
 * on S lam = g (the constant multiplier left out) to relative residual rtol:
 * lam receives the solution, *iters (may be NULL) the iterations.
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_MESH, DG_ERR_UNSUPPORTED. */
int dg_host_multilevel(int64_t n_tri, const int64_t* tri_vertex_ids, const double* tri_coords, int k, double alpha,
                       int64_t info[34], int nr, const double* r, double* z, const double* g, double* lam,
                       double rtol, int64_t* iters);

/* Face numbering of the three-dimensional set-up (dg3_mesh_create's, include/dgdf3.h), on the host.
 * *n_face_out (may be NULL) receives the number of faces; face_tet [n_face][2] and face_loc
 * [n_face][2] (each may be NULL) the two tetrahedra of every face and its local index in each (the
 * face opposite that local vertex); face_vid [n_face][3] (may be NULL) its periodic vertex ids in
 * increasing order (p0, p1, p2 of the canonical parametrisation that dg3_get_pressure's face
 * values use). Call with NULL arrays first for the count; caller-owned host arrays.
 * Errors: DG_ERR_INVALID_ARG (NULL mesh arrays), DG_ERR_MESH, DG_ERR_UNSUPPORTED. */
int dg3_host_faces(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords, int64_t* n_face_out,
                   int64_t* face_tet, int8_t* face_loc, int64_t* face_vid);

/* Three-dimensional host check (include/dgdf3.h conventions): the L2 projection of the field
 * given by lattice values vals [n_tet][n_lat3(k)][3] onto the divergence-free space, computed on
 * the host from the set-up dg3_mesh_create uploads (class operators, face stencil) with a host
 * PCG preconditioned by one V-cycle of the assembled multilevel hierarchy (point-Jacobi smoothing),
 * to 1e-13 relative. out: lattice values, as vals; *iters: PCG iterations (may be NULL).
 * Errors: DG_ERR_INVALID_ARG, DG_ERR_MESH, DG_ERR_UNSUPPORTED. */
int dg3_host_project(int64_t n_tet, const int64_t* tet_vertex_ids, const double* tet_coords, int k, double alpha,
                     const double* vals, double* out, int64_t* iters);

#ifdef __cplusplus
}
#endif

#endif /* DGDF_HOST_H */
