// Host-side FP64 set-up of the three-dimensional path (closed tetrahedral meshes, Sec. 2.1 with
// d = 3): topology with the canonical face parametrisation, reference tables on the tetrahedron
// and the triangle, per-class element operators of eq. (12) and the face stencil of the
// condensed system. Runs once per mesh; no CUDA here.
//
// Conventions shared with the kernels (k_tet.cu):
// * local face e of a tetrahedron is the one opposite its vertex e;
// * a face's canonical vertices p0, p1, p2 are its vertices in increasing periodic vertex id, and
//   x(s, t) = p0 + s (p1 - p0) + t (p2 - p0); both sides of a face evaluate at the same canonical
//   points; the multiplier basis is orthonormal on the reference triangle in (s, t);
// * perm index of a (tetrahedron, local face): which local vertex sits at each canonical vertex,
//   as the index 0..5 of that ordering among the face's three local vertices (kPerm3 in
//   setup3.cpp);
// * face rule (the one choice the CUDA path shares with any other implementation of the method):
//   q = ceil((3k+1)/2) Gauss-Legendre points in a and q Gauss-Jacobi (weight 1 - b) points in b,
//   s = a (1 - b), t = b, a-major; weights sum to 1/2.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dgdf {

constexpr int kMaxDegree3 = 2;

inline int n_lat3(int m) { return (m + 1) * (m + 2) * (m + 3) / 6; }

struct Ref3 {
  int k = 0, ns = 0, nw = 0, nl = 0, nq = 0, nqf = 0;
  std::vector<double> vxi, vw;        // volume rule [nq][3], [nq] (weights sum to 1/6)
  std::vector<double> vphi, vdphi;    // orthonormal basis of P^k on the reference tetrahedron,
                                      // ordered by degree: [nq][ns], [nq][ns][3]
  std::vector<double> fst, fw;        // face rule [nqf][2], [nqf] (canonical coordinates)
  std::vector<double> fphi, fdphi;    // [4 faces][6 perms][nqf][ns], [4][6][nqf][ns][3]
  std::vector<double> mu;             // multiplier basis at the face points [nqf][nl]
  std::vector<double> lat_phi, lat_inv;   // basis at the k-lattice [ns][ns] and its inverse
  std::vector<double> plat_phi;       // the first nw functions (P^(k-1)) at the (k-1)-lattice
                                      // [nw][nw] (the centroid for k = 1)
  std::vector<double> mu_lat;         // multiplier basis at the face's k-lattice points [nl][nl]:
                                      // (s, t) = (i/k, j/k), j = 0..k, i = 0..k-j (i fastest)
};

struct Class3 {
  double J[9], Jinv[9];     // J = [v1-v0, v2-v0, v3-v0] as columns (row-major); Jinv = dxi/dx
  double det;               // 6 |T|
  double normal[4][3];      // outward unit normals of the local faces
  double area[4];
  int perm[4];              // perm index of each local face
  std::vector<double> P;    // [nd][nd]
  std::vector<double> G;    // [4nl][nd]  C P
  std::vector<double> S;    // [4nl][4nl] C P C^T
  std::vector<double> W;    // [nw][nd]   pressure rows of the local solve: w = W (f - C^T lam)
  std::vector<double> WC;   // [nw][4nl]  W C^T
};

struct HostMesh3 {
  int k = 0, ns = 0, nd = 0, nw = 0, nl = 0;
  double alpha = 2.0;
  int64_t n_tet = 0, n_face = 0;
  Ref3 ref;
  std::vector<Class3> classes;
  std::vector<int32_t> tet_class;       // [n_tet]
  std::vector<int32_t> tet_face;        // [n_tet][4]
  std::vector<int32_t> tet_nbr;         // [n_tet][4] the tetrahedron across local face e
  std::vector<int8_t> tet_nbr_loc;      // [n_tet][4] its local face index
  std::vector<int32_t> face_tet;        // [n_face][2]
  std::vector<int8_t> face_loc;         // [n_face][2]
  std::vector<double> face_sigma;       // [n_face] alpha k^2 / max(diam T+, diam T-)
  std::vector<double> diam;             // [n_tet]
  // condensed system: row F couples to itself and the three other faces of each side
  std::vector<int32_t> face_nbr;        // [n_face][6]
  std::vector<int32_t> face_stencil;    // [n_face] stencil class
  int n_stencil = 0;
  std::vector<double> stencil_blocks;   // [n_stencil][7][nl][nl]
  std::vector<double> stencil_binv;     // [n_stencil][nl][nl] inverse of the own block
};

// Builds everything above. tet_vertex_ids int64 [n_tet][4] (periodic ids), tet_coords double
// [n_tet][4][3] (unwrapped corners). Every face must have two sides, with three distinct ids.
int build_host_mesh3(int64_t n_tet, const int64_t* vid, const double* X, int k, double alpha, HostMesh3& hm,
                     std::string& err);

}  // namespace dgdf
