"""Mesh topology of the oracle (test infrastructure only).

Definitions (shared with the C-ABI as conventions, implemented independently):

* local facet e of a triangle is the edge opposite its vertex e, traversed
  counter-clockwise from vertex (e+1)%3 to vertex (e+2)%3;
* a facet's canonical direction is its edge vector d with d_x > 0, or d_x = 0 and d_y > 0;
  the canonical parameter t in [0, 1] runs from the canonical start to end;
* two element edges are the same facet when they join the same pair of
  identified vertices in the same canonical order and have the same edge
  vector (this separates the periodic images on meshes as coarse as 1 x 1);
* facets are numbered in order of first appearance over (triangle, local facet);
* an edge that no other triangle shares is a boundary facet: it has one side, and
  facet_tri / facet_loc / facet_orient hold -1 for the missing second side. Its kind comes
  from the caller's per-edge array (edge e of a triangle is opposite its vertex e): WALL
  (default), INFLOW or OUTFLOW, the boundary parts of Sec. 2.5, eq. (be).
"""
import numpy as np

WALL, INFLOW, OUTFLOW = 0, 1, 2


class Topology:
    def __init__(self, tri_vertex_ids, tri_coords, edge_kind=None):
        vid = np.asarray(tri_vertex_ids, dtype=np.int64)
        X = np.asarray(tri_coords, dtype=np.float64)
        n = vid.shape[0]
        if vid.shape != (n, 3) or X.shape != (n, 3, 2):
            raise ValueError("bad mesh arrays")
        self.n_tri = n
        self.vid = vid
        self.X = X
        J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)  # columns v1-v0, v2-v0
        self.J = J
        self.detJ = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
        if np.any(self.detJ <= 0):
            raise ValueError("triangles must be counter-clockwise and non-degenerate")
        self.area = 0.5 * self.detJ
        self.centroid = X.mean(axis=1)
        edges = np.stack([X[:, 2] - X[:, 1], X[:, 0] - X[:, 2], X[:, 1] - X[:, 0]], axis=1)  # edge e: v(e+1)->v(e+2)
        self.edge_len = np.sqrt((edges ** 2).sum(-1))
        self.diam = self.edge_len.max(axis=1)
        # outward normal of local facet e of a CCW triangle: edge direction rotated clockwise
        self.normal = np.stack([edges[..., 1], -edges[..., 0]], axis=-1) / self.edge_len[..., None]

        scale = np.abs(X).max() + 1.0
        tol = 1e-9 * scale
        key_to_facet = {}
        facet_sides = []     # list of [(t, e, orient), ...]
        for t in range(n):
            for e in range(3):
                a, b = (e + 1) % 3, (e + 2) % 3
                d = X[t, b] - X[t, a]
                positive = d[0] > tol or (abs(d[0]) <= tol and d[1] > 0)
                if positive:
                    cs, ce, orient = a, b, 1
                else:
                    cs, ce, orient, d = b, a, -1, -d
                key = (int(vid[t, cs]), int(vid[t, ce]), int(round(d[0] / tol)), int(round(d[1] / tol)))
                f = key_to_facet.get(key)
                if f is None:
                    f = len(facet_sides)
                    key_to_facet[key] = f
                    facet_sides.append([])
                facet_sides[f].append((t, e, orient))
        for f, s in enumerate(facet_sides):
            if len(s) > 2:
                raise ValueError("facet %d has %d triangles" % (f, len(s)))
            if len(s) == 2 and s[0][2] == s[1][2]:
                raise ValueError("facet %d traversed in the same direction by both triangles" % f)
            if len(s) == 1:
                s.append((-1, -1, -1))
        self.n_facet = len(facet_sides)
        self.facet_tri = np.array([[s[0][0], s[1][0]] for s in facet_sides], dtype=np.int64)
        self.facet_loc = np.array([[s[0][1], s[1][1]] for s in facet_sides], dtype=np.int64)
        self.facet_orient = np.array([[s[0][2], s[1][2]] for s in facet_sides], dtype=np.int64)
        self.boundary = self.facet_tri[:, 1] < 0
        self.interior = np.flatnonzero(~self.boundary)
        self.tri_facet = np.empty((n, 3), dtype=np.int64)
        for f in range(self.n_facet):
            for s in range(2 if not self.boundary[f] else 1):
                self.tri_facet[self.facet_tri[f, s], self.facet_loc[f, s]] = f
        self.facet_len = self.edge_len[self.facet_tri[:, 0], self.facet_loc[:, 0]]
        self.facet_kind = np.full(self.n_facet, WALL, dtype=np.int64)
        if edge_kind is not None:
            ek = np.asarray(edge_kind).reshape(n, 3)
            b = np.flatnonzero(self.boundary)
            self.facet_kind[b] = ek[self.facet_tri[b, 0], self.facet_loc[b, 0]]
            if np.any((self.facet_kind < 0) | (self.facet_kind > 2)):
                raise ValueError("edge kinds are 0 (wall), 1 (inflow) or 2 (outflow)")
        self.facet_kind[~self.boundary] = WALL   # the kind of an interior edge is not used
        self.inflow = np.flatnonzero(self.boundary & (self.facet_kind == INFLOW))
        self.outflow = np.flatnonzero(self.boundary & (self.facet_kind == OUTFLOW))

    def facet_points(self, f, side, t):
        """Physical points (in the side's own unwrapped coordinates) at canonical parameters t.

        f, side: arrays [m]; t: [q]. Returns [m, q, 2].
        """
        tri = self.facet_tri[f, side]
        e = self.facet_loc[f, side]
        o = self.facet_orient[f, side]
        a = (e + 1) % 3
        b = (e + 2) % 3
        pa = self.X[tri, a]
        pb = self.X[tri, b]
        start = np.where((o > 0)[:, None], pa, pb)
        end = np.where((o > 0)[:, None], pb, pa)
        return start[:, None, :] + t[None, :, None] * (end - start)[:, None, :]
