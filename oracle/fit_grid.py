"""Cartesian FIT grid topology, assembled explicitly (oracle; test infrastructure).

Lowest-order edge unknowns of a Ritz-Galerkin / finite-integration
discretisation (Sec. II, weak form and eq. (DAE)).  Everything here is integer
topology: node-edge incidence ``G`` (discrete gradient), edge-face incidence
``C`` (discrete curl) and face-cell incidence ``S`` (discrete divergence).

Numbering (all C order, x index fastest):

* nodes  (i, j, k), i, j, k in [0, N]                       -> i + (N+1)(j + (N+1)k)
* x-edges (i, j, k), i in [0, N), j, k in [0, N]            -> i + N(j + (N+1)k)
* y-edges (i, j, k), j in [0, N), i, k in [0, N]            -> oy + i + (N+1)(j + N k)
* z-edges (i, j, k), k in [0, N), i, j in [0, N]            -> oz + i + (N+1)(j + (N+1)k)
* x-faces (normal x) at node plane i in [0, N], cell (j, k)  -> i + (N+1)(j + N k)
* y-faces at node plane j in [0, N], cell (i, k)             -> fy + i + N(j + (N+1)k)
* z-faces at node plane k in [0, N], cell (i, j)             -> fz + i + N(j + N k)
* cells (i, j, k) in [0, N)^3                                -> i + N(j + N k)

Face loops are right-handed about the face normal; a z-face's flux is
``a_x(i,j,k) + a_y(i+1,j,k) - a_x(i,j+1,k) - a_y(i,j,k)`` and the x-/y-faces
follow by cyclic permutation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class FitGrid:
    """Topology of an N^3-cell grid with homogeneous Dirichlet boundary."""

    def __init__(self, N: int):
        if N < 2:
            raise ValueError("need at least 2 cells per axis")
        self.N = N
        N1 = N + 1
        self.n_nodes = N1 ** 3
        self.n_x = N * N1 * N1
        self.n_y = N1 * N * N1
        self.n_z = N1 * N1 * N
        self.oy = self.n_x
        self.oz = self.n_x + self.n_y
        self.n_edges = self.n_x + self.n_y + self.n_z
        self.n_fx = N1 * N * N
        self.n_fy = N * N1 * N
        self.n_fz = N * N * N1
        self.fy0 = self.n_fx
        self.fz0 = self.n_fx + self.n_fy
        self.n_faces = self.n_fx + self.n_fy + self.n_fz
        self.n_cells = N ** 3

    # --- index maps --------------------------------------------------------
    def node(self, i, j, k):
        N1 = self.N + 1
        return i + N1 * (j + N1 * k)

    def ex(self, i, j, k):
        return i + self.N * (j + (self.N + 1) * k)

    def ey(self, i, j, k):
        return self.oy + i + (self.N + 1) * (j + self.N * k)

    def ez(self, i, j, k):
        N1 = self.N + 1
        return self.oz + i + N1 * (j + N1 * k)

    def fx(self, i, j, k):
        return i + (self.N + 1) * (j + self.N * k)

    def fy(self, i, j, k):
        return self.fy0 + i + self.N * (j + (self.N + 1) * k)

    def fz(self, i, j, k):
        return self.fz0 + i + self.N * (j + self.N * k)

    def cell(self, i, j, k):
        return i + self.N * (j + self.N * k)

    @staticmethod
    def _grid(ni, nj, nk):
        """(i, j, k) index arrays enumerated in C order over shape (nk, nj, ni)."""
        k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
        return i.ravel(), j.ravel(), k.ravel()

    def edge_coords(self):
        """(component, i, j, k) of every edge, in edge-index order."""
        N, N1 = self.N, self.N + 1
        parts = []
        for comp, shape in ((0, (N, N1, N1)), (1, (N1, N, N1)), (2, (N1, N1, N))):
            i, j, k = self._grid(*shape)
            parts.append((np.full(i.size, comp), i, j, k))
        return tuple(np.concatenate([p[t] for p in parts]) for t in range(4))

    # --- incidence matrices -------------------------------------------------
    def gradient(self) -> sp.csr_matrix:
        """G (edges x nodes): +1 at the edge's head node, -1 at its tail."""
        N, N1 = self.N, self.N + 1
        rows, cols, vals = [], [], []
        for emap, shape, step in ((self.ex, (N, N1, N1), (1, 0, 0)),
                                  (self.ey, (N1, N, N1), (0, 1, 0)),
                                  (self.ez, (N1, N1, N), (0, 0, 1))):
            i, j, k = self._grid(*shape)
            e = emap(i, j, k)
            rows += [e, e]
            cols += [self.node(i + step[0], j + step[1], k + step[2]), self.node(i, j, k)]
            vals += [np.ones(e.size), -np.ones(e.size)]
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_edges, self.n_nodes))

    def curl(self) -> sp.csr_matrix:
        """C (faces x edges): right-handed loop sums of the edge values."""
        N, N1 = self.N, self.N + 1
        rows, cols, vals = [], [], []

        def add(f, e, s):
            rows.append(f)
            cols.append(e)
            vals.append(np.full(f.size, float(s)))

        i, j, k = self._grid(N1, N, N)          # x-faces
        f = self.fx(i, j, k)
        add(f, self.ey(i, j, k), +1)
        add(f, self.ez(i, j + 1, k), +1)
        add(f, self.ey(i, j, k + 1), -1)
        add(f, self.ez(i, j, k), -1)
        i, j, k = self._grid(N, N1, N)          # y-faces
        f = self.fy(i, j, k)
        add(f, self.ez(i, j, k), +1)
        add(f, self.ex(i, j, k + 1), +1)
        add(f, self.ez(i + 1, j, k), -1)
        add(f, self.ex(i, j, k), -1)
        i, j, k = self._grid(N, N, N1)          # z-faces
        f = self.fz(i, j, k)
        add(f, self.ex(i, j, k), +1)
        add(f, self.ey(i + 1, j, k), +1)
        add(f, self.ex(i, j + 1, k), -1)
        add(f, self.ey(i, j, k), -1)
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_faces, self.n_edges))

    def divergence(self) -> sp.csr_matrix:
        """S (cells x faces): outward face sum of each cell."""
        N = self.N
        i, j, k = self._grid(N, N, N)
        c = self.cell(i, j, k)
        rows = [c] * 6
        cols = [self.fx(i + 1, j, k), self.fx(i, j, k), self.fy(i, j + 1, k),
                self.fy(i, j, k), self.fz(i, j, k + 1), self.fz(i, j, k)]
        vals = [np.full(c.size, s) for s in (1.0, -1.0, 1.0, -1.0, 1.0, -1.0)]
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n_cells, self.n_faces))

    # --- boundary and adjacency ----------------------------------------------
    def dirichlet_edges(self) -> np.ndarray:
        """True for edges lying in the outer boundary surface."""
        N = self.N
        comp, i, j, k = self.edge_coords()
        onb = lambda v: (v == 0) | (v == N)  # noqa: E731
        return np.where(comp == 0, onb(j) | onb(k),
                        np.where(comp == 1, onb(i) | onb(k), onb(i) | onb(j)))

    def edge_cell_average(self) -> sp.csr_matrix:
        """(edges x cells): 1/4 on each of the up to four cells around an edge
        (cells outside the domain contribute zero)."""
        N = self.N
        comp, i, j, k = self.edge_coords()
        e = np.arange(self.n_edges)
        rows, cols = [], []
        for da in (-1, 0):
            for db in (-1, 0):
                ci = np.where(comp == 0, i, i + da)
                cj = np.where(comp == 1, j, np.where(comp == 0, j + da, j + db))
                ck = np.where(comp == 2, k, k + db)
                ok = (ci >= 0) & (ci < N) & (cj >= 0) & (cj < N) & (ck >= 0) & (ck < N)
                rows.append(e[ok])
                cols.append(self.cell(ci[ok], cj[ok], ck[ok]))
        r, c = np.concatenate(rows), np.concatenate(cols)
        return sp.csr_matrix((np.full(r.size, 0.25), (r, c)), shape=(self.n_edges, self.n_cells))

    def face_cell_average(self) -> sp.csr_matrix:
        """(faces x cells): mean over the two cells sharing a face, or the single
        adjacent cell for a face in the outer boundary."""
        N = self.N
        rows, cols = [], []
        for fmap, shape, axis in ((self.fx, (N + 1, N, N), 0), (self.fy, (N, N + 1, N), 1),
                                  (self.fz, (N, N, N + 1), 2)):
            i, j, k = self._grid(*shape)
            f = fmap(i, j, k)
            for d in (-1, 0):
                ci, cj, ck = i + d * (axis == 0), j + d * (axis == 1), k + d * (axis == 2)
                ok = (ci >= 0) & (ci < N) & (cj >= 0) & (cj < N) & (ck >= 0) & (ck < N)
                rows.append(f[ok])
                cols.append(self.cell(ci[ok], cj[ok], ck[ok]))
        r, c = np.concatenate(rows), np.concatenate(cols)
        cnt = np.bincount(r, minlength=self.n_faces).astype(float)
        return sp.csr_matrix((1.0 / cnt[r], (r, c)), shape=(self.n_faces, self.n_cells))

    def cell_face_pairs(self):
        """Three (cells x faces) matrices summing the two opposite faces of each
        cell normal to x, y and z."""
        N = self.N
        i, j, k = self._grid(N, N, N)
        c = self.cell(i, j, k)
        out = []
        for lo, hi in ((self.fx(i, j, k), self.fx(i + 1, j, k)),
                       (self.fy(i, j, k), self.fy(i, j + 1, k)),
                       (self.fz(i, j, k), self.fz(i, j, k + 1))):
            out.append(sp.csr_matrix((np.ones(2 * c.size), (np.concatenate([c, c]), np.concatenate([lo, hi]))),
                                     shape=(self.n_cells, self.n_faces)))
        return out

    def coil_loop(self, k, i0, j0, i1, j1) -> np.ndarray:
        """Edge vector X_s: +1/-1 along a rectangular loop of edges in node
        plane k around node square [i0,i1] x [j0,j1], counter-clockwise seen
        from +z (Sec. II, J_S = X_S i_S(t))."""
        x = np.zeros(self.n_edges)
        ii = np.arange(i0, i1)
        jj = np.arange(j0, j1)
        x[self.ex(ii, j0, k)] += 1.0
        x[self.ey(i1, jj, k)] += 1.0
        x[self.ex(ii, j1, k)] -= 1.0
        x[self.ey(i0, jj, k)] -= 1.0
        return x
