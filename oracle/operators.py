"""Material matrices and the operator blocks of eq. (DAE) (oracle; test infrastructure).

Sec. II splits the edge unknowns into conducting ``a_c`` and nonconducting
``a_n`` and writes the semi-discrete system (DAE)

    [M_c 0; 0 0] d/dt [a_c; a_n] + [K_c(a_c) K_cn; K_cn^T K_n] [a_c; a_n] = [0; j_Sn].

With the FIT matrices assembled here, ``K(a) = C^T M_nu(a) C`` and

* ``M_kappa[e] = h * (mean sigma of the four cells around e)``,
* ``M_nu[f]   = (mean nu of the two cells sharing f) / h``,
* ``nu = nu0`` in linear cells and ``k1 exp(k2 |B|^2) + k3`` in Brauer cells,
  with ``|B|`` of a cell = norm of the three opposite-face flux sums / (2 h^2),
* an edge is Dirichlet if it lies in the outer surface, conducting (c) if
  not Dirichlet and ``M_kappa > 0``, nonconducting (n) otherwise,
* ``K_n = K[n, n]``, ``K_cn = K[c, n]``, ``K_c(a) = K(a)[c, c]``, ``M_c = M_kappa[c]``.

Every face touching an n-edge borders only nonconducting (hence linear) cells,
so ``K_n`` and ``K_cn`` do not depend on ``a`` (Sec. II calls K_n "typically
constant"); they are assembled once at ``a = 0``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fit_grid import FitGrid


class Discretization:
    """Assembled FIT operators for one problem (all FP64, SI units)."""

    def __init__(self, problem):
        N = problem.N
        self.problem = problem
        self.N = N
        self.h = float(problem.h)
        self.grid = g = FitGrid(N)
        self.G = g.gradient()
        self.C = g.curl()
        self.S = g.divergence()
        self.sigma = np.asarray(problem.sigma_cell, dtype=np.float64).reshape(-1)
        self.brauer = np.asarray(problem.brauer_cell).reshape(-1).astype(bool)
        if np.any(self.brauer & (self.sigma <= 0)):
            raise ValueError("a Brauer (nonlinear) cell must be conducting")
        if np.any(self.sigma < 0):
            raise ValueError("negative conductivity")
        self.nu0, self.k1, self.k2, self.k3 = problem.nu0, problem.k1, problem.k2, problem.k3
        self._Ae = g.edge_cell_average()
        self._Af = g.face_cell_average()
        self._pairs = g.cell_face_pairs()
        self.M_kappa = self.h * (self._Ae @ self.sigma)
        self.dirichlet = g.dirichlet_edges()
        self.c_mask = (~self.dirichlet) & (self.M_kappa > 0)
        self.n_mask = (~self.dirichlet) & (self.M_kappa == 0)
        self.c_idx = np.flatnonzero(self.c_mask)
        self.n_idx = np.flatnonzero(self.n_mask)
        self.X_s = g.coil_loop(problem.coil_k, problem.coil_i0, problem.coil_j0,
                               problem.coil_i1, problem.coil_j1)
        if np.any(self.X_s[~self.n_mask] != 0):
            raise ValueError("coil edges must be nonconducting interior edges")
        K0 = self.K(np.zeros(g.n_edges))
        self.K_n = K0[self.n_idx][:, self.n_idx].tocsr()
        self.K_cn = K0[self.c_idx][:, self.n_idx].tocsr()
        self.M_c = self.M_kappa[self.c_idx]
        self.D = self.K_n.diagonal()       # Jacobi preconditioner diag(K_n)

    # --- material laws -------------------------------------------------------
    def brauer_nu(self, B):
        """Brauer reluctivity nu(B) = k1 exp(k2 B^2) + k3."""
        return self.k1 * np.exp(self.k2 * B * B) + self.k3

    def cell_flux_density(self, a_full):
        """|B| per cell from the face fluxes b = C a (Wb): norm of the sums of
        opposite faces divided by 2 h^2 (mean flux over the cell's area)."""
        b = self.C @ a_full
        comps = [P @ b for P in self._pairs]
        return np.sqrt(comps[0] ** 2 + comps[1] ** 2 + comps[2] ** 2) / (2.0 * self.h * self.h)

    def cell_nu(self, a_full):
        """Reluctivity per cell for the edge state a_full."""
        nu = np.full(self.sigma.size, self.nu0)
        if np.any(self.brauer):
            B = self.cell_flux_density(a_full)
            nu[self.brauer] = self.brauer_nu(B[self.brauer])
        return nu

    def M_nu(self, a_full):
        """Diagonal reluctance matrix per face: mean nu of adjacent cells / h."""
        return (self._Af @ self.cell_nu(a_full)) / self.h

    def K(self, a_full) -> sp.csr_matrix:
        """Full curl-curl matrix K(a) = C^T M_nu(a) C over all edges."""
        return (self.C.T @ sp.diags(self.M_nu(a_full)) @ self.C).tocsr()

    def apply_K(self, a_full, v_full):
        """K(a) v evaluated as C^T (M_nu(a) (C v))."""
        return self.C.T @ (self.M_nu(a_full) * (self.C @ v_full))

    # --- block helpers ---------------------------------------------------------
    def full(self, a_c=None, a_n=None):
        """Scatter conducting / nonconducting parts into a full edge vector."""
        a = np.zeros(self.grid.n_edges)
        if a_c is not None:
            a[self.c_idx] = a_c
        if a_n is not None:
            a[self.n_idx] = a_n
        return a

    def K_c(self, a_c) -> sp.csr_matrix:
        """Nonlinear conducting block K_c(a_c) = K(a)[c, c]; |B| in conducting
        cells depends on c-edges only, so a_n does not enter."""
        return self.K(self.full(a_c=a_c))[self.c_idx][:, self.c_idx].tocsr()

    @property
    def n_c(self):
        return self.c_idx.size

    @property
    def n_n(self):
        return self.n_idx.size
