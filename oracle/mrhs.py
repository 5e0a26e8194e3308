"""Start vectors for the multiple right-hand side problem (oracle; test infrastructure).

Sec. III, eq. (mrhs): every time step solves ``K_n a_p = j_p`` for a new
right-hand side with the same matrix, so earlier solutions carry information
about the next one.

SPE (Sec. III, eq. (SPE_x0)): the columns of ``U_SPE`` are an orthonormal basis,
built with modified Gram-Schmidt, of the span of earlier solutions; the start
vector is the Galerkin projection ``x0 = U (U^T K_n U)^-1 U^T b``.

POD (Sec. III, eqs. (SVD), (relSV2), (keepInfo), (POD_x0)): the snapshot matrix
``X`` of earlier solutions is decomposed ``X = U Sigma V^T``; the first ``k``
left singular vectors are kept, ``x0 = U_k (U_k^T K_n U_k)^-1 U_k^T b``.

Readings of the printed equations used here:

* the right-hand side projected in (SPE_x0)/(POD_x0) is the right-hand side
  ``b`` of the system being solved (the printed ``K_cn^T j_p`` is read as the
  current right-hand side, since the projection must live in the space of b);
* (relSV2) is printed as ``sigma_k / sigma_1 <= eps``; keeping the largest
  singular values means keeping every ``i`` with ``sigma_i / sigma_1 >= eps``;
* the window holds the last ``d`` solutions, newest first; MGS runs twice over
  it (one re-orthogonalisation) and drops a column whose remainder norm is at
  most ``eps_lin`` times its original norm;
* the small Galerkin system is solved by Cholesky, or by a symmetric
  eigen-solve truncated at ``1e-14 lambda_max`` when Cholesky fails.

CSPE (Sec. III, "cascaded SPE"; Sec. IV): only the last column of ``U_SPE``
changes from step to step, so the products with the other columns are reused, and
the number of columns grows during the run, staying below 20.  Reading of that
policy (the paper gives no schedule): the basis holds frozen past solutions plus
one live column, the newest solution; every ``period`` steps the live column is
frozen (the solutions of steps P, 2P, 3P, ... are kept) until ``depth`` columns
are reached, after which only the live column changes (``CspeBasis``).

Parity: pinned (Galerkin orthogonality, orthonormality, exact recovery when the
solution lies in the subspace, constructed snapshot matrices with known
singular values, the CSPE column schedule).
"""
from __future__ import annotations

import numpy as np


def mgs_orthonormal_basis(window, eps_lin=1e-10):
    """Modified Gram-Schmidt (two sweeps) over the columns of ``window``
    (newest first).  Returns the orthonormal columns as an (n, k) array."""
    basis = []
    for s in window:
        v = np.array(s, dtype=np.float64)
        ns = np.linalg.norm(v)
        for _sweep in range(2):
            for q in basis:
                v -= (q @ v) * q
        nv = np.linalg.norm(v)
        if ns == 0.0 or nv <= eps_lin * ns:
            continue
        basis.append(v / nv)
    if not basis:
        return np.zeros((len(window[0]) if len(window) else 0, 0))
    return np.column_stack(basis)


def solve_small_spd(H, g):
    """Solve the small projected system H y = g (H symmetric PSD)."""
    H = 0.5 * (H + H.T)
    try:
        L = np.linalg.cholesky(H)
        return np.linalg.solve(L.T, np.linalg.solve(L, g))
    except np.linalg.LinAlgError:
        lam, V = np.linalg.eigh(H)
        keep = lam > 1e-14 * lam.max() if lam.size and lam.max() > 0 else np.zeros(lam.size, bool)
        return V[:, keep] @ ((V[:, keep].T @ g) / lam[keep])


def galerkin_start(K_n, U, b):
    """x0 = U (U^T K_n U)^-1 U^T b for an (n, k) basis U."""
    if U.shape[1] == 0:
        return np.zeros(b.size)
    W = K_n @ U
    H = U.T @ W
    g = U.T @ b
    return U @ solve_small_spd(H, g)


def spe_start(K_n, window, b, eps_lin=1e-10):
    """SPE start vector (eq. (SPE_x0)); returns (x0, rank used)."""
    if len(window) == 0:
        return np.zeros(b.size), 0
    U = mgs_orthonormal_basis(window, eps_lin)
    return galerkin_start(K_n, U, b), U.shape[1]


def pod_start(K_n, snapshots, b, eps_pod=1e-4):
    """POD start vector (eqs. (SVD), (relSV2), (keepInfo), (POD_x0)).

    Returns (x0, k, singular values, information ratio)."""
    if len(snapshots) == 0:
        return np.zeros(b.size), 0, np.zeros(0), 0.0
    X = np.column_stack(snapshots)
    U, sig, _Vt = np.linalg.svd(X, full_matrices=False)
    if sig[0] == 0.0:
        return np.zeros(b.size), 0, sig, 0.0
    k = int(np.count_nonzero(sig / sig[0] >= eps_pod))
    info = float(sig[:k].sum() / sig.sum())
    return galerkin_start(K_n, U[:, :k], b), k, sig, info


class CspeBasis:
    """Columns of the cascaded SPE basis: frozen past solutions and the live one."""

    def __init__(self, period=25, depth=8):
        self.period = period if period > 0 else 25
        self.depth = depth
        self.frozen = []        # oldest first
        self.live = None
        self.count = 0

    def push(self, w):
        """Record the solution of the step just finished (push number count+1)."""
        self.count += 1
        if self.live is not None and (self.count - 1) % self.period == 0 and len(self.frozen) + 1 < self.depth:
            self.frozen.append(self.live)
        self.live = np.array(w, dtype=np.float64)

    def window(self):
        """The basis columns, newest first (the live column, then the frozen ones)."""
        if self.live is None:
            return []
        return [self.live] + self.frozen[::-1]
