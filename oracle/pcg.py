"""Jacobi-preconditioned conjugate gradients for K_n a_p = j_p (oracle; test infrastructure).

Sec. II evaluates the pseudo-inverse K_n^+ of the singular nonconducting
curl-curl matrix with PCG, relying on the weak-gauging property of Krylov
solvers: for a consistent right-hand side (b in range(K_n)) CG started anywhere
converges to a solution; ``K_cn x`` and ``C x`` are unique even though ``x``
is not (Sec. II, text after eq. (DAE); Sec. III, eq. (mrhs)).

Recurrences (Hestenes-Stiefel form, preconditioner D = diag(K_n)):

    r = b - K x,  z = D^-1 r,  p = z,  rho = r.z
    repeat: q = K p; alpha = rho / p.q; x += alpha p; r -= alpha q
            stop when ||r||_2 <= tol ||b||_2 (confirmed on the true residual
            b - K x; if that fails, restart the recurrences from it)
            z = D^-1 r; rho' = r.z; beta = rho'/rho; p = z + beta p

The iteration count is the number of products K p inside the loop.  If
``||b|| = 0`` the solution is ``x = 0`` after 0 iterations.  ``p.q <= 0`` is
a breakdown.  Parity: pinned (dense pseudo-inverse on 4^3 grids, Krylov
invariants; see the tests).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STATUS_OK = 0
STATUS_NOT_CONVERGED = -4
STATUS_BREAKDOWN = -5
STATUS_NAN = -6


@dataclass
class PcgResult:
    x: np.ndarray
    iterations: int
    relres: float          # true relative residual ||b - K x|| / ||b||
    status: int
    Kx: np.ndarray         # K x from the final true-residual evaluation


def pcg_jacobi(K, b, x0=None, D=None, tol=1e-10, maxit=10000) -> PcgResult:
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    Dinv = 1.0 / (K.diagonal() if D is None else D)
    nb = np.linalg.norm(b)
    if not np.isfinite(nb) or not np.all(np.isfinite(x)):
        return PcgResult(x, 0, float("nan"), STATUS_NAN, np.full(n, np.nan))
    if nb == 0.0:
        x = np.zeros(n)
        return PcgResult(x, 0, 0.0, STATUS_OK, np.zeros(n))
    Kx = K @ x
    r = b - Kx
    if np.linalg.norm(r) <= tol * nb:
        return PcgResult(x, 0, np.linalg.norm(r) / nb, STATUS_OK, Kx)
    z = Dinv * r
    p = z.copy()
    rho = r @ z
    it = 0
    while it < maxit:
        q = K @ p
        pq = p @ q
        it += 1
        if not np.isfinite(pq):
            return PcgResult(x, it, float("nan"), STATUS_NAN, K @ x)
        if pq <= 0.0:
            Kx = K @ x
            return PcgResult(x, it, np.linalg.norm(b - Kx) / nb, STATUS_BREAKDOWN, Kx)
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= tol * nb:
            Kx = K @ x
            rt = b - Kx
            if np.linalg.norm(rt) <= tol * nb:
                return PcgResult(x, it, np.linalg.norm(rt) / nb, STATUS_OK, Kx)
            r = rt                       # restart from the true residual
            z = Dinv * r
            p = z.copy()
            rho = r @ z
            continue
        z = Dinv * r
        rho_new = r @ z
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    Kx = K @ x
    return PcgResult(x, it, np.linalg.norm(b - Kx) / nb, STATUS_NOT_CONVERGED, Kx)
