"""Discrete adjoint of the explicit-Euler / Schur-complement time loop (oracle;
test infrastructure).

Objective: the time-integrated eddy-current loss, in the FIT edge form of
sum over cells of sigma |E|^2 dV (with E = -d a / dt on conducting edges),

    J = sum_m dt e_m^T M_c e_m,   e_m = (a^m - a^{m-1}) / dt = -M_c^-1 F_m,
      = sum_m dt F_m^T M_c^-1 F_m.

Forward step (Sec. II, eqs. (ODE), (acm), one solve per step, as in
``stepper.run_explicit_euler``):

    w_m  = K_n^+ (i(t_m) X_n - K_cn^T a^{m-1})
    u_m  = [a^{m-1}; w_m],   b_m = C u_m
    F_m  = (C^T H(b_m))_c,   H(b) = M_nu(b) b   (secant Brauer law per cell)
    a^m  = a^{m-1} - dt M_c^-1 F_m.

Reverse sweep, lambda_m = dJ/da^m (total derivative through the later steps),
lambda_M = 0, for m = M .. 1:

    mu_m        = dt M_c^-1 (2 F_m - lambda_m)                 (= dJ/dF_m)
    z           = C^T J_H(b_m)^T C P_c^T mu_m,   J_H = dH/db
    v_m         = K_n^+ z_n                      (z_n = K_cn^T mu_m)
    lambda_{m-1} = lambda_m + z_c - K_cn v_m
    dJ/dM_c    += dt F_m (lambda_m - F_m) / M_c^2   (elementwise)
    dJ/dI0     += g(t_m) X_n^T v_m                  (i(t) = I0 g(t))

and dJ/dsigma_cell = h * (4-cell edge average)^T dJ/dM_kappa on conducting
edges (M_kappa = h * mean sigma of the four cells of an edge).  dt and the
edge classes are held fixed; gradients are reported for conducting cells.

J_H(b) = diag(M_nu) + diag(b) A_f dnu/db / h with A_f the face-cell average
and dnu_c/db_f = k1 k2 exp(k2 B_c^2) (P_d b)_c / (2 h^4) for the two faces of
cell c normal to d (B_c = |(P_x b, P_y b, P_z b)_c| / (2 h^2)).

Parity: pinned by central finite differences of the forward objective.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .operators import Discretization
from .pcg import pcg_jacobi
from .stepper import source_current


@dataclass
class AdjointResult:
    J: float
    grad_sigma: np.ndarray      # per cell (N^3, cell order of the problem), 0 on nonconducting cells
    grad_amplitude: float
    a_c: np.ndarray             # final state


def objective(disc: Discretization, dt, n_steps, tol=1e-13, rhs_time=0, a_c0=None, m0=0):
    """Forward run only: J = sum_m dt F_m^T M_c^-1 F_m and the final state."""
    J, _, _, _, a = _forward(disc, dt, n_steps, tol, rhs_time, a_c0, m0)
    return J, a


def _forward(disc, dt, n_steps, tol, rhs_time, a_c0, m0=0):
    p = disc.problem
    jn = disc.X_s[disc.n_idx]
    a = np.zeros(disc.n_c) if a_c0 is None else np.array(a_c0, dtype=np.float64)
    a_prev, u_full, F_all, g_all = [], [], [], []
    J = 0.0
    unit = p.with_(amplitude=1.0)
    for m in range(m0 + 1, m0 + n_steps + 1):
        t_src = (m if rhs_time == 0 else m - 1) * dt
        g = source_current(unit, t_src)
        b = p.amplitude * g * jn - disc.K_cn.T @ a
        w = pcg_jacobi(disc.K_n, b, None, disc.D, tol, 100000).x
        u = disc.full(a, w)
        F = disc.apply_K(u, u)[disc.c_idx]
        J += dt * float(F @ (F / disc.M_c))
        a_prev.append(a.copy())
        u_full.append(u)
        F_all.append(F)
        g_all.append(g)
        a = a - dt * F / disc.M_c
    return J, a_prev, u_full, (F_all, g_all), a


def face_law_jacobian(disc: Discretization, u_full):
    """J_H = d(M_nu(b) b)/db at b = C u (faces x faces, sparse)."""
    b = disc.C @ u_full
    Mnu = disc.M_nu(u_full)
    if not np.any(disc.brauer):
        return sp.diags(Mnu).tocsr()
    h = disc.h
    comps = [P @ b for P in disc._pairs]                       # (P_d b)_c
    B2 = (comps[0] ** 2 + comps[1] ** 2 + comps[2] ** 2) / (4.0 * h ** 4)
    dnu_dB2 = np.where(disc.brauer, disc.k1 * disc.k2 * np.exp(disc.k2 * B2), 0.0)
    # d nu_c / d b_f = dnu/d(B^2) * d(B_c^2)/d b_f, d(B_c^2)/d b_f = 2 (P_d b)_c P_d[c, f] / (4 h^4)
    Q = sum(sp.diags(comps[d] / (2.0 * h ** 4)) @ disc._pairs[d] for d in range(3))
    dnu_db = sp.diags(dnu_dB2) @ Q                              # cells x faces
    return (sp.diags(Mnu) + sp.diags(b / h) @ disc._Af @ dnu_db).tocsr()


def adjoint_gradient(disc: Discretization, dt, n_steps, tol=1e-13, rhs_time=0, a_c0=None,
                     nonlinear_term=True, m0=0):
    """J and dJ/d(sigma_cell), dJ/d(coil amplitude) by the reverse sweep above, over
    steps m0+1 .. m0+n_steps from a_c0.  ``nonlinear_term=False`` drops the Brauer
    derivative from J_H (used by a test to show that the term matters)."""
    J, a_prev, u_full, (F_all, g_all), a_end = _forward(disc, dt, n_steps, tol, rhs_time, a_c0, m0)
    jn = disc.X_s[disc.n_idx]
    Mc = disc.M_c
    lam = np.zeros(disc.n_c)
    gMc = np.zeros(disc.n_c)
    gI = 0.0
    for m in range(n_steps, 0, -1):
        F = F_all[m - 1]
        mu = dt * (2.0 * F - lam) / Mc
        gMc += dt * F * (lam - F) / Mc ** 2
        JH = face_law_jacobian(disc, u_full[m - 1]) if nonlinear_term else sp.diags(disc.M_nu(u_full[m - 1]))
        z = disc.C.T @ (JH.T @ (disc.C @ disc.full(a_c=mu)))
        zn = z[disc.n_idx]
        v = pcg_jacobi(disc.K_n, zn, None, disc.D, tol, 100000).x
        gI += g_all[m - 1] * float(jn @ v)
        lam = lam + z[disc.c_idx] - disc.K_cn @ v
    # M_kappa = h * Ae sigma  ->  dJ/dsigma = h Ae^T dJ/dM_kappa (conducting edges only)
    gMk = np.zeros(disc.grid.n_edges)
    gMk[disc.c_idx] = gMc
    gs = disc.h * (disc._Ae.T @ gMk)
    gs = np.where(disc.sigma > 0, gs, 0.0)
    return AdjointResult(J, gs, gI, a_end)
