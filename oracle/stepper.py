"""Explicit Euler on the Schur-complement ODE (oracle; test infrastructure).

Sec. II, eq. (ODE):  M_c d/dt a_c + K_S(a_c) a_c = -K_cn K_n^+ j_sn  with the
generalised Schur complement K_S(a_c) = K_c(a_c) - K_cn K_n^+ K_cn^T (eq. (SC)).

Explicit Euler (eq. (acm), with the sign of the source term taken from eq.
(ODE); the printed (acm) carries a "+" in front of K_cn K_n^+ j that
contradicts (ODE) and (DAE)):

    a_c^m = a_c^{m-1} - dt M_c^-1 [ K_S(a_c^{m-1}) a_c^{m-1} + K_cn K_n^+ j^m ].

By linearity of K_n^+ on consistent right-hand sides this needs one solve per
step:  w = K_n^+ (j^m - K_cn^T a_c^{m-1})  (which is a_n of eq. (a_n)), then
K_S a_c + K_cn K_n^+ j = K_c a_c + K_cn w = (K(a) [a_c; w])_c.  The mode
``literal=True`` instead solves for j^m and for K_cn^T a_c^{m-1} separately
(the separate right-hand sides listed after eq. (mrhs)) and subtracts.  With the
SPE start each right-hand-side type keeps its own window of past solutions
(Sec. III: the start vector of K_n a_p = j_p projects onto solutions a_p of the
same type), so each solve starts from its own Galerkin projection; other start
modes solve the two types from zero.

Source time level: ``rhs_time = 0`` uses j^m = i(m dt) X_s as printed in
(acm); ``rhs_time = 1`` uses i((m-1) dt).

Step bound (eq. (CFL)): dt <= 2 / lambda_max(M_c^-1 K_S(a_c)); lambda_max by
the power method on the symmetric form M_c^-1/2 K_S M_c^-1/2 at a_c = 0.

Parity: pinned (closed-form amplification on a discrete eigenmode, DC steady
state against the magnetostatic solve, dense eigenvalues on 4^3 grids).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .mrhs import CspeBasis, pod_start, spe_start
from .operators import Discretization
from .pcg import STATUS_OK, pcg_jacobi

START_ZERO, START_PREV, START_SPE, START_POD, START_CSPE = 0, 1, 2, 3, 4


def source_current(problem, t):
    """Coil current i_S(t): sinusoid or the 1 - exp(-t/tau) ramp of Sec. IV."""
    if problem.waveform == 0:
        return problem.amplitude * np.sin(2.0 * np.pi * problem.freq * t)
    return problem.amplitude * (1.0 - np.exp(-t / problem.tau))


def schur_apply(disc: Discretization, u, tol=1e-12, maxit=100000):
    """K_S(0) u = K_c(0) u - K_cn K_n^+ K_cn^T u (one PCG solve)."""
    Kc = disc.K_c(np.zeros(disc.n_c))
    sol = pcg_jacobi(disc.K_n, disc.K_cn.T @ u, None, disc.D, tol, maxit)
    return Kc @ u - disc.K_cn @ sol.x


def lambda_max_power(disc: Discretization, v0, tol_pcg=1e-12, rtol=1e-8, maxit=2000):
    """Power method on S = M_c^-1/2 K_S(0) M_c^-1/2; Rayleigh quotient estimate.

    Returns (lambda_max, iterations)."""
    Kc = disc.K_c(np.zeros(disc.n_c))
    s = 1.0 / np.sqrt(disc.M_c)
    v = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    lam_old = None
    lam = 0.0
    for it in range(1, maxit + 1):
        u = s * v
        sol = pcg_jacobi(disc.K_n, disc.K_cn.T @ u, None, disc.D, tol_pcg, 100000)
        z = s * (Kc @ u - disc.K_cn @ sol.x)
        lam = float(v @ z)
        v = z / np.linalg.norm(z)
        if lam_old is not None and abs(lam - lam_old) < rtol * abs(lam):
            return lam, it
        lam_old = lam
    return lam, maxit


def dt_from_lambda(lam, cfl_factor=0.9):
    return cfl_factor * 2.0 / lam


def dt_gershgorin(disc: Discretization, cfl_factor=0.9):
    """A safe step from a Gershgorin bound: K_S <= K_c in the Loewner order,
    so lambda_max(M_c^-1 K_S) <= max_i sum_j |K_c,ij| / sqrt(M_i M_j)."""
    Kc = disc.K_c(np.zeros(disc.n_c)).tocoo()
    s = 1.0 / np.sqrt(disc.M_c)
    vals = np.abs(Kc.data) * s[Kc.row] * s[Kc.col]
    bound = np.bincount(Kc.row, weights=vals, minlength=disc.n_c).max()
    return cfl_factor * 2.0 / bound


@dataclass
class StepRecord:
    iterations: int
    relres: float
    start_relres: float
    rank: int
    status: int
    pod_info: float = float("nan")


@dataclass
class RunResult:
    a_c: np.ndarray
    w: np.ndarray
    records: list = field(default_factory=list)

    @property
    def iterations(self):
        return np.array([r.iterations for r in self.records])


def run_explicit_euler(disc: Discretization, dt, n_steps, start_mode=START_ZERO,
                       spe_depth=8, pod_snapshots=20, tol=1e-10, maxit=100000,
                       rhs_time=0, eps_lin=1e-10, eps_pod=1e-4, a_c0=None,
                       m0=0, literal=False, history=None, source_scale=1.0, cspe_period=25):
    """Run ``n_steps`` explicit Euler steps starting after step ``m0``.

    ``history`` (newest first) may carry earlier PCG solutions for the start
    vector modes; it is updated in place when given.
    """
    p = disc.problem
    a_c = np.zeros(disc.n_c) if a_c0 is None else np.array(a_c0, dtype=np.float64)
    hist = history if history is not None else []
    hist_s, hist_c = [], []            # literal SPE: past solutions per right-hand-side type
    cspe = CspeBasis(cspe_period, spe_depth)
    depth = max(spe_depth if start_mode == START_SPE else pod_snapshots if start_mode == START_POD else 1, 1)
    jn = disc.X_s[disc.n_idx]
    records = []
    w = np.zeros(disc.n_n)
    for m in range(m0 + 1, m0 + n_steps + 1):
        t_src = (m if rhs_time == 0 else m - 1) * dt
        i_t = source_scale * source_current(p, t_src)
        b = i_t * jn - disc.K_cn.T @ a_c
        rank, info_ratio = 0, float("nan")
        if start_mode == START_CSPE:
            x0, rank = spe_start(disc.K_n, cspe.window(), b, eps_lin)
        elif start_mode == START_ZERO or not hist:
            x0 = np.zeros(disc.n_n)
        elif start_mode == START_PREV:
            x0 = hist[0].copy()
        elif start_mode == START_SPE:
            x0, rank = spe_start(disc.K_n, hist[:spe_depth], b, eps_lin)
        elif start_mode == START_POD:
            x0, rank, _sig, info_ratio = pod_start(disc.K_n, hist[:pod_snapshots], b, eps_pod)
        else:
            raise ValueError("unknown start mode")
        nb = np.linalg.norm(b)
        r0 = np.linalg.norm(b - disc.K_n @ x0) / nb if nb > 0 else 0.0
        if literal:
            b1, b2 = i_t * jn, disc.K_cn.T @ a_c
            x1 = x2 = None
            rank = 0
            if start_mode == START_SPE:
                x1, r1 = spe_start(disc.K_n, hist_s[:spe_depth], b1, eps_lin) if hist_s else (None, 0)
                x2, r2 = spe_start(disc.K_n, hist_c[:spe_depth], b2, eps_lin) if hist_c else (None, 0)
                rank = r1 + r2
            s1 = pcg_jacobi(disc.K_n, b1, x1, disc.D, tol, maxit)
            s2 = pcg_jacobi(disc.K_n, b2, x2, disc.D, tol, maxit)
            w = s1.x - s2.x
            if start_mode == START_SPE:
                hist_s.insert(0, s1.x.copy())
                hist_c.insert(0, s2.x.copy())
                del hist_s[spe_depth:], hist_c[spe_depth:]
            rec = StepRecord(s1.iterations + s2.iterations, max(s1.relres, s2.relres), r0, rank,
                             s1.status if s1.status != STATUS_OK else s2.status)
        else:
            sol = pcg_jacobi(disc.K_n, b, x0, disc.D, tol, maxit)
            w = sol.x
            rec = StepRecord(sol.iterations, sol.relres, r0, rank, sol.status, info_ratio)
        records.append(rec)
        a_full = disc.full(a_c, w)
        F = disc.apply_K(a_full, a_full)[disc.c_idx]
        a_c = a_c - dt * F / disc.M_c
        hist.insert(0, w.copy())
        del hist[depth:]
        cspe.push(w)
    return RunResult(a_c, w, records)
