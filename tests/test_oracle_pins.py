"""Pins of the FP64 oracle against facts fixed by the mathematics, independent
of the oracle's own code: exact integer identities, closed forms, dense
brute force on tiny grids and special cases with known answers."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import workloads as W
from oracle.mrhs import galerkin_start
from oracle.pcg import STATUS_BREAKDOWN, STATUS_OK
from tests.helpers import dense, kn_null_vectors, rel

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


# --- topology -----------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 3, 5])
def test_curl_of_gradient_and_div_of_curl_vanish_exactly(N):
    g = O.FitGrid(N)
    G, C, S = g.gradient(), g.curl(), g.divergence()
    assert G.shape == (3 * N * (N + 1) ** 2, (N + 1) ** 3)
    assert C.shape == (3 * N * N * (N + 1), 3 * N * (N + 1) ** 2)
    assert abs(C @ G).max() == 0          # discrete curl grad = 0
    assert abs(S @ C).max() == 0          # discrete div curl = 0
    assert np.all(np.diff(C.indptr) == 4) and set(np.unique(C.data)) == {-1.0, 1.0}
    assert np.all(np.diff(G.indptr) == 2) and np.all(G.sum(axis=1) == 0)


def test_face_loop_orientation_is_right_handed():
    # uniform B = B0 z from A = B0/2 (-y, x, 0): every z-face carries B0 h^2,
    # x/y faces carry nothing, |B| = B0 in every cell (Stokes)
    p = W.config_linear_block(N=6)
    d = O.Discretization(p)
    comp, i, j, k = d.grid.edge_coords()
    h, B0 = p.h, 0.37
    a = np.where(comp == 0, -0.5 * B0 * (j * h) * h, np.where(comp == 1, 0.5 * B0 * (i * h) * h, 0.0))
    b = d.C @ a
    g = d.grid
    assert np.allclose(b[g.fz0:], B0 * h * h, rtol=1e-12, atol=0)
    assert np.allclose(b[:g.fz0], 0.0, atol=1e-12 * B0 * h * h)
    assert np.allclose(d.cell_flux_density(a), B0, rtol=1e-12)


def test_coil_current_is_divergence_free():
    for p in (W.config_linear_block(), W.scaled_nonlinear(24)):
        d = O.Discretization(p)
        L = p.coil_i1 - p.coil_i0
        assert np.count_nonzero(d.X_s) == 4 * L
        assert abs(d.G.T @ d.X_s).max() == 0


def test_edge_classes_of_a_block():
    # an s^3 conducting block has 3 s (s+1)^2 edges, all conducting
    for N, s in ((16, 4), (12, 3)):
        p = W.config_linear_block(N=N)
        d = O.Discretization(p)
        s = int((p.sigma_cell > 0).sum() ** (1 / 3) + 0.5)
        assert d.n_c == 3 * s * (s + 1) ** 2
        assert d.n_c + d.n_n == 3 * N * (N - 1) ** 2


def test_material_averages():
    p = W.config_linear_block(N=8)
    p.sigma_cell[:] = 0.0
    p.sigma_cell[3, 3, 3] = 8.0e6            # a single conducting cell
    d = O.Discretization(p)
    # its 12 edges each touch it once: M_kappa = h sigma / 4
    assert d.n_c == 12
    assert np.allclose(d.M_c, p.h * 8.0e6 / 4.0, rtol=1e-15)
    # a fully interior edge of a uniform material gets h sigma
    p2 = W.config_linear_block(N=8)
    p2.sigma_cell[:] = 0.0
    p2.sigma_cell[3:5, 3:5, 3:5] = 3.0e6
    d2 = O.Discretization(p2)
    assert np.isclose(d2.M_kappa[d2.grid.ex(3, 4, 4)], p.h * 3.0e6, rtol=1e-15)


def test_brauer_reluctivity_values():
    d = O.Discretization(W.scaled_nonlinear(8))
    assert d.brauer_nu(0.0) == pytest.approx(400.0, rel=1e-15)          # k1 + k3
    assert d.brauer_nu(1.0) == pytest.approx(429.4815, abs=5e-4)        # 3.8 e^2.17 + 396.2
    assert d.brauer_nu(2.0) == pytest.approx(22755.6, abs=0.1)          # 3.8 e^8.68 + 396.2


def test_curl_curl_of_quadratic_potential():
    # A = (0, 0, x^2): curl curl A = (0, 0, -2); FIT gives -2 nu0 h^2 per z-edge
    p = W.config_linear_block(N=7)
    p.sigma_cell[:] = 0.0
    d = O.Discretization(p)
    comp, i, j, k = d.grid.edge_coords()
    h = p.h
    a = np.where(comp == 2, h * (i * h) ** 2, 0.0)
    Ka = d.apply_K(np.zeros_like(a), a)
    sel = (comp == 2) & (i >= 1) & (i <= p.N - 1)
    assert np.allclose(Ka[sel], -2.0 * p.nu0 * h * h, rtol=1e-9)
    inner = (comp != 2) & ~d.dirichlet
    assert np.allclose(Ka[inner], 0.0, atol=1e-9 * p.nu0 * h * h)


# --- operator blocks --------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_kn_symmetric_psd_with_predicted_nullity(seed):
    p = W.random_problem(seed, N=4)
    d = O.Discretization(p)
    Kn = dense(d.K_n)
    assert np.array_equal(Kn, Kn.T)
    lam = np.linalg.eigvalsh(Kn)
    assert lam.min() >= -1e-12 * lam.max()
    nullity = int(np.sum(lam < 1e-10 * lam.max()))
    vecs, comps = kn_null_vectors(d)
    assert nullity == len(vecs)
    V = np.column_stack(vecs)
    assert np.linalg.matrix_rank(V) == len(vecs)
    assert abs(d.K_n @ V).max() <= 1e-14 * abs(d.K_n).max()


@pytest.mark.parametrize("seed", [0, 5])
def test_right_hand_sides_are_consistent(seed):
    p = W.random_problem(seed, N=5)
    d = O.Discretization(p)
    vecs, _ = kn_null_vectors(d)
    a_c = W.random_vector(seed, d.n_c)
    for b in (d.X_s[d.n_idx], d.K_cn.T @ a_c):
        nb = np.linalg.norm(b)
        for v in vecs:
            assert abs(v @ b) <= 1e-14 * nb * np.linalg.norm(v)


def test_kn_and_kcn_do_not_depend_on_the_state():
    p = W.scaled_nonlinear(8, amplitude=1e3)
    d = O.Discretization(p)
    a = W.random_vector(3, d.grid.n_edges) * 1e-6       # |B| of order 1 T
    assert np.max(d.cell_flux_density(a)[d.brauer]) > 0.5
    K = d.K(a)
    assert abs(K[d.n_idx][:, d.n_idx] - d.K_n).max() == 0
    assert abs(K[d.c_idx][:, d.n_idx] - d.K_cn).max() == 0
    assert abs(K[d.c_idx][:, d.c_idx] - d.K_c(np.zeros(d.n_c))).max() > 0


# --- PCG ----------------------------------------------------------------------------
def test_pcg_closed_forms_on_spd_matrix():
    import scipy.sparse as sp
    n = 60
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    b = W.random_vector(1, n)
    res = O.pcg_jacobi(A, b, tol=1e-13)
    assert res.status == STATUS_OK and res.iterations <= n
    assert rel(res.x, np.linalg.solve(A.toarray(), b)) < 1e-11
    assert O.pcg_jacobi(A, np.zeros(n)).iterations == 0
    assert O.pcg_jacobi(A, b, x0=np.linalg.solve(A.toarray(), b), tol=1e-12).iterations == 0
    # Jacobi with a constant diagonal: same iterates as plain CG
    res2 = O.pcg_jacobi(A, b, D=np.full(n, 1.0), tol=1e-13)
    assert res2.iterations == res.iterations and rel(res2.x, res.x) < 1e-12
    assert O.pcg_jacobi(-sp.identity(n, format="csr"), b).status == STATUS_BREAKDOWN


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pcg_matches_dense_pseudo_inverse(seed):
    p = W.random_problem(seed, N=4)
    d = O.Discretization(p)
    Kp = np.linalg.pinv(dense(d.K_n), rcond=1e-12)
    y = W.random_vector(seed + 10, d.n_n)
    for b in (d.K_n @ y, d.X_s[d.n_idx], d.K_cn.T @ W.random_vector(seed, d.n_c)):
        res = O.pcg_jacobi(d.K_n, b, tol=1e-13)
        assert res.status == STATUS_OK
        xp = Kp @ b
        assert rel(d.K_cn @ res.x, d.K_cn @ xp) < 1e-9
        assert np.linalg.norm(d.K_n @ (res.x - xp)) <= 1e-10 * np.linalg.norm(b)


# --- Schur complement, explicit Euler, CFL ---------------------------------------------
def _dense_schur(d):
    Kn = dense(d.K_n)
    Kcn = dense(d.K_cn)
    Kc = dense(d.K_c(np.zeros(d.n_c)))
    return Kc - Kcn @ np.linalg.pinv(Kn, rcond=1e-12) @ Kcn.T


def test_power_iteration_matches_dense_lambda_max():
    p = W.config_linear_block(N=6)
    d = O.Discretization(p)
    KS = _dense_schur(d)
    lam_dense = sla.eigh(0.5 * (KS + KS.T), np.diag(d.M_c), eigvals_only=True).max()
    lam, it = O.lambda_max_power(d, W.power_start_vector(d.n_c), tol_pcg=1e-13, rtol=1e-12, maxit=20000)
    assert lam == pytest.approx(lam_dense, rel=1e-8)


def test_gershgorin_step_is_safe_and_local():
    # the Gershgorin step never exceeds the CFL step of the dense Schur spectrum (eq. (CFL)) ...
    p = W.scaled_nonlinear(8)
    d = O.Discretization(p)
    KS = _dense_schur(d)
    lam_dense = sla.eigh(0.5 * (KS + KS.T), np.diag(d.M_c), eigvals_only=True).max()
    assert O.dt_gershgorin(d) <= 0.9 * 2.0 / lam_dense
    # ... and depends only on the local rows around the conductor, so it is the same at every
    # size of the scaled iron family (which lets a large run take it from a small grid)
    dts = [O.dt_gershgorin(O.Discretization(W.scaled_nonlinear(n))) for n in (16, 24, 32)]
    assert dts[0] == dts[1] == dts[2]


@pytest.mark.parametrize("which", ["top", "middle"])
def test_explicit_euler_amplification_of_an_eigenmode(which):
    p = W.config_linear_block(N=6).with_(amplitude=0.0)
    d = O.Discretization(p)
    KS = _dense_schur(d)
    lam, V = sla.eigh(0.5 * (KS + KS.T), np.diag(d.M_c))
    dt = 0.9 * 2.0 / lam.max()
    idx = len(lam) - 1 if which == "top" else len(lam) // 2
    v = V[:, idx]
    n = 7
    res = O.run_explicit_euler(d, dt, n, tol=1e-14, a_c0=v)
    factor = (1.0 - dt * lam[idx]) ** n
    if which == "top":
        assert (1.0 - dt * lam[idx]) == pytest.approx(-0.8, rel=1e-12)
    assert rel(res.a_c, factor * v) < 1e-10


def test_energy_norm_decays_without_source():
    p = W.config_linear_block(N=6).with_(amplitude=0.0)
    d = O.Discretization(p)
    lam = O.lambda_max_power(d, W.power_start_vector(d.n_c), tol_pcg=1e-13, rtol=1e-10)[0]
    dt = O.dt_from_lambda(lam)
    a = W.random_vector(7, d.n_c)
    norms = []
    for m in range(6):
        a = O.run_explicit_euler(d, dt, 1, tol=1e-13, a_c0=a).a_c
        norms.append(np.sqrt(a @ (d.M_c * a)))
    assert all(n2 <= n1 * (1 + 1e-12) for n1, n2 in zip(norms, norms[1:]))


def test_dc_steady_state_equals_magnetostatics():
    # constant current (ramp with a vanishing time constant) on a linear conductor
    p = W.config_linear_block(N=6).with_(waveform=1, tau=1e-30, amplitude=2.0)
    d = O.Discretization(p)
    Kn, Kcn = dense(d.K_n), dense(d.K_cn)
    Kp = np.linalg.pinv(Kn, rcond=1e-12)
    KS = _dense_schur(d)
    j = p.amplitude * d.X_s[d.n_idx]
    a_c = np.linalg.solve(KS, -Kcn @ (Kp @ j))          # fixed point of eq. (ODE)
    a_n = Kp @ (j - Kcn.T @ a_c)                        # eq. (a_n)
    # magnetostatics on all interior edges: K a = j, flux density unique
    free = np.flatnonzero(~d.dirichlet)
    Kf = dense(d.K(np.zeros(d.grid.n_edges)))[np.ix_(free, free)]
    a_ms = np.zeros(d.grid.n_edges)
    a_ms[free] = np.linalg.pinv(Kf, rcond=1e-12) @ (p.amplitude * d.X_s[free])
    assert rel(d.C @ d.full(a_c, a_n), d.C @ a_ms) < 1e-9
    # the stepper leaves the DC state unchanged (fails by O(1) with the printed + sign)
    dt = 1e-9
    res = O.run_explicit_euler(d, dt, 3, tol=1e-14, a_c0=a_c, m0=5)
    assert rel(res.a_c, a_c) < 1e-9


# --- start vectors ----------------------------------------------------------------------
def _smooth_window(d, depth, seed):
    base = [W.random_vector(seed + q, d.n_n) for q in range(3)]
    return [base[0] + 0.1 * t * base[1] + 0.01 * t * t * base[2] for t in range(depth)]


def test_spe_start_galerkin_and_exact_recovery():
    p = W.config_linear_block(N=8)
    d = O.Discretization(p)
    win = _smooth_window(d, 6, 11)
    Q = O.mgs_orthonormal_basis(win)
    assert Q.shape[1] == 3                       # quadratic family: rank 3
    assert np.abs(Q.T @ Q - np.eye(3)).max() < 1e-12
    b = d.K_n @ W.random_vector(99, d.n_n)
    x0, rank = O.spe_start(d.K_n, win, b)
    assert rank == 3
    assert np.abs(Q.T @ (b - d.K_n @ x0)).max() <= 1e-10 * np.linalg.norm(b)
    # a right-hand side produced by a vector of the span is reproduced exactly
    s = 0.3 * win[0] - 2.0 * win[4]
    b2 = d.K_n @ s
    x2, _ = O.spe_start(d.K_n, win, b2)
    assert np.linalg.norm(b2 - d.K_n @ x2) <= 1e-10 * np.linalg.norm(b2)
    assert O.pcg_jacobi(d.K_n, b2, x2, d.D, tol=1e-9).iterations == 0
    # the Galerkin start minimises the energy error over the span
    xs = O.pcg_jacobi(d.K_n, b, None, d.D, tol=1e-13).x
    e0 = xs - x0
    for t in (1e-3, -1e-3):
        e1 = xs - (x0 + t * Q[:, 1])
        assert e1 @ (d.K_n @ e1) > e0 @ (d.K_n @ e0)


class _CountEigh:
    """Counts calls of numpy.linalg.eigh (the small solve's fallback branch)."""

    def __init__(self, monkeypatch):
        self.calls = 0
        real = np.linalg.eigh

        def wrapped(*a, **k):
            self.calls += 1
            return real(*a, **k)
        monkeypatch.setattr(np.linalg, "eigh", wrapped)


def test_small_solve_fallback_on_a_singular_system(monkeypatch):
    # Cholesky fails on a singular H; the fallback keeps the eigenspace above
    # 1e-14 lambda_max and returns the minimum-norm least-squares solution there
    from oracle.mrhs import solve_small_spd
    rng = np.random.default_rng(7)
    V, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([5.0, 2.0, 0.5, 1e-3, 0.0, 0.0])
    H = (V * lam) @ V.T
    H[1, 0] += 1e-17                                     # asymmetric by rounding: symmetrised first
    g = rng.standard_normal(6)
    count = _CountEigh(monkeypatch)
    y = solve_small_spd(H, g)
    assert count.calls == 1                              # the fallback branch ran
    # the minimum-norm least-squares solution by an SVD-based pseudo-inverse (a different routine)
    Hs = 0.5 * (H + H.T)
    y_pinv = np.linalg.pinv(Hs, rcond=1e-12) @ g
    y_lstsq = np.linalg.lstsq(Hs, g, rcond=1e-12)[0]
    assert rel(y, y_pinv) < 1e-10 and rel(y, y_lstsq) < 1e-10
    # Galerkin orthogonality on the kept eigenspace, nothing in the dropped one
    Vk, V0 = V[:, :4], V[:, 4:]
    assert np.abs(Vk.T @ (g - Hs @ y)).max() <= 1e-12 * np.linalg.norm(g)
    assert np.abs(V0.T @ y).max() <= 1e-12 * np.linalg.norm(y)
    # a wrong truncation (dropping the 1e-3 eigenvalue) would change y by its component
    assert abs(Vk[:, 3] @ y - (Vk[:, 3] @ g) / 1e-3) <= 1e-8 * abs((Vk[:, 3] @ g) / 1e-3)


def test_galerkin_start_fallback_agrees_with_cholesky(monkeypatch):
    # (a) on a nonsingular SPE Galerkin system the eigen-solve branch must give the
    # Cholesky solution: Cholesky is made to fail on purpose
    p = W.config_linear_block(N=6)
    d = O.Discretization(p)
    Q = O.mgs_orthonormal_basis(_smooth_window(d, 3, 21))
    b = d.K_n @ W.random_vector(98, d.n_n)
    x_chol = galerkin_start(d.K_n, Q, b)
    count = _CountEigh(monkeypatch)

    def no_cholesky(*a, **k):
        raise np.linalg.LinAlgError("forced")
    with monkeypatch.context() as m:
        m.setattr(np.linalg, "cholesky", no_cholesky)
        x_eig = galerkin_start(d.K_n, Q, b)
    assert count.calls == 1
    assert rel(x_eig, x_chol) < 1e-10
    # (b) a basis column that K_n annihilates exactly (here: zero) makes U^T K_n U
    # singular, Cholesky fails by itself, and the fallback projects on the other columns
    U = np.column_stack([Q, np.zeros(d.n_n)])
    x0 = galerkin_start(d.K_n, U, b)
    assert count.calls == 2
    assert rel(d.K_n @ x0, d.K_n @ x_chol) < 1e-10
    assert np.abs(U.T @ (b - d.K_n @ x0)).max() <= 1e-10 * np.linalg.norm(b)


def test_pod_recovers_constructed_singular_values():
    rng = np.random.default_rng(5)
    n, m = 400, 8
    U, _ = np.linalg.qr(rng.standard_normal((n, m)))
    V, _ = np.linalg.qr(rng.standard_normal((m, m)))
    sig = np.array([3.0, 1.0, 2e-2, 5e-3, 1e-3, 5e-4, 2e-4, 1e-6])
    X = (U * sig) @ V.T
    import scipy.sparse as sp
    A = sp.diags(np.linspace(1.0, 5.0, n)).tocsr()
    b = A @ rng.standard_normal(n)
    x0, k, s_out, info = O.pod_start(A, [X[:, q] for q in range(m)], b)
    assert np.allclose(s_out, np.sort(sig)[::-1], rtol=1e-10, atol=1e-14)
    assert k == 6                                  # sigma_i / 3 >= 1e-4 keeps six
    assert info == pytest.approx(sig[:6].sum() / sig.sum(), rel=1e-12)
    Uk = U[:, :6]
    assert np.abs(Uk.T @ (b - A @ x0)).max() <= 1e-10 * np.linalg.norm(b)
    assert rel(x0, galerkin_start(A, Uk, b)) < 1e-10
    x0n, *_ = O.pod_start(A, [-X[:, q] for q in range(m)], b)
    assert rel(x0n, x0) < 1e-12


def test_start_vectors_do_not_change_the_result():
    p = W.config_linear_block(N=8)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 30, start_mode=0, tol=1e-12)
    for mode in (1, 2, 3, 4):
        r = O.run_explicit_euler(d, dt, 30, start_mode=mode, tol=1e-12, spe_depth=4, pod_snapshots=6,
                                 cspe_period=5)
        assert rel(r.a_c, ref.a_c) < 1e-8
    lit = O.run_explicit_euler(d, dt, 30, start_mode=0, tol=1e-12, literal=True)
    assert rel(lit.a_c, ref.a_c) < 1e-8
    it = {m: O.run_explicit_euler(d, dt, 30, start_mode=m, tol=1e-12, spe_depth=4, pod_snapshots=6,
                                  cspe_period=5).iterations.sum()
          for m in (0, 2, 4)}
    assert it[2] < it[0] and it[4] < it[0]


def test_literal_spe_keeps_a_history_per_right_hand_side_type():
    # the separate right-hand sides of eq. (mrhs), each started from the SPE projection on
    # its own past solutions: the same a_c as the fused solve; the coil term's solutions are
    # multiples of K_n^+ X_s, so once one is known its start vector is exact (rank 1) and
    # costs no iteration; and the per-type starts save iterations over zero starts
    p = W.scaled_nonlinear(8, amplitude=900.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 20, start_mode=0, tol=1e-12)
    lit0 = O.run_explicit_euler(d, dt, 20, start_mode=0, tol=1e-12, literal=True)
    lit = O.run_explicit_euler(d, dt, 20, start_mode=2, spe_depth=4, tol=1e-12, literal=True)
    assert rel(lit.a_c, ref.a_c) < 1e-8 and rel(lit0.a_c, ref.a_c) < 1e-8
    assert lit.iterations.sum() < lit0.iterations.sum()
    # coil-type solve alone, with its own history, after the first step: exact start
    jn = d.X_s[d.n_idx]
    u = O.pcg_jacobi(d.K_n, jn, None, d.D, 1e-13).x
    from oracle.mrhs import spe_start
    x0, rank = spe_start(d.K_n, [0.3 * u, -0.7 * u], 2.5 * jn)
    assert rank == 1 and rel(x0, 2.5 * u) < 1e-10


def test_cspe_column_schedule():
    # the live column is the newest solution; the solutions of steps P, 2P, ... are frozen
    # until the basis holds `depth` columns (Sec. III cascaded SPE, Sec. IV growth below 20)
    from oracle.mrhs import CspeBasis
    c = CspeBasis(period=3, depth=4)
    seen = {}
    for step in range(1, 15):
        c.push(np.array([float(step)]))
        seen[step] = [int(v[0]) for v in c.window()]
    assert seen[1] == [1] and seen[3] == [3]
    assert seen[4] == [4, 3] and seen[6] == [6, 3]
    assert seen[7] == [7, 6, 3] and seen[10] == [10, 9, 6, 3]
    assert seen[14] == [14, 9, 6, 3]                     # depth reached: only the live column moves
    c1 = CspeBasis(period=3, depth=1)
    for step in range(1, 8):
        c1.push(np.array([float(step)]))
    assert [int(v[0]) for v in c1.window()] == [7]


def test_mirror_symmetry_of_the_field():
    # block and coil are symmetric under i -> N-1-i (cells) / x -> N - x:
    # the x-face flux pattern must be mirrored with the same sign for B_x -> -B_x
    p = W.config_linear_block(N=16)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    res = O.run_explicit_euler(d, dt, 5, tol=1e-13)
    B = d.cell_flux_density(d.full(res.a_c, res.w)).reshape(p.N, p.N, p.N)
    assert np.allclose(B, B[:, :, ::-1], rtol=1e-8, atol=1e-12 * B.max())
    assert np.allclose(B, B[:, ::-1, :], rtol=1e-8, atol=1e-12 * B.max())
    assert np.allclose(B, np.swapaxes(B, 1, 2), rtol=1e-8, atol=1e-12 * B.max())


def test_source_time_level_of_the_first_step():
    # from a_c = 0 the first step is a_c^1 = -dt M_c^-1 K_cn K_n^+ j with
    # j = i(dt) X_s for the printed j^m (rhs_time 0) and i(0) X_s = 0 for j^{m-1}
    p = W.config_linear_block(N=6)
    d = O.Discretization(p)
    dt = 2.5e-4
    Kp = np.linalg.pinv(dense(d.K_n), rcond=1e-12)
    j = p.amplitude * math.sin(2 * math.pi * p.freq * dt) * d.X_s[d.n_idx]
    expect = -dt * (dense(d.K_cn) @ (Kp @ j)) / d.M_c
    r0 = O.run_explicit_euler(d, dt, 1, rhs_time=0, tol=1e-14)
    r1 = O.run_explicit_euler(d, dt, 1, rhs_time=1, tol=1e-14)
    assert rel(r0.a_c, expect) < 1e-9
    assert np.all(r1.a_c == 0.0)
