"""Pins of the oracle's discrete adjoint (eddy-current loss gradient): the face-law
Jacobian against a directional difference of the Brauer law, the reverse sweep
against central differences of the forward objective (conductivities with the
nonlinear term active, coil amplitude), and the objective against its definition
on the state trajectory."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import adjoint as A
from oracle.stepper import run_explicit_euler

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _problem(amp=2000.0):
    p = W.scaled_nonlinear(8, amplitude=amp)
    d = O.Discretization(p)
    return p, d, O.dt_gershgorin(d)


def _with_sigma(p, cell, rel):
    s = p.sigma_cell.copy().reshape(-1)
    s[cell] *= 1.0 + rel
    return p.with_(sigma_cell=s.reshape(p.sigma_cell.shape))


def test_face_law_jacobian_directional_derivative():
    p, d, _ = _problem()
    u = d.full(a_c=3e-7 * W.random_vector(7, d.n_c))
    du = d.full(a_c=W.random_vector(8, d.n_c))
    B = d.cell_flux_density(u)[d.brauer]
    assert 0.3 < B.max() < 2.3                      # the Brauer law is in its nonlinear range
    eps = 1e-7 * np.linalg.norm(u) / np.linalg.norm(du)

    def H(v):
        return d.M_nu(v) * (d.C @ v)
    fd = (H(u + eps * du) - H(u - eps * du)) / (2.0 * eps)
    jac = A.face_law_jacobian(d, u) @ (d.C @ du)
    assert np.linalg.norm(jac - fd) <= 1e-7 * np.linalg.norm(fd)
    lin = d.M_nu(u) * (d.C @ du)                    # without the derivative of nu
    assert np.linalg.norm(lin - fd) > 1e-4 * np.linalg.norm(fd)


def test_sigma_gradient_matches_central_differences_with_brauer_active():
    p, d, dt = _problem()
    a0 = 3e-7 * W.random_vector(7, d.n_c)
    steps, h = 10, 1e-6
    r = A.adjoint_gradient(d, dt, steps, a_c0=a0)
    r_lin = A.adjoint_gradient(d, dt, steps, a_c0=a0, nonlinear_term=False)
    cells = np.flatnonzero(d.sigma > 0)
    for c in cells[[0, len(cells) // 3, len(cells) // 2, -1]]:
        jp = A.objective(O.Discretization(_with_sigma(p, c, h)), dt, steps, a_c0=a0)[0]
        jm = A.objective(O.Discretization(_with_sigma(p, c, -h)), dt, steps, a_c0=a0)[0]
        fd = (jp - jm) / (2.0 * h * d.sigma[c])
        assert abs(r.grad_sigma[c] - fd) <= 5e-8 * abs(fd), (c, r.grad_sigma[c], fd)
    c = cells[0]
    jp = A.objective(O.Discretization(_with_sigma(p, c, h)), dt, steps, a_c0=a0)[0]
    jm = A.objective(O.Discretization(_with_sigma(p, c, -h)), dt, steps, a_c0=a0)[0]
    fd = (jp - jm) / (2.0 * h * d.sigma[c])
    assert abs(r_lin.grad_sigma[c] - fd) > 2e-7 * abs(fd)      # the Brauer term is needed
    assert np.all(r.grad_sigma[d.sigma == 0] == 0.0)


def test_amplitude_gradient_matches_central_differences():
    p, d, dt = _problem(amp=3000.0)
    steps, h = 12, 1e-6
    r = A.adjoint_gradient(d, dt, steps)
    jp = A.objective(O.Discretization(p.with_(amplitude=3000.0 * (1 + h))), dt, steps)[0]
    jm = A.objective(O.Discretization(p.with_(amplitude=3000.0 * (1 - h))), dt, steps)[0]
    fd = (jp - jm) / (2.0 * h * 3000.0)
    assert abs(r.grad_amplitude - fd) <= 1e-7 * abs(fd)
    # J is quadratic in the amplitude from a zero start: dJ/dI0 = 2 J / I0
    assert r.grad_amplitude == pytest.approx(2.0 * r.J / 3000.0, rel=1e-8)


def test_objective_is_the_loss_of_the_state_trajectory():
    p, d, dt = _problem()
    a0 = 1e-7 * W.random_vector(3, d.n_c)
    J, a_end = A.objective(d, dt, 6, a_c0=a0)
    a, loss = a0.copy(), 0.0
    for m in range(6):
        res = run_explicit_euler(d, dt, 1, tol=1e-13, a_c0=a, m0=m)
        e = (res.a_c - a) / dt                                  # -dA/dt on conducting edges
        loss += dt * float(e @ (d.M_c * e))                     # sum over cells of sigma |E|^2 dV, FIT form
        a = res.a_c
    assert J == pytest.approx(loss, rel=1e-9)
    assert np.allclose(a_end, a, rtol=0, atol=1e-9 * np.abs(a).max())
