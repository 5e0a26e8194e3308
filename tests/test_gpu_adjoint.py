"""Discrete adjoint on the GPU (mqs_adjoint): the eddy-current loss and its
gradients against the oracle adjoint (nonlinear Brauer term active), against
central differences of the GPU forward run, and the handle state afterwards."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import adjoint as A
from oracle.stepper import START_SPE, START_ZERO
from tests.helpers import rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as p
    import torch
    assert torch.cuda.is_available()
    return p


@pytest.mark.parametrize("mode,precision", [(START_SPE, 0), (START_ZERO, 0), (START_SPE, 1)])
def test_adjoint_matches_the_oracle_with_brauer_active(pkg, mode, precision):
    p = W.scaled_nonlinear(12, amplitude=2000.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    a0 = 3e-7 * W.random_vector(7, d.n_c)
    steps = 15
    B = d.cell_flux_density(d.full(a_c=a0))[d.brauer]
    assert 0.3 < B.max() < 2.3
    ref = A.adjoint_gradient(d, dt, steps, a_c0=a0)
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-11, start_mode=mode, spe_depth=8, dt=dt,
                                                     precision=precision, pcg_variant=precision))
    s.set_state(a0, 0.0, 0)
    J, gs, gI, info = s.adjoint(steps)
    assert J == pytest.approx(ref.J, rel=1e-9)
    gs = gs.reshape(-1)
    assert rel(gs, ref.grad_sigma) < 1e-7, rel(gs, ref.grad_sigma)
    big = np.abs(ref.grad_sigma) > 1e-3 * np.abs(ref.grad_sigma).max()
    assert np.max(np.abs(gs[big] - ref.grad_sigma[big]) / np.abs(ref.grad_sigma[big])) < 1e-6
    assert np.all(gs[d.sigma == 0] == 0.0)
    assert gI == pytest.approx(ref.grad_amplitude, rel=1e-6, abs=1e-9 * abs(ref.grad_amplitude) + 1e-30)
    assert info.forward_iterations > 0 and info.adjoint_iterations > 0
    a_c, t, m = s.get_state()                       # the handle sits at the forward end state
    assert m == steps and rel(a_c, ref.a_c) < 1e-8
    s.close()


@pytest.mark.parametrize("mode", [START_SPE, START_ZERO])
def test_checkpointed_adjoint_matches_the_full_trajectory(pkg, mode):
    # checkpoints every 4 steps (segments 4, 4, 4, 3) with recomputation in between
    p = W.scaled_nonlinear(12, amplitude=2000.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    a0 = 3e-7 * W.random_vector(7, d.n_c)
    steps = 15
    ref = A.adjoint_gradient(d, dt, steps, a_c0=a0)
    opts = pkg.SolverOptions(tol=1e-11, start_mode=mode, spe_depth=8, dt=dt)
    full = pkg.Solver.from_problem(p, opts)
    full.set_state(a0, 0.0, 0)
    J0, g0, gI0, i0 = full.adjoint(steps)
    s = pkg.Solver.from_problem(p, opts)
    s.set_state(a0, 0.0, 0)
    J, gs, gI, info = s.adjoint(steps, checkpoint_every=4)
    assert J == pytest.approx(J0, rel=1e-12)                 # the same forward sweep
    assert info.forward_iterations == i0.forward_iterations and info.recompute_iterations > 0
    assert rel(gs.reshape(-1), g0.reshape(-1)) < 1e-8       # recomputed records agree to the solve tolerance
    assert rel(gs.reshape(-1), ref.grad_sigma) < 1e-7
    assert gI == pytest.approx(gI0, rel=1e-8)
    a_c, t, m = s.get_state()
    b_c, tb, mb = full.get_state()
    assert m == mb == steps and t == tb and np.array_equal(a_c, b_c)
    # a second call continues from the end state
    J2, gs2, gI2, _ = s.adjoint(9, checkpoint_every=5)
    J2f, gs2f, gI2f, _ = full.adjoint(9)
    assert J2 == pytest.approx(J2f, rel=1e-12) and gI2 == pytest.approx(gI2f, rel=1e-8)
    assert rel(gs2.reshape(-1), gs2f.reshape(-1)) < 1e-8
    s.close()
    full.close()


def test_adjoint_amplitude_gradient_from_rest(pkg):
    p = W.scaled_nonlinear(12, amplitude=3000.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = A.adjoint_gradient(d, dt, 12)
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-11, start_mode=START_SPE, dt=dt))
    J, gs, gI, _ = s.adjoint(12)
    assert J == pytest.approx(ref.J, rel=1e-9)
    assert gI == pytest.approx(ref.grad_amplitude, rel=1e-7)
    assert gI == pytest.approx(2.0 * J / 3000.0, rel=1e-7)     # J is quadratic in the amplitude from rest
    assert rel(gs.reshape(-1), ref.grad_sigma) < 1e-7
    # a second call continues from the end state (source time level m0 + m) and grows the
    # trajectory storage
    ref2 = A.adjoint_gradient(d, dt, 20, a_c0=ref.a_c, m0=12)
    J2, gs2, gI2, _ = s.adjoint(20)
    assert J2 == pytest.approx(ref2.J, rel=1e-9)
    assert rel(gs2.reshape(-1), ref2.grad_sigma) < 1e-7
    assert gI2 == pytest.approx(ref2.grad_amplitude, rel=1e-6)
    s.close()


def test_adjoint_matches_central_differences_of_the_gpu_forward(pkg):
    p = W.scaled_nonlinear(24, amplitude=800.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    a0 = 2e-7 * W.random_vector(11, d.n_c)
    steps, h = 30, 1e-6
    opts = dict(tol=1e-12, start_mode=START_SPE, spe_depth=8, dt=dt)

    def loss(problem):
        s = pkg.Solver.from_problem(problem, pkg.SolverOptions(**opts))
        s.set_state(a0, 0.0, 0)
        out = s.loss(steps)
        s.close()
        return out

    s = pkg.Solver.from_problem(p, pkg.SolverOptions(**opts))
    s.set_state(a0, 0.0, 0)
    J, gs, gI, _ = s.adjoint(steps)
    s.close()
    assert J == pytest.approx(loss(p), rel=1e-12)          # mqs_loss is the forward half
    g = gs.reshape(-1)
    rng = np.random.default_rng(1611)
    # cells whose gradient stands above the finite differences' noise (J is accurate to about
    # the solve tolerance, so a difference quotient resolves about 1e-11 J / (h sigma))
    cand = np.flatnonzero((d.sigma > 0) & (np.abs(g) > 1e-3 * np.abs(g).max()))
    cells = rng.choice(cand, size=6, replace=False)
    for c in cells:
        sp = p.sigma_cell.copy().reshape(-1)
        sm = sp.copy()
        sp[c] *= 1 + h
        sm[c] *= 1 - h
        jp = loss(p.with_(sigma_cell=sp.reshape(p.sigma_cell.shape)))
        jm = loss(p.with_(sigma_cell=sm.reshape(p.sigma_cell.shape)))
        fd = (jp - jm) / (2 * h * d.sigma[c])
        assert abs(g[c] - fd) <= 1e-5 * abs(fd) + 1e-11 * J / (h * d.sigma[c]), (c, g[c], fd)


def test_eddy_loss_autograd_function(pkg):
    import torch
    p = W.scaled_nonlinear(12, amplitude=1500.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    opts = pkg.SolverOptions(tol=1e-11, start_mode=START_SPE, spe_depth=8, dt=dt)
    sig = torch.tensor(p.sigma_cell, dtype=torch.float64, requires_grad=True)
    amp = torch.tensor(1500.0, dtype=torch.float64, requires_grad=True)
    J = pkg.eddy_loss(sig, amp, p, opts, 10)
    (3.0 * J).backward()
    ref = A.adjoint_gradient(d, dt, 10)
    assert float(J.detach()) == pytest.approx(ref.J, rel=1e-9)
    assert rel(sig.grad.numpy().reshape(-1), 3.0 * ref.grad_sigma) < 1e-7
    assert float(amp.grad) == pytest.approx(3.0 * ref.grad_amplitude, rel=1e-7)
    sig2 = sig.detach().clone().requires_grad_(True)
    J2 = pkg.eddy_loss(sig2, amp.detach(), p, opts, 10, checkpoint_every=3)
    J2.backward()
    assert float(J2.detach()) == pytest.approx(ref.J, rel=1e-9)
    assert rel(sig2.grad.numpy().reshape(-1), ref.grad_sigma) < 1e-7
