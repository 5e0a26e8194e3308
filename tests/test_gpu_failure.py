"""Failure paths on the GPU, produced without faulting it: a grid barrier that
can never complete gives up after its poll limit and reports MQS_ERR_TIMEOUT,
and the context stays usable; bad inputs come back as error codes; a step
above the stability bound of eq. (CFL) is caught by the instability monitor,
and a failing step stops the rest of its call."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import oracle_to_layout

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


def test_stuck_barrier_times_out_and_context_survives(pkg):
    lib = pkg.load()
    assert lib.mqs_selftest_barrier_timeout(20000) == -8          # MQS_ERR_TIMEOUT
    p = W.config_linear_block()
    d = O.Discretization(p)
    s = pkg.Solver.from_problem(p, pkg.SolverOptions())
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = d.X_s[d.n_idx]
    x, info = s.pcg_solve(oracle_to_layout(p.N, b_o), tol=1e-10)
    assert info.status == 0 and info.relres <= 1e-10
    s.close()


def test_setup_rejects_bad_inputs(pkg):
    p = W.config_linear_block()
    with pytest.raises(pkg.MqsError):
        pkg.Solver.from_problem(p.with_(coil_i0=7, coil_i1=9, coil_j0=7, coil_j1=9),   # coil through the block
                                pkg.SolverOptions())
    bad = p.with_(brauer_cell=np.ones_like(p.brauer_cell))                            # nonconducting iron
    with pytest.raises(pkg.MqsError):
        pkg.Solver.from_problem(bad, pkg.SolverOptions())
    with pytest.raises(pkg.MqsError):
        pkg.Solver.from_problem(p, pkg.SolverOptions(spe_depth=99))
    # kernel forms that do not exist: a tile-group count other than 2 or 3, halo warps other
    # than 1 or 2, two halo warps beside three tile groups (576 threads)
    for bad_form in (dict(tile_groups=4), dict(halo_warps=3), dict(halo_warps=-1),
                     dict(tile_groups=3, halo_warps=2)):
        with pytest.raises(pkg.MqsError):
            pkg.Solver.from_problem(p, pkg.SolverOptions(pcg_variant=1, **bad_form))
    s = pkg.Solver.from_problem(p, pkg.SolverOptions())
    with pytest.raises(pkg.MqsError):
        s.step(1)                                                                     # dt not set
    with pytest.raises((pkg.MqsError, ValueError)):
        s.set_state(np.zeros(s.n_c + 1))                                              # wrong length
    lib = pkg.load()
    import ctypes as C
    a = np.zeros(s.n_c + 1)
    assert lib.mqs_set_state(s.h, a.ctypes.data_as(C.POINTER(C.c_double)), a.size, 0.0, 0) == -1   # at the ABI
    s.close()


@pytest.mark.parametrize("factor", [10.0, 100.0])
def test_unstable_step_is_reported(pkg, factor):
    # dt at 10x / 100x the stability bound 2 / lambda_max (setup computes lambda_max and
    # scales by cfl_factor): the instability monitor fails the step once the increments
    # have grown with alternating sign over 8 steps in a row, the loop stops there, and
    # the handle stays at the step before it
    p = W.config_linear_block()
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(cfl_factor=factor, start_mode=pkg.START_SPE))
    dt, lam = s.dt_lambda()
    assert lam > 0 and dt == pytest.approx(factor * 2.0 / lam, rel=1e-15)
    rc, stats = s.step(60, allow_fail=True)
    assert rc == -7                                                  # MQS_ERR_UNSTABLE
    codes = [st.status for st in stats]
    f = codes.index(-7)
    assert all(c == 0 for c in codes[:f]) and all(c == -10 for c in codes[f + 1:])   # MQS_ERR_HALTED
    assert 8 <= f <= 30
    assert all(st.iterations == 0 for st in stats[f + 1:])
    a_c, t, m = s.get_state()
    assert m == f and t == pytest.approx(f * dt, rel=1e-15)
    # the same f steps on a fresh handle: bitwise the state the failed call left
    r = pkg.Solver.from_problem(p, pkg.SolverOptions(dt=dt, start_mode=pkg.START_SPE))
    r.step(f)
    a_r, _, _ = r.get_state()
    assert np.array_equal(a_c, a_r)
    r.close()
    # the handle goes on from there at a stable step
    s.set_dt(0.9 * 2.0 / lam)
    rc, stats = s.step(5)
    assert rc == 0 and s.get_state()[2] == f + 5
    s.close()


def test_failed_solve_halts_the_rest_of_the_call(pkg):
    # a solve that stops at maxit fails its step; the later steps of the call do not run
    # and the handle keeps the state of the last good step
    p = W.config_linear_block()
    dt = O.dt_gershgorin(O.Discretization(p))
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(dt=dt, start_mode=pkg.START_ZERO))
    s.step(3)
    a3, _, _ = s.get_state()
    s.set_options(pkg.SolverOptions(dt=dt, start_mode=pkg.START_ZERO, maxit=2))
    rc, stats = s.step(6, allow_fail=True)
    assert rc == -4 and stats[0].status == -4                        # MQS_ERR_NOT_CONVERGED
    assert [st.status for st in stats[1:]] == [-10] * 5
    a_c, _, m = s.get_state()
    assert m == 3 and np.array_equal(a_c, a3)
    s.set_options(pkg.SolverOptions(dt=dt, start_mode=pkg.START_ZERO))
    rc, _ = s.step(2)
    assert rc == 0 and s.get_state()[2] == 5
    s.close()


def test_monitor_is_quiet_at_the_stability_bound(pkg):
    # at 0.99 of the bound (top-mode factor -0.98: alternating, decaying) nothing is flagged
    p = W.config_linear_block()
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(cfl_factor=0.99, start_mode=pkg.START_SPE))
    rc, stats = s.step(200)
    assert rc == 0 and all(st.status == 0 for st in stats)
    s.close()
