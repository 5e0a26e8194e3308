"""Failure paths on the GPU, produced without faulting it: a grid barrier that
can never complete gives up after its poll limit and reports MQS_ERR_TIMEOUT,
and the context stays usable; bad inputs come back as error codes."""
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


def test_unstable_step_is_reported(pkg):
    # far above the CFL bound the explicit update blows up; the PCG reports NaN
    # or non-convergence instead of hanging
    p = W.config_linear_block()
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(dt=1e-3, maxit=2000))
    rc, stats = s.step(60, allow_fail=True)
    assert rc != 0
    assert any(st.status in (-4, -5, -6) for st in stats)
    s.close()
