"""CUDA graphs of the steady-state SPE step: a replayed step issues the launches of the
launch-by-launch step with the same arguments (its time level and statistics slot come
from a device step counter), so every result must be bitwise that of the same steps taken
without graphs, across calls, enqueues, parity of the conductor buffers, and changes of dt,
options, state and block count between calls (each forces a new capture); and the same
for a batch, whose graphs hold several steps of every instance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.stepper import START_PREV, START_SPE
from tests.helpers import rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as p
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return p


def _pair(pkg, p, **kw):
    """The same problem twice: without and with graphs."""
    a = pkg.Solver.from_problem(p, pkg.SolverOptions(graph=0, **kw))
    b = pkg.Solver.from_problem(p, pkg.SolverOptions(graph=1, **kw))
    return a, b


def _same_stats(sa, sb):
    assert [(x.iterations, x.status, x.rank, x.refinements, x.relres, x.start_relres) for x in sa] == \
           [(x.iterations, x.status, x.rank, x.refinements, x.relres, x.start_relres) for x in sb]


def _same_state(a, b):
    xa, ta, ma = a.get_state()
    xb, tb, mb = b.get_state()
    assert ma == mb and ta == tb and np.array_equal(xa, xb)
    return xb, mb


@pytest.mark.parametrize("precision,variant,rhs_time,waveform",
                         [(0, 0, 0, 0), (0, 1, 1, 0), (1, 1, 0, 1), (2, 1, 0, 0)])
def test_graph_steps_are_bitwise_the_launch_by_launch_steps(pkg, precision, variant, rhs_time, waveform):
    p = W.scaled_nonlinear(16, amplitude=900.0).with_(waveform=waveform, tau=0.5)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    kw = dict(start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, precision=precision, pcg_variant=variant,
              rhs_time=rhs_time)
    a, b = _pair(pkg, p, **kw)
    for n in (5, 13, 12):                     # the table fills during the first call
        _, sa = a.step(n)
        _, sb = b.step(n)
        _same_stats(sa, sb)
    for _ in range(2):                        # several enqueues before one finish
        a.step_enqueue(7)
        b.step_enqueue(7)
    _, sa = a.step_finish(14)
    _, sb = b.step_finish(14)
    _same_stats(sa, sb)
    assert all(x.status == 0 for x in sb)
    x, m = _same_state(a, b)
    assert m == 44
    assert a.graph_steps() == 0 and b.graph_steps() >= 44 - 8 - 1
    if precision == 0 and variant == 0:
        ref = O.run_explicit_euler(d, dt, 44, start_mode=START_SPE, spe_depth=8, tol=1e-10, rhs_time=rhs_time)
        assert rel(x, ref.a_c) < 1e-8
    a.close()
    b.close()


def test_graphs_follow_changes_between_calls(pkg):
    # every change a step depends on (dt, options, state, block count, table) makes the
    # next eligible step capture again; the bits stay those of the launch-by-launch path
    p = W.scaled_nonlinear(12, amplitude=700.0)
    dt = O.dt_gershgorin(O.Discretization(p))
    kw = dict(start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10)
    a, b = _pair(pkg, p, **kw)
    s_ = pkg.SolverOptions

    def both(f):
        f(a)
        f(b)
        _, sa = a.step(12)
        _, sb = b.step(12)
        _same_stats(sa, sb)
        _same_state(a, b)

    both(lambda s: None)
    g0 = b.graph_steps()
    assert g0 > 0
    both(lambda s: s.set_dt(0.5 * dt))
    both(lambda s: s.set_options(s_(graph=s.options.graph, **dict(kw, dt=0.5 * dt, tol=1e-11, rhs_time=1))))
    x, t, m = a.get_state()
    both(lambda s: s.set_state(x * 0.5, t, m))
    both(lambda s: s.set_blocks(37))
    both(lambda s: s.reset_history())          # refills the table launch by launch first
    both(lambda s: s.set_options(s_(graph=s.options.graph, **dict(kw, dt=0.5 * dt, spe_depth=4))))
    assert b.graph_steps() > g0 + 40 and a.graph_steps() == 0
    a.close()
    b.close()


def test_graphs_only_for_the_steady_state_spe_step(pkg):
    # a start mode other than SPE, timing and separate right-hand sides stay launch by launch
    p = W.scaled_nonlinear(12, amplitude=700.0)
    dt = O.dt_gershgorin(O.Discretization(p))
    for kw in (dict(start_mode=START_PREV), dict(start_mode=START_SPE, rhs_split=1)):
        s = pkg.Solver.from_problem(p, pkg.SolverOptions(graph=1, dt=dt, **kw))
        s.mqs_step(20)
        assert s.graph_steps() == 0
        s.close()
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(graph=1, dt=dt, start_mode=START_SPE, spe_depth=4))
    s.timing_enable(True)
    s.mqs_step(20)
    assert s.graph_steps() == 0
    s.timing_enable(False)
    s.mqs_step(5)
    assert s.graph_steps() == 5
    s.close()


def _batch_problems():
    return [
        (W.config_linear_block(), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(20, sigma=3.1e6, amplitude=700.0), dict(start_mode=START_SPE, spe_depth=4,
                                                                      precision=1, pcg_variant=1)),
        (W.scaled_nonlinear(12, sigma=4.5e6, amplitude=900.0), dict(start_mode=START_SPE, spe_depth=8,
                                                                      rhs_time=1)),
    ]


def _batch(pkg, graph, extra=()):
    sv = []
    for p, kw in list(_batch_problems()) + list(extra):
        dt = O.dt_gershgorin(O.Discretization(p))
        sv.append(pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, dt=dt, graph=graph, **kw)))
    return sv, pkg.Batch(sv, blocks_scale=2.0)


def test_batch_graphs_are_bitwise_the_launch_by_launch_batch(pkg):
    sa, ba = _batch(pkg, 0)
    sb, bb = _batch(pkg, 1)
    for n in (3, 20, 16, 9):                    # below, across and at whole graph chunks
        _, ra = ba.step(n)
        _, rb = bb.step(n)
        for row_a, row_b in zip(ra, rb):
            _same_stats(row_a, row_b)
    assert ba.graph_steps() == 0 and bb.graph_steps() >= 24
    ba.set_scale(4.0)                           # new block counts: captured again
    bb.set_scale(4.0)
    _, ra = ba.step(16)
    _, rb = bb.step(16)
    for row_a, row_b in zip(ra, rb):
        _same_stats(row_a, row_b)
    assert bb.graph_steps() >= 40
    ba.close()
    bb.close()
    for a, b in zip(sa, sb):
        _same_state(a, b)
        a.close()
        b.close()


def test_batch_with_an_ineligible_instance_stays_launch_by_launch(pkg):
    extra = [(W.scaled_nonlinear(8, amplitude=500.0), dict(start_mode=START_PREV))]
    sv, bt = _batch(pkg, 1, extra)
    _, rows = bt.step(24)
    assert all(x.status == 0 for row in rows for x in row)
    assert bt.graph_steps() == 0
    bt.close()
    for s in sv:
        s.close()
