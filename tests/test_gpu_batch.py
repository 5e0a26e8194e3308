"""Batched multi-query (several independent problems advanced together on one GPU):
every instance against the oracle, the batch against separate runs, persistent PCG
kernels on few blocks, and the batch's argument checks."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.stepper import START_SPE
from tests.helpers import layout_to_oracle, oracle_to_layout, rel

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


def _instances():
    """(problem, options) pairs of different sizes, materials, coils and precisions."""
    return [
        (W.config_linear_block(), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(20, sigma=3.1e6, amplitude=700.0), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(24, sigma=1.4e6, amplitude=250.0), dict(start_mode=START_SPE, spe_depth=8,
                                                                      precision=1, pcg_variant=1)),
        (W.scaled_nonlinear(12, sigma=4.5e6, amplitude=900.0), dict(start_mode=1)),
    ]


def _solvers(pkg, steps_dt):
    out = []
    for (p, kw), dt in zip(_instances(), steps_dt):
        out.append(pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, dt=dt, **kw)))
    return out


def _dts():
    return [O.dt_gershgorin(O.Discretization(p)) for p, _ in _instances()]


def test_batch_instances_match_the_oracle(pkg):
    steps = 30
    dts = _dts()
    sv = _solvers(pkg, dts)
    batch = pkg.Batch(sv)
    _, stats = batch.step(steps)
    assert all(x.status == 0 for row in stats for x in row)
    assert batch.last_ms() > 0.0
    for q, ((p, kw), dt) in enumerate(zip(_instances(), dts)):
        d = O.Discretization(p)
        ref = O.run_explicit_euler(d, dt, steps, start_mode=kw["start_mode"], spe_depth=kw.get("spe_depth", 8),
                                   tol=1e-10)
        a_c, t, m = sv[q].get_state()
        assert m == steps and t == pytest.approx(steps * dt)
        assert rel(a_c, ref.a_c) < 1e-8, (q, rel(a_c, ref.a_c))
    batch.close()
    for s in sv:
        s.close()


def test_batch_equals_separate_runs(pkg):
    steps = 25
    dts = _dts()
    alone = _solvers(pkg, dts)
    for s in alone:
        s.mqs_step(steps)
    sv = _solvers(pkg, dts)
    batch = pkg.Batch(sv, blocks_scale=1.0)
    batch.step(10)
    batch.set_scale(4.0)                         # block counts may change between calls
    batch.step(5)
    batch.set_weighting(True)                    # shares by unknowns x the last call's iterations
    assert batch.weighting()
    batch.step(steps - 15)
    for a, b in zip(alone, sv):
        x, _, _ = a.get_state()
        y, _, _ = b.get_state()
        assert rel(y, x) < 1e-9                  # only the reductions' summation order differs
    batch.close()
    for s in alone + sv:
        s.close()


def test_batch_with_a_two_blocks_per_sm_instance(pkg):
    # a 96^3 instance (its PCG runs two blocks per SM) beside a small one, against the
    # same problems stepped separately
    probs = [W.scaled_nonlinear(96, amplitude=600.0), W.scaled_nonlinear(16, amplitude=800.0)]
    dts = [1.0e-7, 2.0e-7]

    def solvers():
        return [pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, dt=dt, start_mode=START_SPE, spe_depth=8))
                for p, dt in zip(probs, dts)]
    alone = solvers()
    for s in alone:
        s.mqs_step(6)
    sv = solvers()
    batch = pkg.Batch(sv, blocks_scale=2.0)
    _, stats = batch.step(6)
    assert all(x.status == 0 for row in stats for x in row)
    for a, b in zip(alone, sv):
        x, _, _ = a.get_state()
        y, _, m = b.get_state()
        assert m == 6 and rel(y, x) < 1e-9
    batch.close()
    for s in alone + sv:
        s.close()


@pytest.mark.parametrize("nblk", [1, 3, 7])
def test_pcg_on_few_persistent_blocks(pkg, nblk):
    p = W.scaled_nonlinear(24)
    d = O.Discretization(p)
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = 5.0 * d.X_s[d.n_idx]
    ref = O.pcg_jacobi(d.K_n, b_o[d.n_idx], None, d.D, tol=1e-10)
    for prec, var in ((0, 0), (0, 1), (1, 1)):
        s = pkg.Solver.from_problem(p, pkg.SolverOptions(precision=prec, pcg_variant=var))
        s.set_blocks(nblk)
        x, info = s.pcg_solve(oracle_to_layout(p.N, b_o), tol=1e-10)
        assert info.status == 0 and info.relres <= 1e-10
        assert rel(d.K_cn @ layout_to_oracle(p.N, x)[d.n_idx], d.K_cn @ ref.x) < 1e-9
        s.close()


def test_batch_tune_and_argument_checks(pkg):
    dts = _dts()
    sv = _solvers(pkg, dts)
    with pytest.raises(pkg.MqsError):
        pkg.Batch([sv[0], sv[0]])                # the same handle twice
    with pytest.raises(pkg.MqsError):
        sv[1].set_blocks(100000)                 # more blocks than SMs
    batch = pkg.Batch(sv)
    with pytest.raises(pkg.MqsError):
        batch.set_weighting(2)
    best = batch.tune(1)
    assert best in (1.0, 2.0, 4.0, 8.0) and batch.weighting() in (False, True)
    forms = batch.tune_pcg(1)                    # one form per (grid size, precision) group
    assert len(forms) == len(sv) and all(v[0] in (0, 1, 2) and v[1] in (0, 2, 3) and v[2] in (0, 1, 2) for v in forms)
    groups = {}
    for s_, v in zip(sv, forms):
        groups.setdefault((s_.n, s_.options.precision), set()).add(v)
        assert s_.pcg_form() == v
    assert all(len(g) == 1 for g in groups.values())
    _, stats = batch.step(3)
    assert all(x.status == 0 for row in stats for x in row)
    sv[0].close()                                # closes the batch first
    assert batch.b is None
    for s in sv[1:]:
        s.close()


def test_depth_tuner_sets_one_depth_per_grid_size(pkg):
    # the tuner searches the SPE depth group by group (grid size), sets the winner on every
    # SPE handle of the group, leaves other start modes alone; the trajectory stays the
    # oracle's (the start vector decides iteration counts only: a_c within the tolerance floor)
    probs = [
        (W.scaled_nonlinear(12, sigma=2.0e6, amplitude=700.0), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(12, sigma=4.0e6, amplitude=300.0), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(16, sigma=3.0e6, amplitude=500.0), dict(start_mode=START_SPE, spe_depth=8)),
        (W.scaled_nonlinear(8, amplitude=500.0), dict(start_mode=1)),
    ]
    dts = [O.dt_gershgorin(O.Discretization(p)) for p, _ in probs]
    sv = [pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, dt=dt, **kw)) for (p, kw), dt in zip(probs, dts)]
    bt = pkg.Batch(sv)
    with pytest.raises(pkg.MqsError):
        bt.tune_depth(3, depths=(0,))
    with pytest.raises(pkg.MqsError):
        bt.tune_depth(3, depths=(17,))
    chosen = bt.tune_depth(3, depths=(4, 8))
    assert chosen[0] == chosen[1] and chosen[0] in (4, 8) and chosen[2] in (4, 8) and chosen[3] == 8
    assert [s.options.spe_depth for s in sv] == chosen
    _, rows = bt.step(10)
    assert all(x.status == 0 for row in rows for x in row)
    bt.close()
    p, _ = probs[2]
    a_c, _, m = sv[2].get_state()
    assert m == 2 * 4 * (8 + 1 + 3) + 10         # two groups x four trials x (refill + trial), then 10
    ref = O.run_explicit_euler(O.Discretization(p), dts[2], m, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    assert rel(a_c, ref.a_c) < 1e-8
    for s in sv:
        s.close()
