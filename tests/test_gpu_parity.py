"""GPU parity: every row of the hot path through the C ABI against the FP64
oracle on the same seeded inputs.

Tolerances: stencil / conductor rate 1e-12 relative (FP64 summation order);
gauge-invariant solve results (K_cn w, a_c) 1e-9 per solve and 1e-8 after all
steps at PCG relative residual 1e-10 (the bar stated for the FP64 path);
PCG iteration counts within a few iterations (rounding decides the last one).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.stepper import START_POD, START_PREV, START_SPE, START_ZERO
from tests.helpers import layout_to_oracle, oracle_to_layout, rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as p
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return p


def make(pkg, p, **kw):
    return pkg.Solver.from_problem(p, pkg.SolverOptions(**kw))


def golden():
    with open(os.path.join(HERE, "golden", "linear_block_16.json")) as f:
        return json.load(f)


# ---- (a4) the K_n stencil -------------------------------------------------------------
@pytest.mark.parametrize("N", [4, 16, 35, 64])
def test_apply_kn_matches_assembled_matrix(pkg, N):
    p = W.scaled_nonlinear(N) if N >= 8 else W.random_problem(1, N)
    d = O.Discretization(p)
    s = make(pkg, p)
    x_l = W.random_vector(N, 3 * N ** 3)
    y = s.apply_kn(x_l)
    x_o = layout_to_oracle(N, x_l)
    y_o = np.zeros(d.grid.n_edges)
    y_o[d.n_idx] = d.K_n @ x_o[d.n_idx]
    y_ref = oracle_to_layout(N, y_o)
    scale = 4 * p.nu0 / p.h * np.abs(x_l).max()
    assert np.abs(y - y_ref).max() <= 1e-13 * scale
    s.close()


# ---- (a4) PCG ---------------------------------------------------------------------------
# kernel forms (pcg_variant, tile_groups, halo_warps); 35 = 32 + 3 leaves ragged tiles in x and y
@pytest.mark.parametrize("form", [(0, 0, 0), (1, 2, 1), (1, 3, 1), (1, 2, 2)])
@pytest.mark.parametrize("N", [16, 35])
def test_pcg_solve_matches_oracle(pkg, N, form):
    p = W.scaled_nonlinear(N)
    d = O.Discretization(p)
    s = make(pkg, p, pcg_variant=form[0], tile_groups=form[1], halo_warps=form[2])
    a_c = W.random_vector(7, d.n_c) * 1e-9
    b_n = 3.0 * d.X_s[d.n_idx] - d.K_cn.T @ a_c
    ref = O.pcg_jacobi(d.K_n, b_n, None, d.D, tol=1e-10)
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = b_n
    x_l, info = s.pcg_solve(oracle_to_layout(N, b_o), tol=1e-10)
    x_n = layout_to_oracle(N, x_l)[d.n_idx]
    assert info.status == 0 and info.relres <= 1e-10
    assert abs(info.iterations - ref.iterations) <= 3
    assert rel(d.K_cn @ x_n, d.K_cn @ ref.x) < 1e-9
    assert np.linalg.norm(b_n - d.K_n @ x_n) <= 1.01e-10 * np.linalg.norm(b_n)
    s.close()


_REF96 = {}


def _oracle_solve_96():
    # one oracle solve at 96^3 (2.6 M unknowns), shared by the two precisions below
    if not _REF96:
        p = W.scaled_nonlinear(96)
        d = O.Discretization(p)
        a_c = W.random_vector(7, d.n_c) * 1e-9
        b_n = 3.0 * d.X_s[d.n_idx] - d.K_cn.T @ a_c
        _REF96.update(p=p, d=d, b_n=b_n, ref=O.pcg_jacobi(d.K_n, b_n, None, d.D, tol=1e-10))
    return _REF96


@pytest.mark.parametrize("precision,variant,halo", [(0, 0, 0), (0, 1, 0), (0, 1, 2), (1, 1, 0), (1, 2, 0)])
def test_two_blocks_per_sm_solve_matches_oracle_at_96(pkg, precision, variant, halo):
    # from 96^3 on the two-reduction FP64 PCG and the FP32-inner refinement run two blocks
    # per SM (the kernels' second instantiation); the one-reduction FP64 pass keeps one, in
    # both halo forms; every solve against the oracle's
    r = _oracle_solve_96()
    p, d, b_n, ref = r["p"], r["d"], r["b_n"], r["ref"]
    s = make(pkg, p, precision=precision, pcg_variant=variant, halo_warps=halo)
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = b_n
    x_l, info = s.pcg_solve(oracle_to_layout(96, b_o), tol=1e-10)
    x_n = layout_to_oracle(96, x_l)[d.n_idx]
    assert info.status == 0 and info.relres <= 1e-10
    if precision == 0:
        assert abs(info.iterations - ref.iterations) <= 3
    assert rel(d.K_cn @ x_n, d.K_cn @ ref.x) < 1e-9
    assert np.linalg.norm(b_n - d.K_n @ x_n) <= 1.01e-10 * np.linalg.norm(b_n)
    s.close()


def test_pcg_edge_cases(pkg):
    p = W.config_linear_block()
    d = O.Discretization(p)
    s = make(pkg, p)
    L = 3 * p.N ** 3
    x, info = s.pcg_solve(np.zeros(L))                       # zero right-hand side
    assert info.status == 0 and info.iterations == 0 and not x.any()
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = d.X_s[d.n_idx]
    b = oracle_to_layout(p.N, b_o)
    xs, info = s.pcg_solve(b, tol=1e-12)
    _, info2 = s.pcg_solve(b, x0=xs, tol=1e-10)              # start at the solution
    assert info2.iterations == 0 and info2.status == 0
    _, info3 = s.pcg_solve(b, tol=1e-10, maxit=2, allow_fail=True)
    assert info3.status == -4                                # MQS_ERR_NOT_CONVERGED
    bn = b.copy()
    bn[np.flatnonzero(b)[0]] = np.nan
    _, info4 = s.pcg_solve(bn, allow_fail=True)
    assert info4.status == -6                                # MQS_ERR_NAN
    # entries off the n-edges are ignored
    junk = b.copy()
    junk[:p.N ** 2] += 1.0                                   # Dirichlet x-edges at k = 0
    x5, _ = s.pcg_solve(junk, tol=1e-12)
    assert rel(d.K_cn @ layout_to_oracle(p.N, x5)[d.n_idx], d.K_cn @ layout_to_oracle(p.N, xs)[d.n_idx]) < 1e-9
    s.close()


# ---- (a5) conductor rate with the Brauer law ----------------------------------------------
def test_conductor_rate_matches_oracle(pkg):
    p = W.scaled_nonlinear(16, amplitude=2e3)
    d = O.Discretization(p)
    s = make(pkg, p)
    a_c = W.random_vector(3, d.n_c) * 2e-6            # |B| up to a few tesla: strongly nonlinear
    w_n = W.random_vector(4, d.n_n) * 2e-6
    a_full = d.full(a_c, w_n)
    assert d.cell_flux_density(a_full)[d.brauer].max() > 1.0
    F_ref = d.apply_K(a_full, a_full)[d.c_idx]
    F = s.conductor_rate(a_c, oracle_to_layout(p.N, d.full(None, w_n)))
    assert rel(F, F_ref) < 1e-12
    s.close()


# ---- (a7) CFL step by the power method -------------------------------------------------------
def test_lambda_max_matches_oracle(pkg):
    g = golden()
    p = W.config_linear_block()
    s = make(pkg, p)
    lam, it = s.lambda_max(W.power_start_vector(s.n_c))
    assert lam == pytest.approx(g["lambda_max"], rel=1e-6)
    s.close()


def test_setup_sets_dt_from_the_cfl_factor(pkg):
    # mqs_setup with dt <= 0 and cfl_factor > 0 runs the power method itself (its own
    # start vector): lambda_max as the oracle's, dt = cfl_factor 2 / lambda_max
    g = golden()
    s = make(pkg, W.config_linear_block(), cfl_factor=0.9)
    dt, lam = s.dt_lambda()
    assert lam == pytest.approx(g["lambda_max"], rel=1e-6)
    assert dt == 0.9 * 2.0 / lam
    s.close()
    s = make(pkg, W.config_linear_block(), dt=1e-7, cfl_factor=0.9)     # an explicit dt wins
    assert s.dt_lambda() == (1e-7, 0.0)
    s.close()


# ---- full steps (a2-a6), 16^3 linear block, 200 steps, every start vector ---------------------
@pytest.mark.parametrize("mode,name", [(START_ZERO, "zero"), (START_PREV, "prev"), (START_SPE, "spe8"),
                                       (START_POD, "pod20")])
def test_explicit_euler_parity_linear_block(pkg, mode, name):
    g = golden()
    p = W.config_linear_block()
    s = make(pkg, p, start_mode=mode, spe_depth=8, pod_snapshots=20, dt=g["dt"], tol=1e-10)
    stats = s.mqs_step(g["steps"])
    a_c, t, m = s.get_state()
    ref = np.array(g["runs"][name]["a_c"])
    assert m == g["steps"]
    assert rel(a_c, ref) < 1e-8
    its = np.array([st.iterations for st in stats])
    assert abs(its.mean() - g["runs"][name]["mean_iterations"]) <= 1.0
    assert all(st.status == 0 and st.relres <= 1e-10 for st in stats)
    s.close()


# ---- nonlinear iron, ragged size, step-by-step against the oracle -------------------------------
@pytest.mark.parametrize("mode", [START_ZERO, START_SPE, START_POD])
def test_nonlinear_parity(pkg, mode):
    p = W.scaled_nonlinear(24, amplitude=5e4)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    steps = 25
    ref = O.run_explicit_euler(d, dt, steps, start_mode=mode, spe_depth=4, pod_snapshots=10, tol=1e-10)
    s = make(pkg, p, start_mode=mode, spe_depth=4, pod_snapshots=10, dt=dt, tol=1e-10)
    stats = s.mqs_step(steps)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    w = layout_to_oracle(p.N, s.get_solution())[d.n_idx]
    assert rel(d.K_cn @ w, d.K_cn @ ref.w) < 1e-8
    its = np.array([st.iterations for st in stats])
    assert np.abs(its - ref.iterations).max() <= 3
    s.close()


# ---- (a3, a6) start vectors as stand-alone calls ------------------------------------------------
def _window(d, p, steps, dt, depth):
    r = O.run_explicit_euler(d, dt, steps, start_mode=START_ZERO, tol=1e-12, spe_depth=depth,
                             pod_snapshots=depth, history=(hist := []))
    return r, hist


def test_spe_start_matches_oracle(pkg):
    p = W.config_linear_block()
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    hist = []
    O.run_explicit_euler(d, dt, 12, start_mode=START_SPE, spe_depth=6, tol=1e-12, history=hist)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=6)
    for w in reversed(hist):                              # oldest first
        s.push_history(oracle_to_layout(p.N, d.full(None, w)))
    a_c = W.random_vector(5, d.n_c) * 1e-12
    b_n = 0.7 * d.X_s[d.n_idx] - d.K_cn.T @ a_c
    x_ref, rank_ref = O.spe_start(d.K_n, hist, b_n)
    x_l, rank = s.spe_start(oracle_to_layout(p.N, d.full(None, b_n)))
    x_n = layout_to_oracle(p.N, x_l)[d.n_idx]
    nb = np.linalg.norm(b_n)
    r_gpu = np.linalg.norm(b_n - d.K_n @ x_n) / nb
    r_ref = np.linalg.norm(b_n - d.K_n @ x_ref) / nb
    assert r_gpu <= 1.5 * r_ref + 1e-12
    assert rel(d.K_cn @ x_n, d.K_cn @ x_ref) < 1e-6
    for w in hist:                                        # Galerkin orthogonality
        assert abs(w @ (b_n - d.K_n @ x_n)) <= 1e-8 * np.linalg.norm(w) * nb
    assert 1 <= rank <= 6
    s.close()


def test_pod_basis_matches_oracle(pkg):
    p = W.config_linear_block()
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    hist = []
    O.run_explicit_euler(d, dt, 15, start_mode=START_POD, pod_snapshots=12, tol=1e-12, history=hist)
    s = make(pkg, p, start_mode=START_POD, pod_snapshots=12)
    for w in reversed(hist):
        s.push_history(oracle_to_layout(p.N, d.full(None, w)))
    k, sig, info = s.pod_basis()
    b_n = 0.3 * d.X_s[d.n_idx]
    x_ref, k_ref, sig_ref, info_ref = O.pod_start(d.K_n, hist, b_n)
    assert k == k_ref
    big = sig_ref >= 1e-6 * sig_ref[0]
    assert np.allclose(sig[:len(sig_ref)][big], sig_ref[big], rtol=1e-8)
    # the method of snapshots resolves sigma_i only to about sqrt(eps) sigma_1,
    # so the information ratio (a sum over all sigma_i) agrees to ~ m * 1.5e-8
    assert info == pytest.approx(info_ref, abs=len(sig_ref) * 2e-8)
    x_l, k2 = s.pod_start(oracle_to_layout(p.N, d.full(None, b_n)))
    x_n = layout_to_oracle(p.N, x_l)[d.n_idx]
    assert rel(d.K_cn @ x_n, d.K_cn @ x_ref) < 1e-6
    s.close()


# ---- state round trip and checkpoint/resume ----------------------------------------------------------
def test_checkpoint_resume_is_exact(pkg):
    g = golden()
    p = W.config_linear_block()
    s = make(pkg, p, start_mode=START_ZERO, dt=g["dt"])
    s.mqs_step(10)
    a10, t10, m10 = s.get_state()
    s.mqs_step(5)
    a15, _, _ = s.get_state()
    s.set_state(a10, t10, m10)
    s.mqs_step(5)
    b15, _, m = s.get_state()
    assert m == 15 and np.array_equal(a15, b15)
    s.close()


def test_dt_and_source_level_changes_between_calls(pkg):
    # each step forms the next step's right-hand side in advance; a dt or source-level
    # change between calls must not reuse it (oracle: the same three legs)
    p = W.scaled_nonlinear(12, amplitude=900.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    r1 = O.run_explicit_euler(d, dt, 6, start_mode=START_SPE, spe_depth=8, tol=1e-11)
    r2 = O.run_explicit_euler(d, 0.5 * dt, 5, start_mode=START_ZERO, tol=1e-11, a_c0=r1.a_c, m0=6)
    r3 = O.run_explicit_euler(d, 0.5 * dt, 4, start_mode=START_ZERO, tol=1e-11, a_c0=r2.a_c, m0=11, rhs_time=1)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-11)
    s.mqs_step(6)
    s.set_dt(0.5 * dt)
    s.mqs_step(5)
    a2, _, _ = s.get_state()
    assert rel(a2, r2.a_c) < 1e-8
    s.set_options(pkg.SolverOptions(start_mode=START_SPE, spe_depth=8, dt=0.5 * dt, tol=1e-11, rhs_time=1))
    s.mqs_step(4)
    a3, _, m = s.get_state()
    assert m == 15 and rel(a3, r3.a_c) < 1e-8
    s.close()


def test_boundary_touching_coil_and_conductor_match_the_oracle(pkg):
    # the right-hand side's support list at the domain faces: a conductor slab on the x = 0
    # face and a coil loop one node inside the y = 0 face; a loop on the face itself (its
    # edges would be Dirichlet) is refused by both sides
    N = 12
    sig = np.zeros((N, N, N))
    sig[3:7, 3:8, 0:4] = 2e6                       # [k, j, i]: cells with i = 0..3 touch x = 0
    base = W.scaled_nonlinear(N, amplitude=800.0).with_(sigma_cell=sig, brauer_cell=(sig > 0).astype(np.uint8),
                                                        coil_k=9, coil_i0=2, coil_i1=9, coil_j1=7)
    with pytest.raises(ValueError):
        O.Discretization(base.with_(coil_j0=0))
    with pytest.raises(pkg.MqsError):
        make(pkg, base.with_(coil_j0=0), start_mode=START_SPE, dt=1e-7)
    p = base.with_(coil_j0=1)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 12, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    for split in (0, 1):
        s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, rhs_split=split)
        st = s.mqs_step(12)
        a_c, _, m = s.get_state()
        assert m == 12 and all(x.status == 0 for x in st)
        assert rel(a_c, ref.a_c) < 1e-8, (split, rel(a_c, ref.a_c))
        s.close()


@pytest.mark.parametrize("mode", [START_SPE, START_ZERO])
def test_separate_right_hand_sides_match_the_oracle(pkg, mode):
    # rhs_split: the conductor type and the coil type solved separately, each with its own
    # SPE table (eq. (mrhs) and the list after it); oracle: literal mode, same histories
    p = W.scaled_nonlinear(16, amplitude=900.0)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    steps = 25
    ref = O.run_explicit_euler(d, dt, steps, start_mode=mode, spe_depth=8, tol=1e-10, literal=True)
    s = make(pkg, p, start_mode=mode, spe_depth=8, dt=dt, tol=1e-10, rhs_split=1)
    st = s.mqs_step(steps)
    a_c, t, m = s.get_state()
    assert m == steps and rel(a_c, ref.a_c) < 1e-8
    its = np.array([x.iterations for x in st])
    assert all(x.status == 0 for x in st)
    assert np.all(np.abs(its - ref.iterations) <= 4), (its, ref.iterations)
    fused = make(pkg, p, start_mode=mode, spe_depth=8, dt=dt, tol=1e-10)
    fused.mqs_step(steps)
    b_c, _, _ = fused.get_state()
    assert rel(a_c, b_c) < 1e-8
    if mode == START_SPE:
        # per-type starts beat zero starts for both types (the coil type's start is exact
        # once one of its solutions is known)
        zero = O.run_explicit_euler(d, dt, steps, start_mode=START_ZERO, tol=1e-10, literal=True)
        assert its[5:].sum() < 0.5 * zero.iterations[5:].sum()
    with pytest.raises(pkg.MqsError):
        s.adjoint(3)                                   # the adjoint runs the fused solve
    s.close()
    fused.close()
    with pytest.raises(pkg.MqsError):
        make(pkg, p, start_mode=START_POD, dt=dt, rhs_split=1)


def test_step_enqueue_finish_equals_step(pkg):
    # the two halves of mqs_step (with the SPE table push on the side stream) give the
    # bits of mqs_step, also with several enqueues before one finish; mqs_step while
    # steps are enqueued and an unmatched finish are refused
    p = W.scaled_nonlinear(16, amplitude=900.0)
    dt = O.dt_gershgorin(O.Discretization(p))
    a = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt)
    b = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt)
    _, sa = a.step(12)
    with pytest.raises(pkg.MqsError):
        b.step_enqueue(0)
    for _ in range(2):
        b.step_enqueue(4)
        with pytest.raises(pkg.MqsError):
            b.step(1)                                   # steps are enqueued
        rc, sb = b.step_finish(4)
        assert rc == 0 and all(x.status == 0 for x in sb)
    for _ in range(4):
        b.step_enqueue(1)                               # queued behind each other, one finish
    rc, sb = b.step_finish(4)
    assert rc == 0 and len(sb) == 4 and all(x.status == 0 and x.iterations > 0 for x in sb)
    assert [x.iterations for x in sb] == [x.iterations for x in sa[8:]]
    with pytest.raises(pkg.MqsError):
        b.step_finish(4)
    xa, ta, ma = a.get_state()
    xb, tb, mb = b.get_state()
    assert ma == mb == 12 and ta == tb and np.array_equal(xa, xb)
    a.close()
    b.close()


# ---- full-size workload (64^3 nonlinear iron), sampled against the oracle -----------------------------
def test_full_size_nonlinear_first_steps(pkg):
    p = W.config_nonlinear_iron()
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    steps = 2
    ref = O.run_explicit_euler(d, dt, steps, start_mode=START_ZERO, tol=1e-10)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10)
    s.mqs_step(steps)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    # properties over a longer GPU run: SPE and zero start agree, SPE saves iterations
    s2 = make(pkg, p, start_mode=START_ZERO, dt=dt, tol=1e-10)
    st_spe = s.mqs_step(18)
    st_zero = s2.mqs_step(20)
    a1, _, _ = s.get_state()
    a2, _, _ = s2.get_state()
    assert rel(a1, a2) < 1e-8
    assert np.mean([x.iterations for x in st_spe[-8:]]) < 0.5 * np.mean([x.iterations for x in st_zero[-8:]])
    s.close()
    s2.close()


def test_bench_configuration_against_the_oracle(pkg):
    # the timed workload itself: 64^3 Brauer iron, SPE 8 (float-float table full after
    # 8 steps), tol 1e-10, one block per SM, steps issued one at a time as the benchmark
    # issues them, at the step of eq. (CFL) (0.9 * 2 / lambda_max) that the oracle's power
    # method gives (stored by tests/golden/make_golden.py --iron64), given to both sides
    with open(os.path.join(HERE, "golden", "nonlinear_iron_64.json")) as f:
        g64 = json.load(f)
    p = W.config_nonlinear_iron()
    d = O.Discretization(p)
    dt = g64["dt"]
    steps = 30
    ref = O.run_explicit_euler(d, dt, steps, start_mode=START_SPE, spe_depth=8, tol=1e-10, eps_lin=1e-10)
    # pcg_variant 1 (one reduction per iteration, the benchmark's kernel) with one and with
    # two halo warps per tile group (bitwise the same iterates), and pcg_variant 0
    fused = None
    for variant, halo in ((1, 0), (1, 2), (0, 0)):
        s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, eps_lin=1e-10, pcg_variant=variant,
                 halo_warps=halo)
        # the benchmark's own step comes from the GPU power method: the same lambda_max
        lam, _ = s.lambda_max(W.power_start_vector(s.n_c), pcg_tol=1e-12, rtol=1e-8, maxit=2000)
        assert lam == pytest.approx(g64["lambda_max"], rel=1e-6)
        s.set_dt(dt)
        for _ in range(steps):
            s.step_enqueue(1)
        rc, stats = s.step_finish(steps)
        assert rc == 0
        a_c, _, m = s.get_state()
        assert m == steps
        assert rel(a_c, ref.a_c) < 1e-8, variant
        w = layout_to_oracle(p.N, s.get_solution())[d.n_idx]
        assert rel(d.K_cn @ w, d.K_cn @ ref.w) < 1e-8, variant
        its = np.array([st.iterations for st in stats])
        assert np.abs(its - ref.iterations).max() <= 3, (variant, its.tolist(), ref.iterations.tolist())
        if variant == 1:
            if fused is None:
                fused = (a_c, its)
            else:
                assert np.array_equal(a_c, fused[0]) and np.array_equal(its, fused[1])
        s.close()


# ---- other readings of the step and the paper-sized grid ---------------------------------------
@pytest.mark.parametrize("rhs_time,waveform", [(1, 0), (0, 1), (1, 1)])
def test_source_time_level_and_ramp_waveform(pkg, rhs_time, waveform):
    p = W.config_linear_block().with_(waveform=waveform, tau=0.5)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 30, start_mode=START_SPE, spe_depth=8, tol=1e-10, rhs_time=rhs_time)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, rhs_time=rhs_time)
    s.mqs_step(30)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    s.close()


def test_fused_solve_matches_the_literal_two_solve_reading(pkg):
    # eq. (acm) with K_n^+ applied to j and to K_cn^T a_c separately (oracle)
    # equals the single solve of the library
    p = W.config_linear_block()
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    lit = O.run_explicit_euler(d, dt, 30, start_mode=START_ZERO, tol=1e-12, literal=True)
    s = make(pkg, p, start_mode=START_ZERO, dt=dt, tol=1e-12)
    s.mqs_step(30)
    a_c, _, _ = s.get_state()
    assert rel(a_c, lit.a_c) < 1e-8
    s.close()


def test_paper_sized_grid(pkg):
    # 22^3 cells: 3*22*21^2 = 29106 interior edges, the ~30k dofs of the coarse TEAM 10 mesh
    p = W.scaled_nonlinear(22, amplitude=2e4)
    d = O.Discretization(p)
    assert d.n_c + d.n_n == 29106
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 40, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10)
    stats = s.mqs_step(40)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    assert abs(np.mean([x.iterations for x in stats]) - ref.iterations.mean()) <= 2.0
    s.close()


@pytest.mark.parametrize("variant,groups,halo", [(0, 0, 0), (1, 2, 1), (1, 3, 1), (1, 2, 2)])
def test_both_pcg_variants_match_the_oracle(pkg, variant, groups, halo):
    # groups: stencil tile groups per block of the one-reduction pass (3: 480-thread blocks);
    # halo: halo warps per group (2: 384-thread blocks)
    p = W.scaled_nonlinear(24, amplitude=5e4)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 20, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, pcg_variant=variant, tile_groups=groups,
             halo_warps=halo)
    stats = s.mqs_step(20)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    assert np.abs(np.array([x.iterations for x in stats]) - ref.iterations).max() <= 3
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = 2.0 * d.X_s[d.n_idx]
    x, info = s.pcg_solve(oracle_to_layout(p.N, b_o), tol=1e-10)
    res = O.pcg_jacobi(d.K_n, b_o[d.n_idx], None, d.D, tol=1e-10)
    assert info.status == 0 and abs(info.iterations - res.iterations) <= 3
    assert rel(d.K_cn @ layout_to_oracle(p.N, x)[d.n_idx], d.K_cn @ res.x) < 1e-9
    s.close()


@pytest.mark.parametrize("precision,choices", [(0, ((0, 0, 0), (1, 2, 1), (1, 3, 1), (1, 2, 2))),
                                               (1, ((0, 0, 0), (1, 0, 0), (1, 0, 2), (2, 0, 0)))])
def test_pcg_form_tuner_keeps_the_state_and_the_trajectory(pkg, precision, choices):
    # mqs_tune_pcg times the kernel forms on trial solves between steps: the state, the
    # step counter and the start-vector history stay as they were, and the steps after it
    # (in the chosen form) continue the oracle's trajectory
    p = W.scaled_nonlinear(24, amplitude=5e4)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 16, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, precision=precision)
    s.mqs_step(8)
    a0, t0, m0 = s.get_state()
    v = s.tune_pcg(2)
    assert v in choices and s.pcg_form() == v
    a1, t1, m1 = s.get_state()
    assert np.array_equal(a0, a1) and (t0, m0) == (t1, m1)
    stats = s.mqs_step(8)
    a_c, _, m = s.get_state()
    assert m == 16 and all(x.status == 0 for x in stats)
    assert rel(a_c, ref.a_c) < 1e-8
    # the SPE history survived the trial solves: the start vectors still cut the iterations
    assert np.mean([x.iterations for x in stats]) < 0.7 * np.mean(ref.iterations[:2])
    with pytest.raises(pkg.MqsError):
        s.tune_pcg(0)
    s.close()


# ---- mixed precision: FP32 inner solves inside FP64 refinement (same FP64 residual test) ----------
@pytest.mark.parametrize("precision,variant", [(1, 0), (1, 1), (1, 2), (2, 1)])
def test_mixed_precision_solve_meets_the_fp64_tolerance(pkg, precision, variant):
    p = W.scaled_nonlinear(35)
    d = O.Discretization(p)
    s = make(pkg, p, precision=precision, pcg_variant=variant)
    b_n = 3.0 * d.X_s[d.n_idx] - d.K_cn.T @ (W.random_vector(2, d.n_c) * 1e-9)
    b_o = np.zeros(d.grid.n_edges)
    b_o[d.n_idx] = b_n
    x, info = s.pcg_solve(oracle_to_layout(p.N, b_o), tol=1e-10)
    ref = O.pcg_jacobi(d.K_n, b_n, None, d.D, tol=1e-10)
    x_n = layout_to_oracle(p.N, x)[d.n_idx]
    assert info.status == 0 and info.relres <= 1e-10
    assert np.linalg.norm(b_n - d.K_n @ x_n) <= 1.01e-10 * np.linalg.norm(b_n)
    assert rel(d.K_cn @ x_n, d.K_cn @ ref.x) < 1e-9
    s.close()


@pytest.mark.parametrize("precision,variant,halo", [(1, 0, 0), (1, 1, 0), (1, 1, 2), (1, 2, 0), (2, 1, 0)])
@pytest.mark.parametrize("mode,name", [(START_ZERO, "zero"), (START_SPE, "spe8")])
def test_mixed_precision_steps_match_the_oracle(pkg, mode, name, precision, variant, halo):
    g = golden()
    p = W.config_linear_block()
    s = make(pkg, p, start_mode=mode, spe_depth=8, dt=g["dt"], tol=1e-10, precision=precision,
             pcg_variant=variant, halo_warps=halo)
    stats = s.mqs_step(g["steps"])
    a_c, _, _ = s.get_state()
    err = rel(a_c, np.array(g["runs"][name]["a_c"]))
    assert err < 1e-8, err           # the mixed-precision bar is 1e-6; the FP64 residual test keeps it at 1e-8
    assert all(st.status == 0 and st.relres <= 1e-10 for st in stats)
    # a step that ran inner FP32 iterations applied at least one FP64 correction; a good SPE start
    # often meets the FP64 test at the first residual and needs none
    assert all(st.refinements >= 1 for st in stats if st.iterations > 0)
    assert sum(st.refinements for st in stats) >= 1
    s.close()


@pytest.mark.parametrize("precision,variant", [(1, 0), (1, 1), (1, 2), (2, 1)])
def test_mixed_precision_full_size_agrees_with_fp64(pkg, precision, variant):
    p = W.config_nonlinear_iron()
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    s64 = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt)
    s32 = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, precision=precision, pcg_variant=variant)
    s64.mqs_step(30)
    st = s32.mqs_step(30)
    a64, _, _ = s64.get_state()
    a32, _, _ = s32.get_state()
    assert rel(a32, a64) < 1e-8
    assert all(x.status == 0 for x in st)
    if (precision, variant) == (1, 1):
        # two halo warps per group in the FP32 inner pass: bitwise the same steps
        s2 = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, precision=1, pcg_variant=1, halo_warps=2)
        st2 = s2.mqs_step(30)
        b32, _, _ = s2.get_state()
        assert np.array_equal(a32, b32)
        assert [x.iterations for x in st2] == [x.iterations for x in st]
        s2.close()
    s64.close()
    s32.close()


# ---- precision variant at 128^3: mixed precision against the FP64 GPU path at 128^3 and against
# ---- the oracle at 48^3 (block 18x18x12, coil 30x30)
def test_mixed_precision_48_matches_the_oracle(pkg):
    p = W.scaled_nonlinear(48)
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, 8, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10, precision=1, pcg_variant=1)
    st = s.mqs_step(8)
    a_c, _, _ = s.get_state()
    err = rel(a_c, ref.a_c)
    print(f"mixed precision vs oracle, 48^3, 8 steps: {err:.3e}")
    assert err < 1e-8, err
    assert all(x.status == 0 and x.relres <= 1e-10 for x in st)
    s.close()


def test_mixed_precision_128_agrees_with_fp64_over_1000_steps(pkg):
    p = W.scaled_nonlinear(128)
    # the Gershgorin step is local: the same at every size of the scaled family (pinned on the oracle)
    dt = O.dt_gershgorin(O.Discretization(W.scaled_nonlinear(24)))
    s64 = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt)
    s32 = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, precision=1, pcg_variant=1)
    worst = 0.0
    for _ in range(10):
        st64 = s64.mqs_step(100)
        st32 = s32.mqs_step(100)
        assert all(x.status == 0 for x in st64) and all(x.status == 0 and x.relres <= 1e-10 for x in st32)
        a64, _, _ = s64.get_state()
        a32, _, _ = s32.get_state()
        worst = max(worst, rel(a32, a64))
    print(f"mixed precision vs FP64, 128^3, 1000 steps: max relative a_c difference {worst:.3e}")
    assert worst < 1e-6, worst
    s64.close()
    s32.close()


# ---- eq. (anm): a_n^m of the new conductor state, on request ----------------------------------
def test_an_of_eq_anm_matches_the_oracle(pkg):
    g = golden()
    p = W.config_linear_block()
    d = O.Discretization(p)
    dt = g["dt"]
    s = make(pkg, p, start_mode=START_SPE, spe_depth=8, dt=dt, tol=1e-10)
    s.mqs_step(20)
    a_c, _, m = s.get_state()
    a_n, info = s.solve_an()
    assert info.status == 0 and info.relres <= 1e-10
    ref = O.run_explicit_euler(d, dt, 20, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    b = O.stepper.source_current(p, m * dt) * d.X_s[d.n_idx] - d.K_cn.T @ ref.a_c
    x = O.pcg_jacobi(d.K_n, b, None, d.D, 1e-12, 100000).x
    an = layout_to_oracle(p.N, a_n)[d.n_idx]
    # a_n is fixed up to null(K_n); K_cn a_n and the face fluxes C [a_c; a_n] are unique
    assert rel(d.K_cn @ an, d.K_cn @ x) < 1e-8
    assert rel(d.C @ d.full(a_c, an), d.C @ d.full(ref.a_c, x)) < 1e-8
    # the time loop continues as if nothing happened
    s.mqs_step(5)
    a5, _, _ = s.get_state()
    ref5 = O.run_explicit_euler(d, dt, 25, start_mode=START_SPE, spe_depth=8, tol=1e-10)
    assert rel(a5, ref5.a_c) < 1e-8
    s.close()


# ---- cascaded SPE (frozen past solutions + the live one) ---------------------------------------
@pytest.mark.parametrize("case", ["linear16", "iron24"])
def test_cspe_steps_match_the_oracle(pkg, case):
    if case == "linear16":
        p, steps, period, depth = W.config_linear_block(), 120, 10, 8
    else:
        p, steps, period, depth = W.scaled_nonlinear(24, amplitude=5e4), 40, 5, 6
    d = O.Discretization(p)
    dt = O.dt_gershgorin(d)
    ref = O.run_explicit_euler(d, dt, steps, start_mode=4, spe_depth=depth, tol=1e-10, cspe_period=period)
    s = make(pkg, p, start_mode=pkg.START_CSPE, spe_depth=depth, dt=dt, tol=1e-10, cspe_period=period)
    stats = s.mqs_step(steps)
    a_c, _, _ = s.get_state()
    assert rel(a_c, ref.a_c) < 1e-8
    its = np.array([x.iterations for x in stats])
    print(f"CSPE {case}: GPU iterations {its.tolist()}")
    print(f"CSPE {case}: oracle iterations {ref.iterations.tolist()}")
    # the same start vectors up to rounding: both orthogonalise at vector level (the oracle by
    # modified Gram-Schmidt over the raw columns, the GPU against its K-orthonormal frozen ones)
    assert np.abs(its - ref.iterations).max() <= 3
    assert stats[-1].rank >= 2                     # frozen columns are in use
    s.close()
