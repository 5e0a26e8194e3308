"""The allocation-free PCG entry point (mqs_pcg_solve_noalloc) against the
handle-based pcg_solve.

Some callers of this library cannot allocate device memory themselves or let
the library do it: their device memory belongs to their own pool allocator,
or they run a real-time loop where an allocation may synchronise the device.
mqs_pcg_solve_noalloc serves them from a fixed static scratch array.  This
file is collected last so that a run stopping at the first failure has run
every other test before it; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.helpers import layout_to_oracle, oracle_to_layout, rel

pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as g
    g.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1611_06721_gb300 as pkg
    from paper_1611_06721_gb300.binding import pcg_solve_noalloc
    return pkg, torch, pcg_solve_noalloc


def _rhs(d, p, scale, seed):
    a_c = W.random_vector(seed, d.n_c) * 1e-9
    b_n = scale * d.X_s[d.n_idx] - d.K_cn.T @ a_c
    return b_n, oracle_to_layout(p.N, d.full(None, b_n))


@pytest.mark.parametrize("N", [16, 35])
def test_noalloc_matches_pcg_solve_twice(env, N):
    pkg, torch, noalloc = env
    p = W.config_linear_block() if N == 16 else W.scaled_nonlinear(N)
    d = O.Discretization(p)
    s = pkg.Solver.from_problem(p, pkg.SolverOptions())
    mask = torch.tensor((p.sigma_cell > 0).astype(np.uint8).reshape(-1), device="cuda")
    for call, (scale, seed) in enumerate(((3.0, 1), (-0.5, 2))):      # two calls in a row
        b_n, b_l = _rhs(d, p, scale, seed)
        x_ref, info_ref = s.pcg_solve(b_l, tol=1e-10)
        b = torch.tensor(b_l, device="cuda")
        x = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        rc, info = noalloc(N, p.h, p.nu0, mask, b, x, tol=1e-10)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call (which loaded the module), a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        assert rc == 0 and info.status == 0 and info.relres <= 1e-10, (call, rc, info.status)
        assert abs(info.iterations - info_ref.iterations) <= 3
        xg = x.cpu().numpy()
        x_n, xr_n = layout_to_oracle(N, xg)[d.n_idx], layout_to_oracle(N, x_ref)[d.n_idx]
        assert rel(d.K_cn @ x_n, d.K_cn @ xr_n) < 1e-9
        assert np.linalg.norm(b_n - d.K_n @ x_n) <= 1.01e-10 * np.linalg.norm(b_n)
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    pkg, torch, noalloc = env
    N = 49
    mask = torch.zeros(N ** 3, dtype=torch.uint8, device="cuda")
    b = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    rc, _ = noalloc(N, 1e-3, 1.0 / (4e-7 * np.pi), mask, b, x)
    assert rc == -1                                         # MQS_ERR_ARG
