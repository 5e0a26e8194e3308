"""The synthetic inputs are the workloads the measurements name: the 16^3 linear block,
the 64^3 Brauer-iron block, the geometry scaled with N, and the seeded multi-query set.
Host-only checks of the generators (no GPU, no oracle arithmetic)."""
import numpy as np

import workloads as W


def _box(mask):
    """[lo, hi) per axis (k, j, i) of the flagged cells, which must fill that box."""
    idx = np.nonzero(mask)
    lo = [int(a.min()) for a in idx]
    hi = [int(a.max()) + 1 for a in idx]
    assert mask.sum() == np.prod([h - l for l, h in zip(lo, hi)])
    return lo, hi


def test_linear_block_16():
    p = W.config_linear_block()
    assert p.N == 16 and p.h == 1e-3 and p.amplitude == 1.0 and p.freq == 50.0 and p.waveform == 0
    lo, hi = _box(p.sigma_cell > 0)
    assert lo == [6, 6, 6] and hi == [10, 10, 10]                 # cells 6..9 on every axis
    assert np.all(p.sigma_cell[p.sigma_cell > 0] == 1e6) and not p.brauer_cell.any()
    assert (p.coil_k, p.coil_i0, p.coil_j0, p.coil_i1, p.coil_j1) == (8, 3, 3, 13, 13)   # 10 x 10 at z = 8


def test_nonlinear_iron_64():
    p = W.config_nonlinear_iron()
    assert p.N == 64 and p.amplitude == 500.0 and p.freq == 50.0
    lo, hi = _box(p.sigma_cell > 0)
    assert lo == [24, 20, 20] and hi == [40, 44, 44]             # z 24..39, y and x 20..43
    assert np.all(p.sigma_cell[p.sigma_cell > 0] == 2e6)
    assert np.array_equal(p.brauer_cell.astype(bool), p.sigma_cell > 0)
    assert (p.k1, p.k2, p.k3) == (3.8, 2.17, 396.2)
    assert (p.coil_k, p.coil_i1 - p.coil_i0, p.coil_j1 - p.coil_j0) == (32, 40, 40)
    assert p.coil_i0 == p.coil_j0 == 12                          # centred


def test_geometry_scales_with_n():
    for N in (12, 32, 40, 48, 128):
        p = W.scaled_nonlinear(N)
        sxy, sz = round(24 * N / 64), round(16 * N / 64)
        lo, hi = _box(p.sigma_cell > 0)
        assert [h - l for l, h in zip(lo, hi)] == [sz, sxy, sxy]
        assert lo == [(N - sz) // 2, (N - sxy) // 2, (N - sxy) // 2]
        L = round(10 * N / 16)
        assert p.coil_k == N // 2 and p.coil_i1 - p.coil_i0 == L and p.coil_i0 == (N - L) // 2
        assert 0 < p.coil_i0 and p.coil_i1 < N                  # the loop stays off the Dirichlet boundary


def test_multi_query_set_is_seeded():
    a = W.batched_instances(64)
    b = W.batched_instances(64)
    assert len(a) == 64
    for x, y in zip(a, b):
        assert x.N == y.N and x.amplitude == y.amplitude and np.array_equal(x.sigma_cell, y.sigma_cell)
    sizes = {p.N for p in a}
    assert sizes == {32, 40, 48, 64}
    for p in a:
        s = float(p.sigma_cell.max())
        assert 1e6 <= s <= 5e6 and 100.0 <= p.amplitude <= 1000.0
        assert np.all(p.sigma_cell[p.sigma_cell > 0] == s)
        assert np.array_equal(p.brauer_cell.astype(bool), p.sigma_cell > 0)
    c = W.batched_instances(64, seed=7)
    assert any(x.amplitude != y.amplitude for x, y in zip(a, c))
