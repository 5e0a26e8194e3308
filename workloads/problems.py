"""Problem descriptions (inputs only) for the eddy-current time stepper.

Conventions shared by every consumer of these inputs:

* The grid has ``N`` cells per axis, spacing ``h`` metres, nodes ``0..N`` per axis.
* Cell arrays are ``float64``/``uint8`` of shape ``(N, N, N)`` indexed
  ``[k, j, i]`` (x fastest), i.e. flat index ``i + N*(j + N*k)``.
* The coil is one rectangular loop of grid edges in node plane ``k = coil_k``
  around the node square ``[i0, i1] x [j0, j1]``, counter-clockwise seen from
  ``+z``; its current is ``i(t) = amplitude * sin(2 pi freq t)`` (waveform 0)
  or ``amplitude * (1 - exp(-t/tau))`` (waveform 1, the excitation used in the
  paper's TEAM 10 validation, Sec. IV).
* Cells flagged in ``brauer_cell`` use the Brauer reluctivity
  ``nu(B) = k1 exp(k2 B^2) + k3``; all other cells use ``nu0 = 1/mu0``.
  A Brauer cell must also conduct (``sigma > 0``), so the nonconducting
  curl-curl matrix stays constant (Sec. II, "typically constant").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

NU0 = 1.0 / (4.0e-7 * math.pi)          # reluctivity of vacuum [m/H]
BRAUER_STEEL = (3.8, 2.17, 396.2)        # k1 [m/H], k2 [1/T^2], k3 [m/H]


@dataclass
class Problem:
    """One synthetic magnetoquasistatic problem (inputs only)."""
    N: int
    h: float
    sigma_cell: np.ndarray               # (N,N,N) float64, S/m, 0 = nonconducting
    brauer_cell: np.ndarray              # (N,N,N) uint8, 1 = Brauer iron
    coil_k: int
    coil_i0: int
    coil_j0: int
    coil_i1: int
    coil_j1: int
    amplitude: float                     # A
    freq: float = 50.0                   # Hz
    waveform: int = 0                    # 0 sin, 1 1-exp(-t/tau)
    tau: float = 0.5                     # s
    nu0: float = NU0
    k1: float = BRAUER_STEEL[0]
    k2: float = BRAUER_STEEL[1]
    k3: float = BRAUER_STEEL[2]
    n_steps: int = 200
    name: str = ""
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)


def _coil_square(N: int):
    L = int(round(10 * N / 16))
    c0 = (N - L) // 2
    return N // 2, c0, c0, c0 + L, c0 + L


def config_linear_block(N: int = 16, n_steps: int = 200) -> Problem:
    """Linear 4x4x4 conducting block (sigma = 1e6 S/m, mu_r = 1) at cells 6..9
    of a 16^3 grid, 10x10 coil in node plane z = 8, 1 A at 50 Hz."""
    sigma = np.zeros((N, N, N))
    s, o = 4 * N // 16, (N - 4 * N // 16) // 2
    sigma[o:o + s, o:o + s, o:o + s] = 1.0e6
    k, i0, j0, i1, j1 = _coil_square(N)
    return Problem(N=N, h=1.0e-3, sigma_cell=sigma,
                   brauer_cell=np.zeros((N, N, N), np.uint8),
                   coil_k=k, coil_i0=i0, coil_j0=j0, coil_i1=i1, coil_j1=j1,
                   amplitude=1.0, n_steps=n_steps, name=f"linear-block-{N}^3")


def scaled_nonlinear(N: int, sigma: float = 2.0e6, amplitude: float = 500.0,
                     n_steps: int = 2000) -> Problem:
    """Brauer iron block round(24N/64) x round(24N/64) x round(16N/64) centred
    in an N^3 grid, coil of side round(10N/16) in node plane N/2."""
    sxy, sz = int(round(24 * N / 64)), int(round(16 * N / 64))
    oxy, oz = (N - sxy) // 2, (N - sz) // 2
    sig = np.zeros((N, N, N))
    sig[oz:oz + sz, oxy:oxy + sxy, oxy:oxy + sxy] = sigma
    br = (sig > 0).astype(np.uint8)
    k, i0, j0, i1, j1 = _coil_square(N)
    return Problem(N=N, h=1.0e-3, sigma_cell=sig, brauer_cell=br,
                   coil_k=k, coil_i0=i0, coil_j0=j0, coil_i1=i1, coil_j1=j1,
                   amplitude=amplitude, n_steps=n_steps,
                   name=f"nonlinear-iron-{N}^3")


def config_nonlinear_iron() -> Problem:
    """64^3 grid, Brauer iron 24x24x16 at cells (20..43, 20..43, 24..39),
    sigma = 2e6 S/m, 40x40 coil at z = 32, 500 A at 50 Hz, 2000 steps."""
    return scaled_nonlinear(64)


def random_problem(seed: int, N: int = 6, brauer: bool = False,
                   amplitude: float = 1.0) -> Problem:
    """Small random problem for property tests: one or two random conducting
    boxes (random sigma per cell), a coil loop that avoids them."""
    rng = np.random.default_rng(seed)
    sig = np.zeros((N, N, N))
    nbox = int(rng.integers(1, 3)) if N > 5 else 1
    for _ in range(nbox):
        lo = rng.integers(1, N - 2, size=3)
        ext = rng.integers(1, 3, size=3)
        if N <= 5:
            ext[2] = 1            # leave a free node plane for the coil
        hi = np.minimum(lo + ext, N - 1)
        sig[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = rng.uniform(1e5, 5e6, size=tuple(hi[::-1] - lo[::-1]))
    br = ((sig > 0) & brauer).astype(np.uint8)
    # first rectangular loop (largest side first, scanning node planes and
    # positions) whose edges touch no conducting cell
    cond = sig > 0

    def touches(k, i0, j0, i1, j1):
        for kk in (k - 1, k):
            if not 0 <= kk < N:
                continue
            for t in range(i0, i1):
                for f in (j0 - 1, j0, j1 - 1, j1):
                    if 0 <= f < N and cond[kk, f, t]:
                        return True
            for t in range(j0, j1):
                for f in (i0 - 1, i0, i1 - 1, i1):
                    if 0 <= f < N and cond[kk, t, f]:
                        return True
        return False

    for L in range(N - 2, 0, -1):
        for k in range(1, N):
            for i0 in range(1, N - L):
                for j0 in range(1, N - L):
                    if not touches(k, i0, j0, i0 + L, j0 + L):
                        return Problem(N=N, h=1.0e-3, sigma_cell=sig, brauer_cell=br,
                                       coil_k=k, coil_i0=i0, coil_j0=j0, coil_i1=i0 + L,
                                       coil_j1=j0 + L, amplitude=amplitude, n_steps=20,
                                       name=f"random-{seed}-{N}^3")
    raise ValueError("no coil placement clear of the conductors")


def random_vector(seed: int, n: int) -> np.ndarray:
    """Seeded standard-normal float64 vector (used as generic test data)."""
    return np.random.default_rng(seed).standard_normal(n)


def power_start_vector(n_c: int, seed: int = 1611) -> np.ndarray:
    """Start vector of the power iteration for lambda_max (seeded Gaussian on
    the conducting unknowns); both implementations receive it as an input."""
    return np.random.default_rng(seed).standard_normal(n_c)


def batched_instances(count: int = 64, seed: int = 1611, sizes=(32, 40, 48, 64)):
    """Multi-query instances: N from `sizes` (default {32, 40, 48, 64}), sigma ~
    U[1e6, 5e6], amplitude ~ U[100, 1000] A, Brauer iron scaled with N."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        N = int(rng.choice(list(sizes)))
        sig = float(rng.uniform(1e6, 5e6))
        amp = float(rng.uniform(100.0, 1000.0))
        out.append(scaled_nonlinear(N, sigma=sig, amplitude=amp, n_steps=500).with_(name=f"instance-{q}-{N}^3"))
    return out
