"""FP64 CPU oracle for the semi-explicit eddy-current scheme (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct reference that the CUDA path
is checked against.  It assembles the FIT incidence matrices explicitly as
sparse matrices and follows the paper's equations step by step:

* Sec. II, eq. (DAE)  - block system with the conducting / nonconducting split
* Sec. II, eq. (SC)   - generalised Schur complement (applied, never formed)
* Sec. II, eqs. (ODE), (a_n), (acm), (anm), (CFL) - explicit Euler, step bound
* Sec. III, eq. (mrhs) - PCG evaluation of the pseudo-inverse of K_n
* Sec. III, eq. (SPE_x0) - SPE start vector (modified Gram-Schmidt + Galerkin)
* Sec. III, eqs. (SVD), (relSV2), (keepInfo), (POD_x0) - POD start vector

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
may import it; the product library never does and shares no code with it.

Parity status of each function is stated in its docstring; every function here
is pinned by a ``-m "not gpu"`` test against closed forms, invariants or
brute-force dense linear algebra on tiny grids.
"""
from .fit_grid import FitGrid  # noqa: F401
from .operators import Discretization  # noqa: F401
from .pcg import pcg_jacobi, PcgResult  # noqa: F401
from .mrhs import mgs_orthonormal_basis, spe_start, pod_start  # noqa: F401
from .stepper import (  # noqa: F401
    run_explicit_euler, lambda_max_power, dt_from_lambda, dt_gershgorin,
    source_current,
)
