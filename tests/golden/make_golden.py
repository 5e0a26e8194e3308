"""Writes the stored expected values used by the GPU parity tests.

Calls only the FP64 oracle (and the seeded input generators): the 16^3
linear-block problem (4^3 conductor, sigma 1e6 S/m, 10x10 coil, 1 A at 50 Hz),
lambda_max of M_c^-1 K_S by the power method (eq. (CFL)), dt = 0.9 * 2 /
lambda_max, and 200 explicit-Euler steps (eq. (acm)) for every start vector
(zero, previous, SPE with 8 columns, POD with 20 snapshots; Sec. III).

With --iron64: lambda_max and dt = 0.9 * 2 / lambda_max of the 64^3 nonlinear
iron workload (24x24x16 Brauer iron, sigma 2e6 S/m, 40x40 coil, 500 A at 50 Hz)
by the same power method (PCG tol 1e-12, stop at |dlambda| < 1e-8 lambda), for
the parity test that runs both sides on that workload with this step.

Run:  python tests/golden/make_golden.py [--iron64]
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    p = W.config_linear_block()
    d = O.Discretization(p)
    lam, it = O.lambda_max_power(d, W.power_start_vector(d.n_c))
    dt = O.dt_from_lambda(lam)
    out = {"problem": p.name, "N": p.N, "n_c": int(d.n_c), "n_n": int(d.n_n),
           "lambda_max": lam, "power_iterations": it, "dt": dt, "steps": p.n_steps,
           "tol": 1e-10, "runs": {}}
    for mode, name in ((0, "zero"), (1, "prev"), (2, "spe8"), (3, "pod20")):
        r = O.run_explicit_euler(d, dt, p.n_steps, start_mode=mode, spe_depth=8, pod_snapshots=20, tol=1e-10)
        out["runs"][name] = {"a_c": r.a_c.tolist(), "iterations": r.iterations.tolist(),
                             "mean_iterations": float(r.iterations.mean())}
        print(name, r.iterations.mean(), np.linalg.norm(r.a_c))
    with open(os.path.join(HERE, "linear_block_16.json"), "w") as f:
        json.dump(out, f, indent=0)


def iron64():
    p = W.config_nonlinear_iron()
    d = O.Discretization(p)
    lam, it = O.lambda_max_power(d, W.power_start_vector(d.n_c))
    out = {"problem": "nonlinear iron 64^3", "N": p.N, "n_c": int(d.n_c), "n_n": int(d.n_n),
           "lambda_max": lam, "power_iterations": it, "cfl_factor": 0.9, "dt": O.dt_from_lambda(lam)}
    print(out)
    with open(os.path.join(HERE, "nonlinear_iron_64.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    if "--iron64" in sys.argv:
        iron64()
    else:
        main()
