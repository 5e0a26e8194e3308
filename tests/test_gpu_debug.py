"""The debug variant of the library (compiled with MQS_DEBUG_CHECKS): every index a
hot kernel computes is range-checked and every device buffer carries guard bytes.
A child process loads it (MQS_DEBUG=1), runs the stepping paths -- FP64 PCG in
both forms, the FP32 inner passes, the float-float inner solve, separate
right-hand sides, CSPE, POD, the adjoint, a batch -- and the stand-alone calls,
then reads mqs_debug_check: no index may have left its array and no guard byte
may have changed.  The same problems run in the release library must give the
same states (the checks only guard accesses, they do not change arithmetic).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import workloads as W
import paper_1611_06721_gb300 as pkg

out = {"lib": pkg.LIB_PATH, "states": {}}
p = W.scaled_nonlinear(24)
cases = {
    "fp64_cg": dict(start_mode=pkg.START_SPE, spe_depth=4, pcg_variant=0),
    "fp64_fused": dict(start_mode=pkg.START_SPE, spe_depth=4, pcg_variant=1),
    "fp32_v1": dict(start_mode=pkg.START_SPE, spe_depth=4, precision=1, pcg_variant=1),
    "fp32_v2": dict(start_mode=pkg.START_SPE, spe_depth=4, precision=1, pcg_variant=2),
    "ff": dict(start_mode=pkg.START_SPE, spe_depth=4, precision=2),
    "split": dict(start_mode=pkg.START_SPE, spe_depth=4, rhs_split=1),
    "cspe": dict(start_mode=pkg.START_CSPE, spe_depth=4, cspe_period=3),
    "pod": dict(start_mode=pkg.START_POD, pod_snapshots=6),
    "graph": dict(start_mode=pkg.START_SPE, spe_depth=4, graph=1),
}
solvers = []
for name, kw in cases.items():
    s = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, cfl_factor=0.9, **kw))
    s.mqs_step(12)
    a_c, t, m = s.get_state()
    out["states"][name] = a_c.tolist()
    solvers.append(s)
s = solvers[0]
rng = np.random.default_rng(5)
y = s.apply_kn(rng.standard_normal(s.n_layout))
out["apply"] = float(np.abs(y).sum())
b = pkg.Batch([pkg.Solver.from_problem(W.scaled_nonlinear(n), pkg.SolverOptions(tol=1e-10, cfl_factor=0.9,
               start_mode=pkg.START_SPE, spe_depth=4)) for n in (16, 20)])
b.step(6)
out["batch"] = [sv.get_state()[0].tolist() for sv in b.solvers]
sa = pkg.Solver.from_problem(p, pkg.SolverOptions(tol=1e-10, cfl_factor=0.9, start_mode=pkg.START_SPE,
                                                  spe_depth=4))
J, g, gI, _ = sa.adjoint(6)
J2, g2, gI2, _ = sa.adjoint(6, checkpoint_every=2)
out["grad"] = [float(J), float(np.abs(g).sum()), float(gI), float(J2), float(np.abs(g2).sum())]
solvers.append(sa)
out["check"] = pkg.debug_check(solvers + list(b.solvers))
b.close()
for sv in solvers:
    sv.close()
print("RESULT " + json.dumps(out))
"""


def run_child(debug):
    env = dict(os.environ)
    env["MQS_DEBUG"] = "1" if debug else "0"
    code = "ROOT = %r\n" % ROOT + CHILD
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    line = [ln for ln in res.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    from paper_1611_06721_gb300 import build as bld
    bld.build(debug=True)


def test_debug_variant_is_clean_and_agrees_with_release(built):
    import numpy as np
    dbg = run_child(True)
    rel_ = run_child(False)
    assert dbg["lib"].endswith(os.path.join("_lib_debug", "libmqs.so"))
    chk = dbg["check"]
    assert chk["enabled"] == 1
    assert chk["faults"] == 0, f"index out of range at site {chk['site']}: {chk['index']}"
    assert chk["buffers"] > 100 and chk["canaries_bad"] == 0
    assert rel_["check"]["enabled"] == 0
    for name, a in dbg["states"].items():
        a, b = np.asarray(a), np.asarray(rel_["states"][name])
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), name
    for a, b in zip(dbg["batch"], rel_["batch"]):
        a, b = np.asarray(a), np.asarray(b)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    assert abs(dbg["apply"] - rel_["apply"]) <= 1e-12 * abs(rel_["apply"])
    for a, b in zip(dbg["grad"], rel_["grad"]):
        assert abs(a - b) <= 1e-9 * max(abs(b), 1e-300)
