"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point declared in include/mqs.h (no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    txt = open(os.path.join(ROOT, "include", "mqs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_1611_06721_gb300 as pkg
    return pkg.load()


def test_every_declared_entry_point_is_exported(lib):
    names = declared_entry_points()
    assert "mqs_setup" in names and "pcg_solve" in names and "spe_start" in names and "pod_basis" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_1611_06721_gb300 as pkg
    assert sorted(pkg.EXPORTS) == declared_entry_points()


def test_no_cpu_fallback_without_library(tmp_path, monkeypatch):
    import paper_1611_06721_gb300.binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.load()


def test_layout_mapping_round_trip():
    import numpy as np
    from tests.helpers import layout_to_oracle, oracle_to_layout, layout_index_of_oracle_edges
    import oracle as O
    for N in (3, 5):
        g = O.FitGrid(N)
        m = layout_index_of_oracle_edges(N)
        assert np.unique(m[m >= 0]).size == (m >= 0).sum() == 3 * N ** 3
        d = g.dirichlet_edges()
        assert np.all(d[m < 0])                     # unstored edges are Dirichlet
        v = np.random.default_rng(0).standard_normal(g.n_edges) * (m >= 0)
        assert np.array_equal(layout_to_oracle(N, oracle_to_layout(N, v)), v)


def test_binding_structs_match_the_header_layout(tmp_path):
    # every ctypes mirror of a header struct has the C compiler's size and field offsets
    # (a field added to the header but not to the binding would shift the ones after it)
    import ctypes
    import shutil
    import subprocess
    import paper_1611_06721_gb300.binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"mqs_grid": b.Grid, "mqs_materials": b.Materials, "mqs_coil": b.Coil, "mqs_options": b.Options,
             "mqs_layout_info": b.LayoutInfo, "mqs_adjoint_info": b.AdjointInfo, "mqs_step_stats": b.StepStats,
             "mqs_timing": b.Timing, "mqs_pcg_info": b.PcgInfo, "mqs_debug_report": b.DebugReport}
    lines = ['#include <stdio.h>', '#include "mqs.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)



def test_release_debug_check_reports_disabled(lib):
    # the release library answers without touching the device
    import ctypes
    import paper_1611_06721_gb300.binding as b
    rep = b.DebugReport(7, 7, 7, 7, 7, 7)
    assert lib.mqs_debug_check(None, ctypes.byref(rep)) == 0
    assert (rep.enabled, rep.site, rep.index, rep.faults, rep.canaries_bad, rep.buffers) == (0, 0, 0, 0, 0, 0)
    assert lib.mqs_debug_check(None, None) == -1


def test_debug_variant_builds_and_exports_the_header(tmp_path):
    import ctypes
    from paper_1611_06721_gb300 import build as bld
    path = bld.build(debug=True)
    assert path.endswith(os.path.join("_lib_debug", "libmqs.so"))
    dbg = ctypes.CDLL(path)
    missing = [n for n in declared_entry_points() if not hasattr(dbg, n)]
    assert not missing, missing
