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
