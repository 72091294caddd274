"""CPU checks of the boundary: the library builds, loads and exports every
function include/cfc_gb300.h declares (no compute calls without a GPU), and
the product path does not touch the oracle."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cfc_gb300.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:lap|cfc)_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def P():
    from paper_1607_02955_gb300 import build_ext
    build_ext.build()
    import paper_1607_02955_gb300 as P
    return P


def test_library_exports_every_declared_symbol(P):
    import ctypes
    L = ctypes.CDLL(P.lib_path)
    decl = _declared()
    assert len(decl) >= 15
    missing = [s for s in decl if not hasattr(L, s)]
    assert not missing, missing
    assert set(decl) == set(P._binding.SYMBOLS)


def test_status_strings_and_defaults(P):
    assert P.lap_status_string(P.LAP_OK) == "LAP_OK"
    assert "not connected" in P.lap_status_string(P.LAP_ENOTCONN)
    o = P.lap_default_solve_opts()
    assert o.tol == 1e-8 and o.precision == P.LAP_FP32_REFINED
    h = P.lap_default_hier_opts()
    assert h.coarse_max == 0 and h.agg_passes == 2 and h.eliminate == 1 and h.reorder == 0
    assert h.aggregation == 0 and h.hub_factor == 0 and h.chunking == 0
    # options the autotuner fills in are left open; cycles are replayed as graphs
    assert (o.levels_used, o.nu_coarse, o.cycle, o.coarse_scale, o.w_levels, o.k_tile) == (0, 0, 0, 0.0, 0, 0)
    assert o.graphs == 1 and o.first_residual_ff == 1
    assert "not finished" in P.lap_status_string(P.LAP_EPENDING)
    sv = P.cfc_server_default_opts()
    assert sv.slots == 4 and sv.hbm_budget == 0 and sv.resident_pivots == 0
    assert sv.solve.tol == 1e-8 and sv.solve.graphs == 1


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1607_02955_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, flags=re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1607_02955_gb300", txt, flags=re.M), f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1607_02955_gb300 import _binding
    monkeypatch.setattr(_binding, "lib_path", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        _binding.lib()


def test_tune_table_round_trip(P, tmp_path):
    # host logic only (no GPU): a table read from JSON is written back entry
    # for entry, loading it twice adds nothing, and a malformed line is
    # rejected with LAP_EINVAL
    before = P.lap_tune_entries()
    src = tmp_path / "tune.json"
    keys = [("00000000deadbeef", 1000, 5000, 64, 1, 64, 1, 2, 2, 1, 1, 1.0, 0, 64, 1, 1, 1, 1.0, 0),
            ("0123456789abcdef", 2304, 9024, 32, 0, 32, 1, 2, 2, 4, 2, 1.5, 2, 32, 5, 4, 2, 1.5, 2)]
    lines = ['{"format": "lap_tune_v1", "entries": [']
    for i, e in enumerate(keys):
        k = '"%s", %d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %.17g, %d' % e[:13]
        c = "%d, %d, %d, %d, %.17g, %d" % e[13:]
        lines.append('{"key": [%s], "choice": [%s]}%s' % (k, c, "," if i + 1 < len(keys) else ""))
    lines.append("]}")
    src.write_text("\n".join(lines) + "\n")
    assert P.lap_tune_load(str(src)) == 2
    assert P.lap_tune_load(str(src)) == 0  # already there
    assert P.lap_tune_entries() == before + 2
    out = tmp_path / "out.json"
    P.lap_tune_save(str(out))
    text = out.read_text()
    for e in keys:
        assert '"%s", %d, %d' % e[:3] in text
    assert P.lap_tune_load(str(out)) == 0
    bad = tmp_path / "bad.json"
    bad.write_text('{"key": ["00ff", 1, 2], "choice": [1]}\n')
    with pytest.raises(P.LapError) as err:
        P.lap_tune_load(str(bad))
    assert err.value.status == P.LAP_EINVAL
    with pytest.raises(P.LapError):
        P.lap_tune_load(str(tmp_path / "missing.json"))


def test_hierarchy_options_are_checked_before_device_work(P):
    # option checks run before any CUDA call, so they hold without a GPU
    import numpy as np
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    for bad in (dict(agg_passes=0), dict(agg_passes=5), dict(eliminate=2), dict(reorder=3), dict(aggregation=2),
                dict(hub_factor=-1), dict(chunking=3), dict(coarse_max=-1)):
        with pytest.raises(P.LapError) as err:
            P.lap_build_hierarchy(3, src, dst, None, P.lap_default_hier_opts(**bad))
        assert err.value.status == P.LAP_EINVAL, bad
        assert P.lap_last_error(), bad
