"""The autotuner's table: choices are kept per graph (its fingerprint), and
a saved table makes another process repeat the choice and the solve's bits.

A 32 x 32 torus and a random 4-regular graph have the same size (n = 1024,
2048 edges) and the same degrees, but different structure: each gets its own
entry, and both solves converge (FP64 residual checked on the CPU)."""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import synth
from oracle.graph import canonical_graph, laplacian

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02955_gb300 import build_ext
    build_ext.build()
    import paper_1607_02955_gb300 as P
    torch.cuda.init()
    return P


def _solve(P, gen, B):
    import torch
    n, s, d, w = gen
    h = P.lap_build_hierarchy(n, s, d, w)
    X = torch.empty((n, B.shape[1]), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts())
    return P.lap_hierarchy_info(h)["fingerprint"], info, X.cpu().numpy()


def test_equal_size_graphs_are_tuned_separately_and_a_saved_table_repeats_the_bits(P, tmp_path):
    torus, regular = synth.torus2d(32), synth.random_regular(1024, 4, seed=7)
    B = np.random.default_rng(8).standard_normal((1024, 24))
    before = P.lap_tune_entries()
    fp_t, info_t, X_t = _solve(P, torus, B)
    fp_r, info_r, X_r = _solve(P, regular, B)
    assert fp_t != fp_r
    assert P.lap_tune_entries() == before + 2
    for gen, X, info in ((torus, X_t, info_t), (regular, X_r, info_r)):
        assert info["max_rel_residual"] <= 1e-8
        g = canonical_graph(*gen)
        Bp = B - B.mean(axis=0)
        assert np.all(np.linalg.norm(Bp - laplacian(g) @ X, axis=0) <= 1.01e-8 * np.linalg.norm(Bp, axis=0))
    # the same graph again: the table answers, nothing is tuned
    _, info_t2, X_t2 = _solve(P, torus, B)
    assert P.lap_tune_entries() == before + 2 and np.array_equal(X_t2, X_t)
    table = tmp_path / "tune.json"
    P.lap_tune_save(str(table))
    entries = json.loads(table.read_text())["entries"]
    assert {int(e["key"][0], 16) for e in entries} >= {fp_t, fp_r}
    np.save(tmp_path / "B.npy", B)
    # a fresh process loads the table: same choice, same bits, no new entry
    script = textwrap.dedent(f"""
        import sys, json
        import numpy as np
        sys.path.insert(0, {ROOT!r})
        import torch, synth
        import paper_1607_02955_gb300 as P
        torch.cuda.init()
        added = P.lap_tune_load({str(table)!r})
        n, s, d, w = synth.torus2d(32)
        h = P.lap_build_hierarchy(n, s, d, w)
        B = torch.tensor(np.load({str(tmp_path / 'B.npy')!r}), device="cuda")
        X = torch.empty_like(B)
        info = P.lap_solve_multi(h, B, X, P.lap_default_solve_opts())
        np.save({str(tmp_path / 'X.npy')!r}, X.cpu().numpy())
        print(json.dumps({{"added": added, "entries": P.lap_tune_entries(),
                          "choice": [info[k] for k in ("k_tile", "levels_used", "nu_coarse", "cycle",
                                                       "coarse_scale", "w_levels")]}}))
    """)
    out = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    child = json.loads(out.stdout.strip().splitlines()[-1])
    assert child["added"] == len(entries) and child["entries"] == len(entries)
    assert child["choice"] == [info_t[k] for k in ("k_tile", "levels_used", "nu_coarse", "cycle", "coarse_scale",
                                                   "w_levels")]
    assert np.array_equal(np.load(tmp_path / "X.npy"), X_t)


def test_tune_table_errors(P, tmp_path):
    with pytest.raises(P.LapError):
        P.lap_tune_load(str(tmp_path / "missing.json"))
    bad = tmp_path / "bad.json"
    bad.write_text('{"format": "lap_tune_v1", "entries": [\n{"key": ["zz", 1], "choice": []}\n]}\n')
    with pytest.raises(P.LapError):
        P.lap_tune_load(str(bad))
