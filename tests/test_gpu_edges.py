"""Parity on the paths the large workloads take, and the method's edge cases
(through the C ABI, against the CPU oracle).

* R-MAT (skewed degrees, Sec. 6.3's complex networks): scale 14, largest
  connected component.  Its row lengths are uneven enough that the row
  kernels take the rows longest first, and its hubs are split into chunks:
  the paths the R-MAT benchmark runs.
* Pinned configurations the autotuner may or may not pick: every level of
  the hierarchy in FP32 and FP64, and the 128-column tile.
* Inputs at the edge of the arithmetic: a right-hand side with a non-finite
  entry is rejected; conductances of any magnitude (Sec. 2 allows any
  positive weight) give the oracle's answer, scaled (L(c w) = c L(w), so the
  farness of c w is the farness of w over c); weights spanning 80 orders of
  magnitude either converge or report LAP_ENOCONV, never LAP_OK with a
  non-finite value.
* The aggregation options of Sec. 3.1 (LAMG's affinity-based aggregation,
  and hubs kept out of aggregates): every combination gives the oracle's
  answer; the hub rule does what it says on a star.
"""
import numpy as np
import pytest

import synth
from oracle import dense, jl
from oracle.graph import canonical_graph, laplacian

pytestmark = pytest.mark.gpu

FARNESS_RTOL = 1e-6


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


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300))


PRECISIONS = {"fp32": dict(precision=1), "fp64": dict(precision=0),
              "bf16coarse": dict(precision=2, levels_used=-1),
              "fp32_all_levels": dict(precision=1, levels_used=-1),
              "fp64_all_levels": dict(precision=0, levels_used=-1),
              # one level, one smoothing step: Jacobi-PCG, the fused path R-MAT takes
              "fp32_jacobi": dict(precision=1, levels_used=1, nu_coarse=1),
              "fp64_jacobi": dict(precision=0, levels_used=1, nu_coarse=1)}


@pytest.fixture(scope="module")
def rmat14():
    n, s, d, _ = synth.rmat(14, seed=3)
    w = synth.uniform_weights(s.size, seed=5)
    return n, s, d, w, canonical_graph(n, s, d, w)


def _certify(g, B, X, tol=1e-8):
    """Independent FP64 residual check on the CPU: ||Bp - L X|| <= tol ||Bp||
    per column, Bp the zero-mean projection of B, and X of zero mean."""
    Bp = B - B.mean(axis=0)
    R = Bp - laplacian(g) @ X
    assert np.all(np.linalg.norm(R, axis=0) <= 1.01 * tol * np.linalg.norm(Bp, axis=0))
    np.testing.assert_allclose(X.mean(axis=0), 0, atol=1e-12 * np.abs(X).max())


# ------------------------------------------------------------------ R-MAT: longest-first rows, split hubs
def test_rmat_takes_the_longest_first_row_order(P, rmat14):
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w)
    info = P.lap_hierarchy_info(h)
    assert info["level_row_order"][0] == 1
    assert np.bincount(np.concatenate([s, d])).max() > 128  # hubs: rows split into several chunks
    grid = P.lap_build_hierarchy(*synth.grid2d(32)[:3])
    assert P.lap_hierarchy_info(grid)["level_row_order"][0] == 0


@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_rmat_solve_is_certified(P, rmat14, precision):
    import torch
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w)
    B = np.random.default_rng(2).standard_normal((n, 40))
    Xt = torch.empty((n, 40), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), Xt, P.lap_default_solve_opts(**PRECISIONS[precision]))
    assert info["max_rel_residual"] <= 1e-8
    _certify(g, B, Xt.cpu().numpy())


@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_rmat_farness_jl_matches_oracle(P, rmat14, precision):
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w)
    hub = int(np.argmax(np.bincount(np.concatenate([s, d]))))
    nodes = np.array([0, hub, n // 2, n - 1], np.int32)
    f = P.cfc_farness_jl(h, 32, 4, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    fo = jl.jl_farness(g, 32, 4, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL


@pytest.mark.parametrize("levels", [0, -1])
def test_rmat_k128_tile128(P, rmat14, levels):
    import torch
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w)
    opts = P.lap_default_solve_opts(k_tile=128, levels_used=levels)
    B = np.random.default_rng(3).standard_normal((n, 128))
    Xt = torch.empty((n, 128), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), Xt, opts)
    assert info["k_tile"] == 128 and info["max_rel_residual"] <= 1e-8
    _certify(g, B, Xt.cpu().numpy())
    nodes = np.array([1, n - 2], np.int32)
    f = P.cfc_farness_jl(h, 128, 6, nodes, opts=opts)
    fo = jl.jl_farness(g, 128, 6, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL


# ------------------------------------------------------------------ non-finite right-hand sides
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 1e200])
def test_nonfinite_rhs_is_rejected(P, bad):
    import torch
    n, s, d, _ = synth.grid2d(20)
    h = P.lap_build_hierarchy(n, s, d)
    B = np.random.default_rng(0).standard_normal((n, 8))
    B[17, 3] = bad  # 1e200 is finite, but its square is not
    X = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(P.LapError) as e:
        P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X)
    assert e.value.status == P.LAP_EINVAL


# ------------------------------------------------------------------ conductances far from 1
SCALES = [2.0 ** 133, 2.0 ** -133, 1e40, 1e-40]


@pytest.mark.parametrize("c", SCALES)
@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_weights_far_from_one_scale_the_farness(P, c, precision):
    n, s, d, _ = synth.grid2d(16)
    w = synth.uniform_weights(s.size, seed=3)
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w * c)
    assert P.lap_hierarchy_info(h)["weight_exp"] == int(np.floor(np.log2((w * c).max())))
    nodes = np.array([0, 37, n - 1], np.int32)
    f = P.cfc_farness_jl(h, 32, 2, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    assert np.all(np.isfinite(f))
    # L(c w) = c L(w): Z scales by c^-1/2 (Y by c^1/2), the farness by 1/c
    fo = jl.jl_farness(g, 32, 2, nodes.tolist(), solver="dense")
    assert _rel(f * c, fo) <= FARNESS_RTOL


@pytest.mark.parametrize("c", SCALES)
def test_exact_small_with_weights_far_from_one(P, c):
    n, s, d, _ = synth.grid2d(12, 9)
    w = synth.uniform_weights(s.size, seed=4)
    g = canonical_graph(n, s, d, w)
    f, cl = P.cfc_exact_small(n, s, d, w * c)
    assert _rel(f * c, dense.farness(g)) <= 1e-9
    assert _rel(cl / c, dense.closeness(g)) <= 1e-9


@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_weights_spanning_80_orders_never_ok_with_nonfinite(P, precision):
    import torch
    n, s, d, _ = synth.grid2d(16)
    w = np.where(np.random.default_rng(1).random(s.size) < 0.5, 1e40, 1e-40)
    h = P.lap_build_hierarchy(n, s, d, w)
    opts = P.lap_default_solve_opts(**PRECISIONS[precision])
    try:
        f = P.cfc_farness_jl(h, 32, 2, np.array([0, 100], np.int32), opts=opts)
        assert np.all(np.isfinite(f)) and np.all(f > 0)
    except P.LapError as e:
        assert e.status == P.LAP_ENOCONV
    B = torch.tensor(np.random.default_rng(5).standard_normal((n, 16)), device="cuda")
    X = torch.empty_like(B)
    info = P.lap_solve_multi(h, B, X, opts, allow_noconv=True)
    if info["status"] == P.LAP_OK:
        assert info["max_rel_residual"] <= 1e-8 and bool(torch.isfinite(X).all())
    else:
        assert info["status"] == P.LAP_ENOCONV
        assert not (info["max_rel_residual"] <= 1e-8)


# ------------------------------------------------------------------ low-degree elimination (Sec. 3.1, LAMG)
@pytest.mark.parametrize("gen", [lambda: synth.path_graph(300), lambda: synth.random_tree(400, seed=3)])
def test_elimination_then_dense_solve_is_exact(P, gen):
    # on a path or a tree, eliminating the nodes with one or two neighbours
    # leaves a graph small enough for the dense solve: elimination, dense
    # solve and back-substitution are then an exact preconditioner, so FP64
    # PCG takes at most two iterations in its one refinement step
    import torch
    n, s, d, _ = gen()
    w = synth.uniform_weights(s.size, seed=9)
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(coarse_max=256))
    info = P.lap_hierarchy_info(h)
    assert info["elim_levels"] == 1 and info["levels"] == 2
    assert info["level_n"][1] <= 256 and info["coarse_n"] == info["level_n"][1]
    B = np.random.default_rng(1).standard_normal((n, 16))
    X = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    # convergence read after every inner iteration, so the count is exact
    si = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(precision=0, check_every=1))
    # what is left is FP64 rounding: about eps x cond(L) of the eliminated graph
    # (a weighted path of ~150 nodes: cond ~ 1e4, so ~1e-12), far below the 1e-8 target
    assert si["outer_iters"] == 1 and si["inner_iters"] <= 2 and si["max_rel_residual"] < 1e-10
    _certify(canonical_graph(n, s, d, w), B, X.cpu().numpy(), tol=1e-10)


def test_elimination_applies_where_it_removes_nodes(P, rmat14):
    n, s, d, w, g = rmat14
    on = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, w))
    assert on["elim_levels"] == 1 and on["level_n"][1] < 0.8 * n
    off = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eliminate=0)))
    assert off["elim_levels"] == 0
    for gen in (lambda: synth.grid2d(40), lambda: synth.barabasi_albert(3000, 5, seed=2)):
        assert P.lap_hierarchy_info(P.lap_build_hierarchy(*gen()[:3]))["elim_levels"] == 0


@pytest.mark.parametrize("eliminate", [0, 1])
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_all_levels"])
def test_rmat_farness_with_and_without_elimination(P, rmat14, eliminate, precision):
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eliminate=eliminate))
    nodes = np.array([3, n // 3], np.int32)
    f = P.cfc_farness_jl(h, 48, 8, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    fo = jl.jl_farness(g, 48, 8, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL


# ------------------------------------------------------------------ aggregation: affinity, hub rule (Sec. 3.1)
AGGREGATIONS = {"strength": dict(aggregation=0), "affinity": dict(aggregation=1),
                "strength_hubs": dict(aggregation=0, hub_factor=4),
                "affinity_hubs": dict(aggregation=1, hub_factor=4)}


@pytest.mark.parametrize("agg", sorted(AGGREGATIONS))
@pytest.mark.parametrize("precision", ["fp32_all_levels", "fp64_all_levels", "bf16coarse"])
def test_rmat_farness_with_each_aggregation(P, rmat14, agg, precision):
    n, s, d, w, g = rmat14
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1, **AGGREGATIONS[agg]))
    assert P.lap_hierarchy_info(h)["levels"] >= 3
    hub = int(np.argmax(np.bincount(np.concatenate([s, d]))))
    nodes = np.array([1, hub, n - 2], np.int32)
    f = P.cfc_farness_jl(h, 32, 6, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    fo = jl.jl_farness(g, 32, 6, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL


@pytest.mark.parametrize("agg", sorted(AGGREGATIONS))
def test_grid_solve_with_each_aggregation(P, agg):
    import torch
    n, s, d, _ = synth.grid2d(90, 70)
    w = synth.uniform_weights(s.size, seed=4)
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(coarse_max=64, **AGGREGATIONS[agg]))
    B = np.random.default_rng(8).standard_normal((n, 24))
    X = torch.empty((n, 24), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(precision=1, levels_used=-1))
    assert info["max_rel_residual"] <= 1e-8
    assert P.lap_hierarchy_info(h)["levels"] >= 4  # coarsening went on to the coarse_max cap
    _certify(canonical_graph(n, s, d, w), B, X.cpu().numpy())


@pytest.mark.parametrize("aggregation", [0, 1])
def test_hub_rule_keeps_a_star_centre_out_of_every_aggregate(P, aggregation):
    # a star without elimination: the centre's only neighbours are leaves, and
    # a leaf's only neighbour is the centre.  With the hub rule the centre
    # stays a singleton and so does every leaf: coarsening stalls at one
    # level.  Without it the pairwise matching merges the star.
    n, s, d, _ = synth.star_graph(3000)
    ho = dict(eliminate=0, coarse_max=16, eager=1, aggregation=aggregation)
    with_rule = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, None, P.lap_default_hier_opts(hub_factor=8, **ho)))
    without = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, None, P.lap_default_hier_opts(**ho)))
    assert with_rule["levels"] == 1
    assert without["levels"] >= 2 and without["level_n"][1] < n // 2


def test_aggregation_options_are_validated(P):
    n, s, d, _ = synth.grid2d(8)
    for bad in (dict(aggregation=2), dict(aggregation=-1), dict(hub_factor=-1), dict(hub_factor=2000000),
                dict(chunking=3), dict(chunking=-1)):
        with pytest.raises(P.LapError):
            P.lap_build_hierarchy(n, s, d, None, P.lap_default_hier_opts(**bad))


# ------------------------------------------------------------------ first residual in two FP32 words
@pytest.mark.parametrize("weights", ["unit", "pow2", "uniform"])
def test_first_residual_in_two_fp32_words(P, weights):
    # with weights that FP32 holds exactly (unit, or powers of two over 8
    # octaves) the first refinement step's residual is formed in two FP32
    # words; the result is still certified by the FP64 residual, matches the
    # oracle's farness, and takes as many steps as with every residual in
    # FP64.  Other weights take the FP64 residual throughout.
    import torch
    n, s, d, _ = synth.rmat(14, seed=3)
    rng = np.random.default_rng(12)
    w = {"unit": None, "pow2": 2.0 ** rng.integers(-4, 5, s.size).astype(np.float64),
         "uniform": synth.uniform_weights(s.size, seed=5)}[weights]
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    B = rng.standard_normal((n, 40))
    X = torch.empty((n, 40), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(precision=1))
    assert info["first_residual_ff"] == (0 if weights == "uniform" else 1)
    assert info["outer_iters"] >= 2 and info["max_rel_residual"] <= 1e-8
    _certify(g, B, X.cpu().numpy())
    X64 = torch.empty_like(X)
    ref = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X64,
                            P.lap_default_solve_opts(precision=1, first_residual_ff=0))
    assert ref["first_residual_ff"] == 0 and ref["outer_iters"] == info["outer_iters"]
    np.testing.assert_allclose(X.cpu().numpy(), X64.cpu().numpy(), rtol=0, atol=1e-6 * np.abs(X64.cpu().numpy()).max())
    nodes = np.array([2, n // 2], np.int32)
    f = P.cfc_farness_jl(h, 32, 4, nodes)
    fo = jl.jl_farness(g, 32, 4, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL
    # FP64 mode never takes it
    info64 = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(precision=0))
    assert info64["first_residual_ff"] == 0


# ------------------------------------------------------------------ long-row chunking modes
@pytest.mark.parametrize("chunking", [1, 2])
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32_all_levels", "bf16coarse"])
def test_rmat_with_each_chunking(P, rmat14, chunking, precision):
    # 1: rows longer than 32 in chunks of 16 (small levels); 2: rows longer
    # than 128 in chunks of 128 (large levels, R-MAT 24's fine level): the
    # SpMV, the residuals and the elimination's pull lists take them
    import torch
    n, s, d, w, g = rmat14
    assert np.bincount(np.concatenate([s, d])).max() > 2 * 128  # hubs span several long chunks
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(chunking=chunking))
    B = np.random.default_rng(4).standard_normal((n, 24))
    X = torch.empty((n, 24), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(**PRECISIONS[precision]))
    assert info["max_rel_residual"] <= 1e-8
    _certify(g, B, X.cpu().numpy())
    nodes = np.array([0, n - 1], np.int32)
    f = P.cfc_farness_jl(h, 32, 9, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    fo = jl.jl_farness(g, 32, 9, nodes.tolist(), solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL



def test_first_residual_in_two_fp32_words_without_elimination(P):
    # a unit-weight grid has no node with fewer than two neighbours: no
    # elimination level, so the first correction lives at the PCG level itself
    import torch
    n, s, d, _ = synth.grid2d(40, 30)
    g = canonical_graph(n, s, d, None)
    h = P.lap_build_hierarchy(n, s, d, None)
    assert P.lap_hierarchy_info(h)["elim_levels"] == 0
    B = np.random.default_rng(21).standard_normal((n, 24))
    X = torch.empty((n, 24), dtype=torch.float64, device="cuda")
    info = P.lap_solve_multi(h, torch.tensor(B, device="cuda"), X, P.lap_default_solve_opts(precision=1))
    assert info["first_residual_ff"] == 1
    assert info["outer_iters"] >= 2 and info["max_rel_residual"] <= 1e-8
    _certify(g, B, X.cpu().numpy())
