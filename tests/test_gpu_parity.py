"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Tolerances: the solver stops at a per-column relative residual of 1e-8
(FP64 outer residual); farness estimates must match the oracle to relative
error <= 1e-6 in the FP64-refined modes, the dense exact path to 1e-9,
integer outputs (pivots) bit for bit.
"""
import numpy as np
import pytest

import synth
from oracle import cg as ocg
from oracle import dense, jl, sampling
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


def _graph(gen, weighted=True, seed=7):
    n, s, d, _ = gen
    w = synth.uniform_weights(s.size, seed=seed) if weighted else None
    return n, s, d, w


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(np.asarray(b)), 1e-300))


# ------------------------------------------------------------------ ingest / hierarchy
def test_hierarchy_sizes(P):
    n, s, d, w = _graph(synth.grid2d(48))
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1, coarse_max=64))
    info = P.lap_hierarchy_info(h)
    assert info["n"] == 2304 and info["m"] == 4512
    assert info["level_nnz"][0] == 2 * 4512
    assert info["levels"] >= 3
    assert info["coarse_n"] == info["level_n"][-1] <= 64
    for a, b in zip(info["level_n"], info["level_n"][1:]):
        assert b < a
    # the default (automatic coarse_max: 256 up to 1M nodes) stops at 256 nodes
    # or fewer on this graph and solves that level densely; 2048 is the cap
    dflt = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1)))
    assert dflt["coarse_n"] == dflt["level_n"][-1] <= 256 < dflt["level_n"][-2]
    big = P.lap_hierarchy_info(P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1, coarse_max=5000)))
    assert big["levels"] == 2 and big["coarse_n"] == big["level_n"][-1] <= 2048
    with pytest.raises(P.LapError):
        P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(coarse_max=-1))


def test_duplicates_selfloops_merged(P):
    # parallel edges add, self-loops vanish, orientation is ignored
    src = np.array([0, 1, 1, 2, 2, 3, 0], np.int32)
    dst = np.array([1, 0, 2, 2, 3, 0, 1], np.int32)
    w = np.array([1.0, 2.0, 4.0, 9.0, 1.0, 1.0, 3.0])
    f, c = P.cfc_exact_small(4, src, dst, w)
    g = canonical_graph(4, src, dst, w)
    np.testing.assert_allclose(f, dense.farness(g), rtol=1e-12)
    np.testing.assert_allclose(c, dense.closeness(g), rtol=1e-12)


@pytest.mark.parametrize("bad", ["disconnected", "range", "weight", "nan"])
def test_input_errors(P, bad):
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 3], np.int32)
    w = np.ones(3)
    n = 4
    want = P.LAP_EINVAL
    if bad == "disconnected":
        n, want = 6, P.LAP_ENOTCONN
    elif bad == "range":
        dst = np.array([1, 2, 4], np.int32)
    elif bad == "weight":
        w = np.array([1.0, 0.0, 1.0])
    else:
        w = np.array([1.0, np.nan, 1.0])
    with pytest.raises(P.LapError) as e:
        P.lap_build_hierarchy(n, src, dst, w)
    assert e.value.status == want


# ------------------------------------------------------------------ JL right-hand sides
@pytest.mark.parametrize("k", [32, 5, 300])
def test_jl_rhs_matches_oracle(P, k):
    import torch
    n, s, d, w = _graph(synth.barabasi_albert(1500, 5, seed=3))  # hubs: split rows
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    Y = torch.empty((n, k), dtype=torch.float64, device="cuda")
    P.cfc_jl_rhs(h, k, 11, Y)
    Yo = jl.jl_rhs(g, k, 11).T
    np.testing.assert_allclose(Y.cpu().numpy(), Yo, rtol=0, atol=1e-13 * np.abs(Yo).max())


# ------------------------------------------------------------------ solver
SOLVE_CASES = [
    ("grid48", lambda: synth.grid2d(48), 32),
    ("ba3000", lambda: synth.barabasi_albert(3000, 5, seed=2), 17),
    ("star", lambda: synth.star_graph(700), 8),
    ("path", lambda: synth.path_graph(400), 16),
    ("er", lambda: synth.erdos_renyi_connected(500, 0.02, seed=5), 70),
]


PRECISIONS = {"fp32": dict(precision=1), "fp64": dict(precision=0),
              # BF16 coarse weights only matter below the finest level: use every level
              "bf16coarse": dict(precision=2, levels_used=-1)}


@pytest.mark.parametrize("name,gen,k", SOLVE_CASES)
@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_solve_matches_dense_pinv(P, name, gen, k, precision):
    import torch
    n, s, d, w = _graph(gen())
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    rng = np.random.default_rng(1)
    B = rng.standard_normal((n, k))
    Bt = torch.tensor(B, device="cuda")
    Xt = torch.empty_like(Bt)
    opts = P.lap_default_solve_opts(**PRECISIONS[precision])
    info = P.lap_solve_multi(h, Bt, Xt, opts)
    assert info["max_rel_residual"] <= 1e-8
    X = Xt.cpu().numpy()
    Bp = B - B.mean(axis=0)
    # independent residual check in FP64 on the CPU
    R = Bp - laplacian(g) @ X
    assert np.all(np.linalg.norm(R, axis=0) <= 1.01e-8 * np.linalg.norm(Bp, axis=0))
    np.testing.assert_allclose(X.mean(axis=0), 0, atol=1e-12 * np.abs(X).max())
    Xd = dense.pinv(g) @ Bp
    err = np.linalg.norm(X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
    # ||x - x*|| / ||x*|| <= kappa * ||r|| / ||b||, kappa = lambda_max / lambda_2 on 1-perp
    lam = np.linalg.eigvalsh(laplacian(g).toarray())
    kappa = lam[-1] / lam[1]
    assert err.max() <= kappa * 1.01e-8, (err.max(), kappa)


def test_solve_is_deterministic_and_column_independent(P):
    import torch
    n, s, d, w = _graph(synth.barabasi_albert(4000, 5, seed=9))
    h = P.lap_build_hierarchy(n, s, d, w)
    B = torch.randn((n, 48), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    X1, X2 = torch.empty_like(B), torch.empty_like(B)
    o = P.lap_default_solve_opts(k_tile=16, levels_used=-1)
    P.lap_solve_multi(h, B, X1, o)
    P.lap_solve_multi(h, B, X2, o)
    assert torch.equal(X1, X2)
    # the first 16 columns alone give the same bits (same tile width)
    Xs = torch.empty((n, 16), dtype=torch.float64, device="cuda")
    P.lap_solve_multi(h, B[:, :16].contiguous(), Xs, o)
    assert torch.equal(Xs, X1[:, :16])


def test_lazy_levels_and_depth_choices(P):
    import torch
    n, s, d, w = _graph(synth.grid2d(64))
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(coarse_max=64))
    assert P.lap_hierarchy_info(h)["levels"] == 1  # coarse levels are built on demand
    B = torch.randn((n, 16), dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    P.lap_solve_multi(h, B, X, P.lap_default_solve_opts(levels_used=2))
    assert P.lap_hierarchy_info(h)["levels"] == 2
    ref = None
    for lv in (1, 3, -1, 0):
        info = P.lap_solve_multi(h, B, X, P.lap_default_solve_opts(levels_used=lv))
        assert info["max_rel_residual"] <= 1e-8
        if ref is None:
            ref = X.clone()
        else:
            err = (X - ref).norm(dim=0) / ref.norm(dim=0)
            assert float(err.max()) <= 1e-5
    assert P.lap_hierarchy_info(h)["levels"] >= 4


def test_solve_noconv_reports(P):
    import torch
    n, s, d, w = _graph(synth.grid2d(40))
    h = P.lap_build_hierarchy(n, s, d, w)
    B = torch.randn((n, 4), dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    o = P.lap_default_solve_opts(max_outer=1, max_inner=2, inner_tol=1e-2)
    info = P.lap_solve_multi(h, B, X, o, allow_noconv=True)
    assert info["status"] == P.LAP_ENOCONV and info["max_rel_residual"] > 1e-8
    assert torch.isfinite(X).all()


# ------------------------------------------------------------------ estimators
@pytest.mark.parametrize("gen,k", [(lambda: synth.grid2d(48), 32), (lambda: synth.barabasi_albert(2000, 5, 4), 64),
                                   (lambda: synth.star_graph(300), 24)])
@pytest.mark.parametrize("precision", sorted(PRECISIONS))
def test_farness_jl_matches_oracle(P, gen, k, precision):
    n, s, d, w = _graph(gen())
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    nodes = np.array([0, 1, n // 2, n - 1], np.int32)
    f = P.cfc_farness_jl(h, k, 1, nodes, opts=P.lap_default_solve_opts(**PRECISIONS[precision]))
    fo = jl.jl_farness(g, k, 1, nodes.tolist(), solver="dense")
    assert _rel(f, fo) <= FARNESS_RTOL


@pytest.mark.parametrize("k,world", [(64, 2), (100, 3), (40, 4)])
def test_farness_jl_row_shards_sum_to_the_full_query(P, k, world):
    from paper_1607_02955_gb300.sharding import shard_rows
    n, s, d, w = _graph(synth.barabasi_albert(2500, 5, seed=8))
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    nodes = np.array([0, 5, n - 1], np.int32)
    full = P.cfc_farness_jl(h, k, 3, nodes)
    Z = jl.jl_solve(g, jl.jl_rhs(g, k, 3))  # k x n, oracle
    total = np.zeros(len(nodes))
    for r in range(world):
        r0, c = shard_rows(k, world, r)
        if c == 0:
            continue
        part = P.cfc_farness_jl_rows(h, k, r0, c, 3, nodes)
        rows = Z[r0:r0 + c]
        want = np.array([((rows - rows[:, [v]]) ** 2).sum() for v in nodes])
        assert _rel(part, want) <= FARNESS_RTOL
        total += part
    # separate solves stop at different iterations (all columns of a block
    # iterate until the slowest converges): equal to the solve tolerance
    assert _rel(total, full) <= FARNESS_RTOL
    with pytest.raises(P.LapError):  # shards start on a multiple of 32 rows
        P.cfc_farness_jl_rows(h, k, 16, 8, 3, nodes)


@pytest.mark.parametrize("cycle,w_levels", [(1, 0), (2, 0), (2, 1)])
def test_graph_replay_matches_plain_launches(P, cycle, w_levels):
    # the captured cycle is the same kernels in the same order: identical bits
    import torch
    n, s, d, w = _graph(synth.grid2d(64))
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1, coarse_max=64))
    assert P.lap_hierarchy_info(h)["levels"] >= 3
    rng = np.random.default_rng(4)
    B = torch.tensor(rng.standard_normal((n, 24)), device="cuda")
    out = []
    for graphs in (1, 0):
        X = torch.empty_like(B)
        o = P.lap_default_solve_opts(levels_used=-1, cycle=cycle, w_levels=w_levels, coarse_scale=1.5,
                                     k_tile=32, graphs=graphs)
        info = P.lap_solve_multi(h, B, X, o)
        assert info["max_rel_residual"] <= 1e-8
        out.append(X.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_bf16_coarse_changes_only_the_preconditioner(P):
    # same FP64 stopping test: both modes reach 1e-8 and agree to the solve
    # tolerance; the coarse operators differ, so the inner iterations may differ
    import torch
    n, s, d, w = _graph(synth.grid2d(64))
    h = P.lap_build_hierarchy(n, s, d, w, P.lap_default_hier_opts(eager=1, coarse_max=64))
    assert P.lap_hierarchy_info(h)["levels"] >= 3
    rng = np.random.default_rng(3)
    B = torch.tensor(rng.standard_normal((n, 16)), device="cuda")
    X1, X2 = torch.empty_like(B), torch.empty_like(B)
    i1 = P.lap_solve_multi(h, B, X1, P.lap_default_solve_opts(precision=1, levels_used=-1))
    i2 = P.lap_solve_multi(h, B, X2, P.lap_default_solve_opts(precision=2, levels_used=-1))
    assert i1["max_rel_residual"] <= 1e-8 and i2["max_rel_residual"] <= 1e-8
    g = canonical_graph(n, s, d, w)
    lam = np.linalg.eigvalsh(laplacian(g).toarray())
    diff = (X1 - X2).norm(dim=0) / X1.norm(dim=0)
    assert float(diff.max()) <= 2 * lam[-1] / lam[1] * 1.01e-8


def test_farness_jl_all_nodes(P):
    # the estimator for every node at once (q = n): one solve block, O(nk) sums
    n, s, d, w = _graph(synth.grid2d(48))
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    nodes = np.arange(n, dtype=np.int32)
    f = P.cfc_farness_jl(h, 32, 1, nodes)
    fo = jl.jl_farness(g, 32, 1, nodes.tolist(), solver="dense")
    assert _rel(f, fo) <= FARNESS_RTOL


@pytest.mark.parametrize("n,k", [(3000, 64), (517, 5), (2, 1), (1000, 300)])
def test_farness_from_solution_matches_literal_sum(P, n, k):
    import torch
    rng = np.random.default_rng(n + k)
    Z = rng.standard_normal((n, k))
    nodes = np.unique(rng.integers(0, n, size=min(n, 9))).astype(np.int32)
    f = P.cfc_farness_from_solution(torch.tensor(Z, device="cuda"), nodes)
    # literal sum over w of ||Z_v - Z_w||^2 (Algorithm 1, step 4)
    fo = np.array([((Z - Z[v]) ** 2).sum() for v in nodes])
    assert _rel(f, fo) <= 1e-12


def test_farness_jl_eps_rule(P):
    n, s, d, w = _graph(synth.grid2d(20))
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    f = P.cfc_farness_jl(h, 0, 3, [5], eps=0.5)
    k = jl.k_from_eps(n, 0.5)
    assert _rel(f, jl.jl_farness(g, k, 3, [5])) <= FARNESS_RTOL


@pytest.mark.parametrize("n,kk,seed", [(2304, 200, 1), (100, 100, 2), (5000, 7, 3), (64, 1, 4)])
def test_pivots_bit_exact(P, n, kk, seed):
    ns, s, d, w = _graph(synth.path_graph(n))
    h = P.lap_build_hierarchy(ns, s, d, w)
    piv = P.cfc_sample_pivots(h, kk, seed)
    assert np.array_equal(piv, sampling.floyd_pivots(n, kk, seed))


@pytest.mark.parametrize("gen,kk", [(lambda: synth.grid2d(30), 20), (lambda: synth.barabasi_albert(1200, 5, 6), 50)])
def test_farness_sampled_matches_pair_solves(P, gen, kk):
    n, s, d, w = _graph(gen())
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    nodes = np.array([3, n - 2, 17], np.int32)
    f = P.cfc_farness_sampled(h, kk, 9, nodes)
    fo = sampling.sampled_farness(g, kk, 9, nodes.tolist(), solver="dense")
    assert _rel(f, fo) <= FARNESS_RTOL


def test_farness_sampled_all_pivots_is_exact(P):
    n, s, d, w = _graph(synth.barabasi_albert(90, 3, seed=1))
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    f = P.cfc_farness_sampled(h, n, 5, [0, 45, 89])
    assert _rel(f, dense.farness(g)[[0, 45, 89]]) <= FARNESS_RTOL


@pytest.mark.parametrize("gen", [lambda: synth.grid2d(48), lambda: synth.barabasi_albert(1000, 5, 2),
                                 lambda: synth.complete_graph(30), lambda: synth.path_graph(2)])
def test_exact_small_matches_dense_oracle(P, gen):
    n, s, d, w = _graph(gen())
    g = canonical_graph(n, s, d, w)
    f, c = P.cfc_exact_small(n, s, d, w)
    fo = dense.farness(g)
    assert _rel(f, fo) <= 1e-9
    assert _rel(c, dense.closeness(g, fo)) <= 1e-9


def test_exact_small_cross_checked_by_cg_solves(P):
    # exact farness (dense L+) against n CG solves with b = e_v - 1/n (Sec. 4 exact methods)
    n, s, d, w = _graph(synth.grid2d(12, 10))
    g = canonical_graph(n, s, d, w)
    f, _ = P.cfc_exact_small(n, s, d, w)
    X, _, _ = ocg.cg_solve(laplacian(g), np.eye(n), tol=1e-13)
    fo = n * np.diag(X) + np.trace(X)
    assert _rel(f, fo) <= 1e-8


# ------------------------------------------------------------------ full-size sampled parity
@pytest.mark.slow
def test_ba100k_jl_node0_matches_oracle(P):
    """The 100k-node Barabasi-Albert configuration with k = 64 in the
    benchmark's launch configuration (default options): farness of node 0
    against the oracle's FP64 CG (1e-12) on the same right-hand sides."""
    n, s, d, _ = synth.barabasi_albert(100000, 5, seed=2)
    w = synth.uniform_weights(s.size, seed=2)
    g = canonical_graph(n, s, d, w)
    h = P.lap_build_hierarchy(n, s, d, w)
    f = P.cfc_farness_jl(h, 64, 1, [0])
    fo = jl.jl_farness(g, 64, 1, [0], solver="cg", tol=1e-12)
    assert _rel(f, fo) <= FARNESS_RTOL
