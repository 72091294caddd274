"""Pins for the CG oracle, the JL estimator (Algorithm 1) and the sampling
estimator (Sec. 5.1, Proposition 1), against the dense oracle, brute force
and exact expectations."""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import dense, jl, sampling
from oracle.cg import cg_solve
from oracle.graph import canonical_graph, incidence, laplacian


def _weighted(gen, seed=7):
    n, s, d, _ = gen
    return canonical_graph(n, s, d, synth.uniform_weights(s.size, seed=seed))


# ---------------------------------------------------------------- CG

@pytest.mark.parametrize("gen,jac", [
    (lambda: synth.grid2d(48), False),
    (lambda: synth.grid2d(48), True),
    (lambda: synth.barabasi_albert(2000, 5, seed=2), True),
    (lambda: synth.barabasi_albert(2000, 5, seed=2), False),
])
def test_cg_matches_dense_pinv(gen, jac):
    g = _weighted(gen())
    rng = np.random.default_rng(1)
    B = rng.standard_normal((g.n, 5))
    X, it, rel = cg_solve(laplacian(g), B, tol=1e-13, jacobi=jac)
    Xd = dense.pinv(g) @ (B - B.mean(axis=0))
    assert np.all(rel <= 1e-12)
    np.testing.assert_allclose(X, Xd, rtol=0, atol=1e-10 * np.abs(Xd).max())
    np.testing.assert_allclose(X.mean(axis=0), 0, atol=1e-12)


def test_cg_projects_rhs_and_handles_zero_column():
    g = _weighted(synth.grid2d(6, 5))
    B = np.ones((g.n, 3))
    B[0, 1] += 1.0
    X, _, rel = cg_solve(laplacian(g), B, tol=1e-12)
    np.testing.assert_allclose(X[:, 0], 0)  # 1 is the null space: projected to 0
    np.testing.assert_allclose(X[:, 2], 0)
    assert rel[1] <= 1e-12


# ---------------------------------------------------------------- JL

def _y_brute(g, Q):
    """Y = Q W^{1/2} B by an explicit loop over edges and rows."""
    k = Q.shape[0]
    Y = np.zeros((k, g.n))
    for e in range(g.m):
        a, b, w = int(g.u[e]), int(g.v[e]), float(g.w[e])
        for i in range(k):
            Y[i, a] += Q[i, e] * math.sqrt(w)
            Y[i, b] -= Q[i, e] * math.sqrt(w)
    return Y


def test_jl_rhs_matches_brute_force_and_sums_to_zero():
    g = _weighted(synth.erdos_renyi_connected(25, 0.2, seed=4))
    k = 300  # spans two 256-row Philox blocks
    Q = jl.projection_matrix(g, k, seed=99)
    np.testing.assert_allclose(np.abs(Q), 1.0 / math.sqrt(k), rtol=1e-15)
    Y = jl.jl_rhs(g, k, seed=99, chunk=7)
    np.testing.assert_allclose(Y, _y_brute(g, Q), atol=1e-13)
    np.testing.assert_allclose(Y.sum(axis=1), 0, atol=1e-12)  # B 1 = 0


@pytest.mark.parametrize("k", [5, 64, 300])
def test_jl_rhs_at_nodes_matches_brute_force(k):
    # the node-restricted right-hand side against the brute-force edge loop
    # over the explicit Q (a hub, a leaf of the star and an arbitrary node)
    g = _weighted(synth.barabasi_albert(60, 3, seed=5))
    Q = jl.projection_matrix(g, k, seed=13)
    nodes = [0, 17, g.n - 1]
    np.testing.assert_allclose(jl.jl_rhs_at(g, k, 13, nodes), _y_brute(g, Q)[:, nodes], atol=1e-13)
    gs = _weighted(synth.star_graph(12))
    np.testing.assert_allclose(jl.jl_rhs_at(gs, k, 2, [0, 5]), _y_brute(gs, jl.projection_matrix(gs, k, 2))[:, [0, 5]],
                               atol=1e-13)


def test_identity_projection_gives_exact_resistance():
    # with Q = I_m (no projection) Algorithm 1 returns d_ER exactly:
    # d_ER(u,v) = ||W^{1/2} B L^+ (e_u - e_v)||^2 (Sec. 5.2)
    g = _weighted(synth.barabasi_albert(40, 3, seed=6))
    Y = (incidence(g).T.multiply(np.sqrt(g.w)[None, :])).T.toarray()  # W^{1/2} B, m x n
    Z = jl.jl_solve(g, Y, "dense")
    R = dense.resistance_matrix(g)
    for u, v in [(0, 1), (3, 39), (10, 22)]:
        assert jl.pair_distance(Z, u, v) == pytest.approx(R[u, v], rel=1e-10)


def test_jl_cg_matches_dense_for_fixed_q():
    g = _weighted(synth.grid2d(20, 15))
    fd = jl.jl_farness(g, 32, seed=1, nodes=[0, 77], solver="dense")
    fc = jl.jl_farness(g, 32, seed=1, nodes=[0, 77], solver="cg", tol=1e-13)
    np.testing.assert_allclose(fc, fd, rtol=1e-9)


def test_jl_farness_single_node_identity():
    # sum_w ||Z_v - Z_w||^2 = sum_i [n Z_iv^2 - 2 Z_iv S_i + T_i], S_i = sum_w Z_iw,
    # T_i = sum_w Z_iw^2: the O(kn) form the GPU reduction uses
    g = _weighted(synth.barabasi_albert(150, 4, seed=3))
    f, Z = jl.jl_farness(g, 24, seed=5, nodes=[0, 9, 149], return_Z=True)
    S = Z.sum(axis=1)
    T = (Z * Z).sum(axis=1)
    for t, v in enumerate([0, 9, 149]):
        alt = np.sum(g.n * Z[:, v] ** 2 - 2 * Z[:, v] * S + T)
        assert alt == pytest.approx(f[t], rel=1e-12)


def test_jl_unbiased_over_seeds():
    # E[Q^T Q] = I for iid +-1/sqrt(k) entries, so E[d~(u,v)] = d_ER(u,v)
    g = _weighted(synth.erdos_renyi_connected(30, 0.15, seed=2))
    R = dense.resistance_matrix(g)
    P = dense.pinv(g)
    k, trials = 8, 600
    acc = np.zeros((g.n, g.n))
    sq = np.zeros((g.n, g.n))
    for s in range(trials):
        Z = (P @ jl.jl_rhs(g, k, seed=1000 + s).T).T
        G = Z.T @ Z
        dg = np.diag(G)
        D = dg[:, None] + dg[None, :] - 2 * G
        acc += D
        sq += D * D
    mean = acc / trials
    sd = np.sqrt(np.maximum(sq / trials - mean ** 2, 0) / trials)
    iu = np.triu_indices(g.n, 1)
    z = (mean[iu] - R[iu]) / np.maximum(sd[iu], 1e-15)
    assert np.abs(z).max() < 5.0
    assert abs(np.mean(z)) < 0.2


def test_jl_bound_frequency():
    # k = ceil(ln n / eps^2) (Sec. 6.4).  The O(log n / eps^2) bound of Sec. 5.2
    # has no stated constant, so the per-pair check is a frequency; the
    # farness of every node lies within (1 +- eps), as Sec. 6.4 reports for
    # the closeness of every tested node.
    g = _weighted(synth.barabasi_albert(400, 4, seed=8))
    eps = 0.3
    k = jl.k_from_eps(g.n, eps)
    assert k == math.ceil(math.log(400) / 0.09)
    R = dense.resistance_matrix(g)
    Z = jl.jl_solve(g, jl.jl_rhs(g, k, seed=3), "dense")
    G = Z.T @ Z
    dg = np.diag(G)
    D = dg[:, None] + dg[None, :] - 2 * G
    iu = np.triu_indices(g.n, 1)
    ratio = D[iu] / R[iu]
    assert np.mean(np.abs(ratio - 1) <= eps) > 0.9
    f = D.sum(axis=1)
    assert np.all(np.abs(f / dense.farness(g, R) - 1) <= eps)


# ---------------------------------------------------------------- sampling

def test_floyd_pivots_valid_and_uniform():
    n, k = 9, 3
    counts = np.zeros(n)
    for seed in range(3000):
        S = sampling.floyd_pivots(n, k, seed)
        assert S.size == k and len(set(S.tolist())) == k
        assert S.min() >= 0 and S.max() < n and np.all(np.diff(S) > 0)
        counts[S] += 1
    expected = 3000 * k / n
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 30.0  # 8 dof; p ~ 2e-4
    assert np.array_equal(sampling.floyd_pivots(50, 50, 1), np.arange(50))


def test_pair_solves_match_resistance():
    g = _weighted(synth.grid2d(7, 6))
    R = dense.resistance_matrix(g)
    piv = [0, 5, 20, 41, 13]
    np.testing.assert_allclose(sampling.pair_resistance_solves(g, 13, piv), R[13, piv], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(sampling.pair_resistance_solves(g, 13, piv, solver="cg"), R[13, piv],
                               rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("n,k", [(7, 1), (8, 2), (9, 3), (10, 4)])
def test_proposition1_exhaustive(n, k):
    # mean over all k-combinations S of V of (n/k) sum_{s in S} d_ER(v, s)
    # equals the exact electrical farness (Proposition 1)
    g = _weighted(synth.erdos_renyi_connected(n, 0.4, seed=n))
    R = dense.resistance_matrix(g)
    f = dense.farness(g, R)
    for v in range(n):
        vals = [n / k * sum(R[v, s] for s in S) for S in itertools.combinations(range(n), k)]
        assert np.mean(vals) == pytest.approx(f[v], rel=1e-12)
    # the estimator itself, with given pivots, is that summand
    S = (1, 4, 6)[: k] if k <= 3 else (0, 2, 5, 6)
    est = sampling.sampled_farness(g, k, 0, [3], pivots=np.array(S))
    assert est[0] == pytest.approx(n / k * sum(R[3, s] for s in S), rel=1e-10)


def test_sampling_all_pivots_is_exact():
    g = _weighted(synth.barabasi_albert(60, 3, seed=9))
    f = dense.farness(g)
    est = sampling.sampled_farness(g, g.n, seed=4, nodes=[0, 30, 59])
    np.testing.assert_allclose(est, f[[0, 30, 59]], rtol=1e-10)
