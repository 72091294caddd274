"""Pins for the dense oracle (L^+, d_ER, farness, closeness) against closed
forms and identities fixed by the mathematics (Sec. 2, Sec. 4)."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import dense
from oracle.graph import NotConnected, canonical_graph, degrees, laplacian_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _g(gen):
    n, s, d, w = gen
    return canonical_graph(n, s, d, w)


def test_golden_closed_forms():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        e = np.array(c["edges"])
        g = canonical_graph(c["n"], e[:, 0].astype(int), e[:, 1].astype(int), e[:, 2])
        R = dense.resistance_matrix(g)
        for u, v, r in c["pairs"]:
            assert R[int(u), int(v)] == pytest.approx(r, rel=1e-12), c["name"]
        if "farness" in c:
            np.testing.assert_allclose(dense.farness(g, R), c["farness"], rtol=1e-12)


def test_tree_resistance_is_path_length():
    # random weighted tree: R(u, v) = sum of 1/w along the unique path
    n, s, d, _ = synth.random_tree(40, seed=11)
    w = synth.uniform_weights(n - 1, seed=12)
    g = canonical_graph(n, s, d, w)
    R = dense.resistance_matrix(g)
    par = {int(b): (int(a), float(x)) for a, b, x in zip(s, d, w)}  # parent of b is a

    def up(v):
        path = {v: 0.0}
        acc = 0.0
        while v in par:
            a, x = par[v]
            acc += 1.0 / x
            v = a
            path[v] = acc
        return path

    for u in range(0, n, 3):
        pu = up(u)
        for v in range(1, n, 4):
            pv = up(v)
            lca_cost = min(pu[a] + pv[a] for a in pu if a in pv)
            assert R[u, v] == pytest.approx(lca_cost, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("n", [3, 7, 20])
def test_complete_graph(n):
    g = _g(synth.complete_graph(n))
    R = dense.resistance_matrix(g)
    off = R[~np.eye(n, dtype=bool)]
    np.testing.assert_allclose(off, 2.0 / n, rtol=1e-12)
    f = dense.farness(g, R)
    np.testing.assert_allclose(f, 2.0 * (n - 1) / n, rtol=1e-12)
    np.testing.assert_allclose(dense.closeness(g, f), n / 2.0, rtol=1e-12)


@pytest.mark.parametrize("n", [5, 12, 31])
def test_cycle(n):
    g = _g(synth.cycle_graph(n))
    R = dense.resistance_matrix(g)
    for u in range(n):
        for v in range(n):
            d = abs(u - v)
            d = min(d, n - d)
            assert R[u, v] == pytest.approx(d * (n - d) / n, abs=1e-12)


@pytest.mark.parametrize("gen", [
    lambda: synth.barabasi_albert(300, 3, seed=5),
    lambda: synth.grid2d(9, 13),
    lambda: synth.erdos_renyi_connected(60, 0.1, seed=3),
])
def test_foster_symmetry_triangle(gen):
    n, s, d, _ = gen()
    w = synth.uniform_weights(s.size, seed=9)
    g = canonical_graph(n, s, d, w)
    R = dense.resistance_matrix(g)
    # Foster's theorem: sum_e w_e R_e = n - 1
    assert float(np.sum(g.w * R[g.u, g.v])) == pytest.approx(n - 1, rel=1e-10)
    np.testing.assert_allclose(R, R.T, atol=1e-12)
    assert R.min() >= -1e-12
    # triangle inequality on a sample of triples
    rng = np.random.default_rng(0)
    a, b, c = rng.integers(0, n, size=(3, 2000))
    assert np.all(R[a, c] <= R[a, b] + R[b, c] + 1e-10)
    # every R_e <= 1/w_e (Rayleigh monotonicity: the edge itself is a path)
    assert np.all(R[g.u, g.v] <= 1.0 / g.w + 1e-12)


def test_grounded_inverse_equals_pseudoinverse_form():
    # Sec. 4 grounded inverse vs the L^+ = (L + J/n)^-1 - J/n route
    n, s, d, _ = synth.barabasi_albert(120, 4, seed=1)
    w = synth.uniform_weights(s.size, seed=4)
    g = canonical_graph(n, s, d, w)
    np.testing.assert_allclose(dense.grounded_resistance(g, ground=17), dense.resistance_matrix(g),
                               rtol=1e-9, atol=1e-12)


def test_pinv_properties():
    n, s, d, _ = synth.erdos_renyi_connected(50, 0.15, seed=8)
    g = canonical_graph(n, s, d, synth.uniform_weights(s.size, seed=2))
    L = laplacian_dense(g)
    P = dense.pinv(g)
    np.testing.assert_allclose(L @ P @ L, L, atol=1e-10)
    np.testing.assert_allclose(P @ L @ P, P, atol=1e-10)
    np.testing.assert_allclose(P @ np.ones(n), 0, atol=1e-10)
    np.testing.assert_allclose(L @ P, np.eye(n) - 1.0 / n, atol=1e-10)


def _grid_pinv_dct(a, b):
    """L^+ of the unit a x b grid from its separable eigenbasis:
    eigenvectors phi_i(r) phi_j(c) with phi_i(r) = cos(pi i (r + 1/2) / a)
    (normalised) and eigenvalues 2 - 2cos(pi i/a) + 2 - 2cos(pi j/b)."""
    def basis(a):
        r = np.arange(a) + 0.5
        P = np.cos(np.pi * np.outer(np.arange(a), r) / a)  # rows i
        P /= np.linalg.norm(P, axis=1, keepdims=True)
        lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(a) / a)
        return P, lam
    Pa, la = basis(a)
    Pb, lb = basis(b)
    lam = la[:, None] + lb[None, :]
    inv = np.where(lam > 0, 1.0 / np.where(lam > 0, lam, 1), 0.0)
    # L^+ = sum_{ij} inv_ij (phi_i x phi_j)(phi_i x phi_j)^T
    V = np.einsum("ir,jc->ijrc", Pa, Pb).reshape(a * b, a * b)  # row (i,j), col node
    return V.T @ (inv.reshape(-1)[:, None] * V)


def test_grid_pinv_matches_dct_closed_form():
    a, b = 12, 17
    g = _g(synth.grid2d(a, b))
    np.testing.assert_allclose(dense.pinv(g), _grid_pinv_dct(a, b), atol=1e-11)


@pytest.mark.slow
def test_grid_48_closed_form_farness():
    # the 48 x 48 configuration: farness from the DCT closed form
    a = 48
    g = _g(synth.grid2d(a))
    Pd = _grid_pinv_dct(a, a)
    fd = a * a * np.diag(Pd) + np.trace(Pd)
    np.testing.assert_allclose(dense.farness(g), fd, rtol=1e-10)


def test_farness_identity_n_diag_plus_trace():
    # f(v) = sum_w [L+_vv - 2 L+_vw + L+_ww] = n L+_vv + tr L+  (L+ 1 = 0)
    n, s, d, _ = synth.barabasi_albert(200, 5, seed=2)
    g = canonical_graph(n, s, d, synth.uniform_weights(s.size, seed=3))
    P = dense.pinv(g)
    np.testing.assert_allclose(dense.farness(g), n * np.diag(P) + np.trace(P), rtol=1e-10)


def test_input_rules():
    with pytest.raises(NotConnected):
        canonical_graph(4, [0, 2], [1, 3])
    with pytest.raises(ValueError):
        canonical_graph(3, [0], [3])
    with pytest.raises(ValueError):
        canonical_graph(3, [0, 1], [1, 2], [1.0, -1.0])
    with pytest.raises(ValueError):
        canonical_graph(3, [0, 1], [1, 2], [1.0, np.nan])
    g = canonical_graph(3, [2, 1, 0, 1, 1], [1, 0, 1, 1, 2], [1.0, 2.0, 3.0, 9.0, 4.0])
    assert list(g.u) == [0, 1] and list(g.v) == [1, 2]
    np.testing.assert_allclose(g.w, [5.0, 5.0])
    np.testing.assert_allclose(degrees(g), [5.0, 10.0, 5.0])
