"""Shape checks for the seeded input generators (no method arithmetic)."""
import numpy as np

import synth


def test_grid_counts():
    n, s, d, w = synth.grid2d(48)
    assert n == 2304 and s.size == 4512 and w is None
    assert np.all(s < d)


def test_ba_counts_and_determinism():
    n, s, d, _ = synth.barabasi_albert(3000, 5, seed=2)
    assert s.size == 15 + 5 * (3000 - 6)
    key = np.minimum(s, d).astype(np.int64) * n + np.maximum(s, d)
    assert np.unique(key).size == key.size  # simple graph
    n2, s2, d2, _ = synth.barabasi_albert(3000, 5, seed=2)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


def test_rmat_lcc():
    n, s, d, _ = synth.rmat(12, seed=3)
    assert n <= 4096 and np.all(s < d)
    import scipy.sparse as sp
    import scipy.sparse.csgraph as cg
    a = sp.coo_matrix((np.ones(s.size), (s, d)), shape=(n, n))
    assert cg.connected_components(a, directed=False)[0] == 1


def test_rmat_stream_does_not_depend_on_the_process_count(monkeypatch):
    # chunks of samples each draw from their own seeded stream, so a spawned
    # pool of any size yields the same graph as a serial run (small chunks
    # here, so that scale 15 has 16 of them)
    import synth.graphs as G
    monkeypatch.setattr(G, "_RMAT_CHUNK", 1 << 14)
    a = synth.rmat(15, seed=7, processes=1)
    b = synth.rmat(15, seed=7, processes=3)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    c = synth.rmat(15, seed=8, processes=1)
    assert not (c[0] == a[0] and np.array_equal(c[1], a[1]))
    key = a[1].astype(np.int64) * a[0] + a[2]
    assert np.all(np.diff(key) > 0)  # sorted, no duplicate pairs


def test_torus_and_random_regular_have_equal_sizes_and_degrees():
    n1, s1, d1, _ = synth.torus2d(32)
    n2, s2, d2, _ = synth.random_regular(1024, 4, seed=7)
    assert n1 == n2 == 1024 and s1.size == s2.size == 2048
    for n, s, d in ((n1, s1, d1), (n2, s2, d2)):
        deg = np.bincount(np.concatenate([s, d]), minlength=n)
        assert np.all(deg == 4)
        key = np.minimum(s, d).astype(np.int64) * n + np.maximum(s, d)
        assert np.unique(key).size == key.size and np.all(s != d)  # simple
