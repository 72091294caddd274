"""The request loop (cfc_server_*): continuous batching of sampling-estimator
queries (Sec. 5.1) over resident graphs.

Each request's farness must be the same alone and in a mix of overlapping
requests (bit for bit: the configuration is pinned per graph and every
reduction has a fixed order), and must match the oracle's sampling estimate
to the FP64-refined tolerance (relative error <= 1e-6).
"""
import numpy as np
import pytest

import synth
from oracle import sampling
from oracle.graph import canonical_graph

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


def _graphs():
    out = []
    for gen, seed in [(synth.grid2d(40), 1), (synth.barabasi_albert(3000, 5, seed=4), 2),
                      (synth.erdos_renyi_connected(800, 0.01, seed=6), 3)]:
        n, s, d, _ = gen
        out.append((n, s, d, synth.uniform_weights(s.size, seed=seed)))
    return out


def _queries(graphs, count, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(count):
        gid = int(rng.integers(len(graphs)))
        n = graphs[gid][0]
        q = int(rng.integers(1, 9))
        nodes = rng.choice(n, size=q, replace=False).astype(np.int32)
        qs.append((gid, nodes, int(rng.integers(30, 90)), int(rng.integers(1 << 40))))
    return qs


def test_server_results_same_alone_and_in_mix(P):
    graphs = _graphs()
    sv = P.cfc_server_create(P.cfc_server_default_opts(slots=4))
    try:
        gids = [P.cfc_server_add_graph(sv, n, s, d, w) for n, s, d, w in graphs]
        assert gids == [0, 1, 2]
        qs = _queries(graphs, 16, 5)
        # alone: one request on the device at a time
        alone = []
        for gid, nodes, kk, seed in qs:
            rid = P.cfc_server_submit(sv, gid, nodes, kk, seed)
            f, info = P.cfc_server_poll(sv, rid, -1)
            assert info["status"] == P.LAP_OK and info["q"] == len(nodes)
            alone.append(f)
        P.cfc_server_reset_stats(sv)
        # mix: everything at once, admitted as slots free up
        rids = [P.cfc_server_submit(sv, gid, nodes, kk, seed) for gid, nodes, kk, seed in qs]
        mix = [P.cfc_server_poll(sv, r, -1)[0] for r in rids]
        for a, m in zip(alone, mix):
            assert np.array_equal(a, m)
        st = P.cfc_server_stats(sv)
        assert st["completed"] == len(qs) and st["pending"] == 0 and st["in_flight"] == 0
        assert st["max_in_flight"] >= 2  # requests overlapped on the device
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["rhs_per_s"] > 0
        # against the oracle's sampling estimator on the same pivots
        for (gid, nodes, kk, seed), f in list(zip(qs, alone))[:4]:
            n, s, d, w = graphs[gid]
            fo = sampling.sampled_farness(canonical_graph(n, s, d, w), kk, seed, nodes.tolist(), solver="dense")
            assert np.max(np.abs(f - fo) / np.abs(fo)) <= FARNESS_RTOL
    finally:
        sv.destroy()


def test_server_matches_the_one_shot_call(P):
    n, s, d, w = _graphs()[1]
    sv = P.cfc_server_create(P.cfc_server_default_opts(slots=2))
    try:
        gid = P.cfc_server_add_graph(sv, n, s, d, w)
        nodes = np.array([0, 7, n - 1], np.int32)
        f, _ = P.cfc_server_poll(sv, P.cfc_server_submit(sv, gid, nodes, 64, 77), -1)
        h = P.lap_build_hierarchy(n, s, d, w)
        ref = P.cfc_farness_sampled(h, 64, 77, nodes)
        assert np.max(np.abs(f - ref) / np.abs(ref)) <= FARNESS_RTOL
    finally:
        sv.destroy()


def test_server_budget_and_errors(P):
    n, s, d, w = _graphs()[0]
    tiny = P.cfc_server_create(P.cfc_server_default_opts(slots=1, hbm_budget=1 << 16))
    try:
        with pytest.raises(P.LapError) as e:
            P.cfc_server_add_graph(tiny, n, s, d, w)
        assert e.value.status == P.LAP_EBUDGET
    finally:
        tiny.destroy()
    sv = P.cfc_server_create(P.cfc_server_default_opts(slots=2, hbm_budget=256 << 20))
    try:
        gid = P.cfc_server_add_graph(sv, n, s, d, w)
        for bad, status in [(dict(graph_id=5), P.LAP_EINVAL), (dict(nodes=[n]), P.LAP_EINVAL),
                            (dict(n_pivots=0), P.LAP_EINVAL), (dict(n_pivots=n + 1), P.LAP_EINVAL)]:
            args = dict(graph_id=gid, nodes=[1, 2], n_pivots=20, seed=1)
            args.update(bad)
            with pytest.raises(P.LapError) as e:
                P.cfc_server_submit(sv, args["graph_id"], args["nodes"], args["n_pivots"], args["seed"])
            assert e.value.status == status
        with pytest.raises(P.LapError) as e:
            P.cfc_server_poll(sv, 12345, 0)
        assert e.value.status == P.LAP_EINVAL
        rid = P.cfc_server_submit(sv, gid, [3], 20, 1)
        assert P.cfc_server_poll(sv, rid, -1) is not None
        with pytest.raises(P.LapError):  # a result is handed out once
            P.cfc_server_poll(sv, rid, 0)
    finally:
        sv.destroy()


def test_server_resident_pivot_sets(P):
    # requests with n_pivots = 0 solve only their nodes' columns against the
    # graph's pivot solutions kept on the device: the same estimate as the
    # oracle's with that pivot set, and the same bits alone and in a mix
    graphs = _graphs()
    sv = P.cfc_server_create(P.cfc_server_default_opts(slots=3, resident_pivots=40, pivot_seed=11))
    try:
        gids = [P.cfc_server_add_graph(sv, n, s, d, w) for n, s, d, w in graphs]
        qs = [(gid, nodes, 0, 0) for gid, nodes, _, _ in _queries(graphs, 9, 8)]
        qs += _queries(graphs, 5, 9)  # fresh pivot sets in the same stream of requests
        alone = [P.cfc_server_poll(sv, P.cfc_server_submit(sv, g, nodes, kk, seed), -1)[0]
                 for g, nodes, kk, seed in qs]
        rids = [P.cfc_server_submit(sv, g, nodes, kk, seed) for g, nodes, kk, seed in qs]
        mix = [P.cfc_server_poll(sv, r, -1)[0] for r in rids]
        for a, m in zip(alone, mix):
            assert np.array_equal(a, m)
        for (gid, nodes, kk, seed), f in zip(qs[:4], alone[:4]):
            n, s, d, w = graphs[gid]
            fo = sampling.sampled_farness(canonical_graph(n, s, d, w), 40, 11 + gids[gid], nodes.tolist(),
                                          solver="dense")
            assert np.max(np.abs(f - fo) / np.abs(fo)) <= FARNESS_RTOL
    finally:
        sv.destroy()
    plain = P.cfc_server_create(P.cfc_server_default_opts(slots=1))
    try:
        n, s, d, w = graphs[0]
        gid = P.cfc_server_add_graph(plain, n, s, d, w)
        with pytest.raises(P.LapError) as e:  # no resident set on this server
            P.cfc_server_submit(plain, gid, [1, 2], 0)
        assert e.value.status == P.LAP_EINVAL
    finally:
        plain.destroy()


@pytest.mark.parametrize("resident", [False, True])
def test_server_merges_queued_requests_with_the_same_bits(P, resident):
    # one slot: while the first request runs, the rest queue up and the next
    # admission solves the queued requests on the same graph as one block;
    # every result equals the one the request got alone
    graphs = _graphs()[:2]
    opts = P.cfc_server_default_opts(slots=1, batch_columns=1024, resident_pivots=60 if resident else 0,
                                     pivot_seed=7)
    sv = P.cfc_server_create(opts)
    try:
        for n, s, d, w in graphs:
            P.cfc_server_add_graph(sv, n, s, d, w)
        qs = [(gid, nodes, 0 if resident else kk, seed) for gid, nodes, kk, seed in _queries(graphs, 12, 9)]
        alone = []
        for gid, nodes, kk, seed in qs:
            f, info = P.cfc_server_poll(sv, P.cfc_server_submit(sv, gid, nodes, kk, seed), -1)
            assert info["status"] == P.LAP_OK
            alone.append(f)
        P.cfc_server_reset_stats(sv)
        rids = [P.cfc_server_submit(sv, gid, nodes, kk, seed) for gid, nodes, kk, seed in qs]
        merged = [P.cfc_server_poll(sv, r, -1)[0] for r in rids]
        st = P.cfc_server_stats(sv)
        assert st["max_batch"] >= 2 and st["completed"] == len(qs)
        for a, m in zip(alone, merged):
            assert np.array_equal(a, m)
    finally:
        sv.destroy()
