"""Edge-list generators.  Every function returns ``(n, src, dst, w)`` with
``src``/``dst`` int32 arrays of length m and ``w`` a float64 array (or
``None`` for unit weights).  Edges are undirected; each appears once.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Distinct values of an integer array in increasing order (a plain sort
    and a neighbour comparison: much faster than np.unique at 10^7+ values)."""
    s = np.sort(a)
    if s.size == 0:
        return s
    keep = np.empty(s.size, bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def uniform_weights(m: int, seed: int, lo: float = 1.0, hi: float = 2.0) -> np.ndarray:
    """Edge weights drawn uniformly from [lo, hi)."""
    return _rng(seed).uniform(lo, hi, size=m).astype(np.float64)


def grid2d(a: int, b: int | None = None):
    """a x b 4-neighbour grid; node (r, c) has id r*b + c.  m = a(b-1) + b(a-1)."""
    b = a if b is None else b
    ids = np.arange(a * b, dtype=np.int64).reshape(a, b)
    right_s = ids[:, :-1].ravel()
    right_d = ids[:, 1:].ravel()
    down_s = ids[:-1, :].ravel()
    down_d = ids[1:, :].ravel()
    src = np.concatenate([right_s, down_s]).astype(np.int32)
    dst = np.concatenate([right_d, down_d]).astype(np.int32)
    return a * b, src, dst, None


def torus2d(a: int):
    """a x a 4-neighbour grid with wrap-around edges (every degree 4);
    node (r, c) has id r*a + c.  m = 2 a^2 (a >= 3)."""
    ids = np.arange(a * a, dtype=np.int64).reshape(a, a)
    src = np.concatenate([ids.ravel(), ids.ravel()]).astype(np.int32)
    dst = np.concatenate([np.roll(ids, -1, axis=1).ravel(), np.roll(ids, -1, axis=0).ravel()]).astype(np.int32)
    return a * a, src, dst, None


def random_regular(n: int, d: int, seed: int):
    """Uniform random d-regular simple connected graph by the configuration
    model: the n*d edge stubs are paired by a random permutation, and the
    pairing is drawn again until it has no self-loop, no repeated pair and
    one component.  m = n d / 2 (n d even)."""
    rng = _rng(seed)
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    while True:
        p = rng.permutation(stubs).reshape(-1, 2)
        lo, hi = p.min(axis=1), p.max(axis=1)
        if np.any(lo == hi) or np.unique(lo * n + hi).size != lo.size:
            continue
        parent = np.arange(n)  # connectivity by union-find over the pairs

        def find(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        for u, v in zip(lo.tolist(), hi.tolist()):
            ru, rv = find(u), find(v)
            if ru != rv:
                parent[ru] = rv
        if len({find(x) for x in range(n)}) == 1:
            return n, lo.astype(np.int32), hi.astype(np.int32), None


def path_graph(n: int):
    s = np.arange(n - 1, dtype=np.int32)
    return n, s, s + 1, None


def cycle_graph(n: int):
    s = np.arange(n, dtype=np.int32)
    return n, s, ((s + 1) % n).astype(np.int32), None


def complete_graph(n: int):
    iu, ju = np.triu_indices(n, 1)
    return n, iu.astype(np.int32), ju.astype(np.int32), None


def star_graph(leaves: int):
    d = np.arange(1, leaves + 1, dtype=np.int32)
    return leaves + 1, np.zeros(leaves, np.int32), d, None


def random_tree(n: int, seed: int):
    """Random recursive tree: node i > 0 attaches to a uniform earlier node."""
    rng = _rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int32)
    return n, parent, np.arange(1, n, dtype=np.int32), None


def erdos_renyi_connected(n: int, p: float, seed: int):
    """G(n, p) plus a random spanning path, so the result is connected."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    perm = rng.permutation(n)
    ps, pd = perm[:-1], perm[1:]
    src = np.concatenate([iu[keep], np.minimum(ps, pd)])
    dst = np.concatenate([ju[keep], np.maximum(ps, pd)])
    key = np.unique(src.astype(np.int64) * n + dst)
    return n, (key // n).astype(np.int32), (key % n).astype(np.int32), None


def barabasi_albert(n: int, m_per_node: int = 5, seed: int = 2, clique: int = 6):
    """Preferential attachment: a seed clique on ``clique`` nodes, then each new
    node attaches to ``m_per_node`` distinct earlier nodes drawn from the
    list of all edge endpoints so far (probability proportional to degree).
    m = clique(clique-1)/2 + m_per_node (n - clique)."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(clique, 1)
    m_total = iu.size + m_per_node * (n - clique)
    src = np.empty(m_total, np.int32)
    dst = np.empty(m_total, np.int32)
    src[: iu.size] = iu
    dst[: iu.size] = ju
    ends = np.empty(2 * m_total, np.int32)
    ends[: iu.size] = iu
    ends[iu.size: 2 * iu.size] = ju
    n_ends = 2 * iu.size
    e = iu.size
    # draw in batches of candidate endpoints; reject repeats within a node
    for v in range(clique, n):
        chosen: list[int] = []
        while len(chosen) < m_per_node:
            cand = ends[rng.integers(0, n_ends, size=2 * m_per_node)]
            for c in cand:
                c = int(c)
                if c not in chosen:
                    chosen.append(c)
                    if len(chosen) == m_per_node:
                        break
        for c in chosen:
            src[e] = c
            dst[e] = v
            ends[n_ends] = c
            ends[n_ends + 1] = v
            n_ends += 2
            e += 1
    return n, src, dst, None


def largest_component(n: int, src: np.ndarray, dst: np.ndarray, w=None):
    """Restrict an edge list to its largest connected component and relabel the
    kept nodes 0..n'-1 in increasing original order (Sec. 6.3 uses the LCC of
    every instance)."""
    a = sp.coo_matrix((np.ones(src.size), (src, dst)), shape=(n, n))
    ncomp, lab = csgraph.connected_components(a, directed=False)
    if ncomp == 1:
        return n, src, dst, w
    big = np.argmax(np.bincount(lab))
    keep = lab == big
    newid = np.full(n, -1, np.int64)
    newid[keep] = np.arange(int(keep.sum()))
    em = keep[src] & keep[dst]
    w2 = None if w is None else w[em]
    return int(keep.sum()), newid[src[em]].astype(np.int32), newid[dst[em]].astype(np.int32), w2


_RMAT_CHUNK = 1 << 22


def _rmat_chunk(args):
    """Samples [c * 2^22, ...) of the R-MAT stream: quadrant bits, level by
    level, from a generator seeded by (seed, chunk), so the stream does not
    depend on how the chunks are spread over processes."""
    scale, count, a, b, c, seed, chunk = args
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x524D4154, int(chunk)])))
    ab = a + b
    c_norm = c / (1.0 - ab)
    a_norm = a / ab
    uu = np.zeros(count, np.int64)
    vv = np.zeros(count, np.int64)
    for bit in range(scale):
        r1 = rng.random(count)
        r2 = rng.random(count)
        ubit = r1 > ab
        vbit = np.where(ubit, r2 > c_norm, r2 > a_norm)
        uu |= ubit.astype(np.int64) << bit
        vv |= vbit.astype(np.int64) << bit
    return uu.astype(np.int32), vv.astype(np.int32)


def rmat(scale: int, edge_factor: int = 8, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 3, permute: bool = True, processes: int | None = None):
    """R-MAT (Chakrabarti et al.) with ``edge_factor * 2**scale`` directed
    samples: at each of ``scale`` levels pick quadrant (a, b, c, d).  Then a
    random vertex permutation, symmetrisation, removal of self-loops and
    duplicate pairs, and restriction to the largest connected component.
    ``edge_factor=8`` directed samples per node give average degree ~16 after
    symmetrisation.  Samples come in chunks of 2^22 with their own seeded
    streams; large instances spread the chunks over a spawned process pool
    (the result is the same).  Returns (n, src, dst, None) with src < dst."""
    nsamp = edge_factor << scale
    jobs = [(scale, min(_RMAT_CHUNK, nsamp - lo), a, b, c, seed, i)
            for i, lo in enumerate(range(0, nsamp, _RMAT_CHUNK))]
    if processes is None:
        processes = min(16, os.cpu_count() or 1) if len(jobs) >= 8 else 1
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.map(_rmat_chunk, jobs)
    else:
        parts = [_rmat_chunk(j) for j in jobs]
    u = np.concatenate([p[0] for p in parts]).astype(np.int64)
    v = np.concatenate([p[1] for p in parts]).astype(np.int64)
    del parts
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0x524D4154, 1 << 40])))
    n = 1 << scale
    if permute:
        perm = rng.permutation(n)
        u = perm[u]
        v = perm[v]
    lo_ = np.minimum(u, v)
    hi_ = np.maximum(u, v)
    keep = lo_ != hi_
    key = _sorted_unique(lo_[keep] * n + hi_[keep])
    src = (key // n).astype(np.int32)
    dst = (key % n).astype(np.int32)
    return largest_component(n, src, dst, None)
