"""Host logic of the multi-GPU split of a JL query (row shards + one
all-reduce of q partial sums), run as two gloo ranks on the CPU.  The
partial sums come from the oracle (Algorithm 1 with a dense solve), so the
test checks the partition and the reduction, not the kernels."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import jl
from oracle.graph import canonical_graph
from paper_1607_02955_gb300.sharding import allreduce_partials, shard_rows


@pytest.mark.parametrize("k", [1, 5, 31, 32, 33, 64, 100, 257, 4096])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_rows_partition(k, world):
    got = [shard_rows(k, world, r) for r in range(world)]
    pos = 0
    for r0, c in got:
        assert c >= 0
        if c > 0:
            assert r0 == pos and r0 % 32 == 0
            pos += c
    assert pos == k
    sizes = [c for _, c in got]
    assert max(sizes) - min(sizes) < 64  # whole blocks dealt out evenly (the last may be partial)


def test_shard_rows_rejects_bad_arguments():
    for args in [(0, 1, 0), (10, 0, 0), (10, 2, 2), (10, 2, -1)]:
        with pytest.raises(ValueError):
            shard_rows(*args)


GRAPH = dict(a=10, k=70, seed=3, nodes=[0, 17, 55, 99])


def _oracle_rows():
    n, s, d, _ = synth.grid2d(GRAPH["a"])
    g = canonical_graph(n, s, d, synth.uniform_weights(s.size, seed=1))
    Z = jl.jl_solve(g, jl.jl_rhs(g, GRAPH["k"], GRAPH["seed"]))  # k x n
    return g, Z


def _partial(Z, nodes, r0, c):
    # literal row terms sum_{i in rows} sum_w (Z_iv - Z_iw)^2 (Algorithm 1, step 4)
    rows = Z[r0:r0 + c]
    return np.array([((rows - rows[:, [v]]) ** 2).sum() for v in nodes])


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, Z = _oracle_rows()
        f = allreduce_partials(lambda r0, c: _partial(Z, GRAPH["nodes"], r0, c), GRAPH["k"], len(GRAPH["nodes"]))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), f)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_allreduce_of_row_shards_gives_full_farness(tmp_path, world):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    g, Z = _oracle_rows()
    full = jl.jl_farness(g, GRAPH["k"], GRAPH["seed"], GRAPH["nodes"])
    for r in range(world):
        f = np.load(tmp_path / f"rank{r}.npy")
        np.testing.assert_allclose(f, full, rtol=1e-12)
