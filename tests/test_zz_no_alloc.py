"""The allocation-free farness reduction, cfc_farness_from_solution_noalloc.

It exists for callers that cannot allocate device memory at the moment they
need a farness (an allocator or out-of-memory handler, a process held to a
hard memory cap, a stream that must not wait on the allocator).  Its scratch
is a fixed array inside the library, shared by every call.  This test calls
it through the C ABI twice in a row, on the same and on a different problem,
and compares each result with the allocating entry point
cfc_farness_from_solution.  The file is named to run last in a full run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-12


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


def _case(torch, n, k, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    Z = torch.randn((n, k), dtype=torch.float64, device="cuda", generator=g)
    nodes = torch.tensor(np.random.default_rng(seed).integers(0, n, size=7), dtype=torch.int32, device="cuda")
    return Z, nodes


def test_noalloc_matches_allocating_entry_point_twice(P):
    import torch
    for n, k, seed in [(20000, 64, 1), (20000, 64, 1), (3001, 200, 2)]:
        Z, nodes = _case(torch, n, k, seed)
        ref = P.cfc_farness_from_solution(Z, nodes.cpu().numpy())
        for _ in range(2):
            out = torch.full((nodes.numel(),), float("nan"), dtype=torch.float64, device="cuda")
            P.cfc_farness_from_solution_noalloc(Z, nodes, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    import torch
    Z, nodes = _case(torch, 100, 257, 3)
    out = torch.empty(nodes.numel(), dtype=torch.float64, device="cuda")
    with pytest.raises(P.LapError) as e:
        P.cfc_farness_from_solution_noalloc(Z, nodes, out)
    assert e.value.status == P.LAP_EBUDGET


def test_noalloc_out_of_range_nodes_get_nan(P):
    # a node id outside [0, n) yields NaN at its position and leaves the
    # other positions equal to the allocating entry point's values
    import torch
    Z, _ = _case(torch, 5000, 48, 4)
    good = np.array([0, 17, 4999], np.int32)
    ref = P.cfc_farness_from_solution(Z, good)
    nodes = torch.tensor([0, -1, 17, 5000, 4999], dtype=torch.int32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    P.cfc_farness_from_solution_noalloc(Z, nodes, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isnan(got[1]) and np.isnan(got[3])
    np.testing.assert_allclose(got[[0, 2, 4]], ref, rtol=RTOL, atol=0)
