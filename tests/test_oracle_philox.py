"""Pin the oracle's Philox4x64-10 against numpy's own Philox bit generator
(the same published generator), and check the derived sign stream."""
import numpy as np

from oracle import philox
from oracle.jl import jl_sign_bits


def _numpy_block(ctr, key):
    # numpy advances the 256-bit counter by one before producing each block
    # of four words, so seeding it with ctr - 1 yields philox(ctr, key)
    c = list(ctr)
    c[0] -= 1
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return [int(x) for x in bg.random_raw(4)]


def test_scalar_matches_numpy():
    for ctr, key in [((1, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (5, 7)),
                     ((12345, 3, 0, 0), (2**63 + 11, philox.TAG_JL)),
                     ((2**40 + 1, 2**33, 7, 2**64 - 1), (2**64 - 1, 2**64 - 2))]:
        assert philox.philox4x64_10_int(ctr, key) == _numpy_block(ctr, key)


def test_vector_matches_scalar():
    e = np.arange(1, 200, dtype=np.uint64) * np.uint64(7919)
    w = philox.philox4x64_10(e, np.uint64(2), np.uint64(0), np.uint64(0), 77, philox.TAG_SAMPLE)
    for j in range(0, 199, 17):
        ref = philox.philox4x64_10_int((int(e[j]), 2, 0, 0), (77, philox.TAG_SAMPLE))
        assert [int(w[t][j]) for t in range(4)] == ref


def test_sign_bits_layout_and_balance():
    bits = jl_sign_bits(seed=3, k=300, edge_ids=np.arange(4000))
    # row i of edge e: bit (i % 64) of word (i % 256) // 64 of counter (e, i // 256)
    for e in (0, 17, 3999):
        for i in (0, 63, 64, 255, 256, 299):
            word = philox.philox4x64_10_int((e, i // 256, 0, 0), (3, philox.TAG_JL))[(i % 256) // 64]
            assert bits[e, i] == (word >> (i % 64)) & 1
    p = bits.mean()
    assert abs(p - 0.5) < 0.005
    # adjacent-row correlation of the +-1 signs is ~0
    s = 1.0 - 2.0 * bits
    assert abs(np.mean(s[:, :-1] * s[:, 1:])) < 0.01
