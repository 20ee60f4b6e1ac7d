"""Pins of the oracle's sort (the tile-list and depth sort of the path, Sec. 1) against a brute
force on small inputs and against the properties that define a stable sort."""
import numpy as np
import pytest

import oracle


def _insertion_sort(keys, vals, key_bits):
    """Stable sort by repeated insertion, in plain Python."""
    mask = (1 << key_bits) - 1
    out = []
    for k, v in zip(keys.tolist(), vals.tolist()):
        pos = len(out)
        while pos > 0 and (out[pos - 1][0] & mask) > (k & mask):
            pos -= 1
        out.insert(pos, (k, v))
    return np.array([k for k, _ in out], np.uint32), np.array([v for _, v in out], np.uint32)


@pytest.mark.parametrize("n,key_bits,seed", [(0, 8, 1), (1, 8, 2), (37, 3, 3), (200, 11, 4), (300, 32, 5),
                                             (257, 1, 6)])
def test_sort_matches_insertion_sort(n, key_bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    ok, ov = oracle.sort_pairs(keys, vals, key_bits)
    bk, bv = _insertion_sort(keys, vals, key_bits)
    assert np.array_equal(ok, bk) and np.array_equal(ov, bv)


def test_sort_is_a_stable_permutation_ordered_by_the_low_bits():
    rng = np.random.default_rng(7)
    n, key_bits = 50_000, 13
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)  # values are the input positions
    ok, ov = oracle.sort_pairs(keys, vals, key_bits)
    low = ok & np.uint32((1 << key_bits) - 1)
    assert np.all(low[1:] >= low[:-1])                   # ordered
    assert np.array_equal(np.sort(ov), vals)             # a permutation
    assert np.array_equal(ok, keys[ov])                  # keys travel with their values
    same = low[1:] == low[:-1]
    assert np.all(ov[1:][same] > ov[:-1][same])          # equal low bits keep input order


def test_sort_ignores_the_high_bits():
    keys = np.array([0x100 | 3, 0x200 | 1, 0x000 | 3, 0x300 | 1], np.uint32)
    vals = np.arange(4, dtype=np.uint32)
    ok, ov = oracle.sort_pairs(keys, vals, 8)
    assert ov.tolist() == [1, 3, 0, 2]
