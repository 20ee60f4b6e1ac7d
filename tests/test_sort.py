"""Device parity of the path's radix sort (the tile-list and depth sort, Sec. 1) through
wipes_sort_pairs: keys and values bit-exact against the oracle's stable sort, for pass counts
odd and even, ragged last tiles, heavy ties, and a size far above the tile lists of the
workloads."""
import numpy as np
import pytest

import oracle
from helpers import lib_ready, torch_cuda

pytestmark = pytest.mark.gpu


def _run(keys, vals, key_bits):
    torch = torch_cuda()
    w = lib_ready()
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    w.sort_pairs(k, v, key_bits)
    torch.cuda.synchronize()
    return k.cpu().numpy().view(np.uint32), v.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,key_bits,seed", [
    (2, 1, 1), (100, 6, 2), (4095, 11, 3), (4096, 11, 4), (4097, 17, 5), (8197, 32, 6),
    (250_001, 13, 7), (3_000_017, 32, 8), (1_000_003, 17, 9), (777_777, 8, 10),
])
def test_sort_matches_oracle(n, key_bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    dk, dv = _run(keys, vals, key_bits)
    ok, ov = oracle.sort_pairs(keys, vals, key_bits)
    assert np.array_equal(dk, ok)
    assert np.array_equal(dv, ov)


@pytest.mark.parametrize("n,key_bits,shape,seed", [
    (300_001, 32, "top byte 0", 13),      # the last of four one-sweep passes has one digit
    (300_003, 24, "low byte 0", 14),      # the first pass has one digit
    (4097, 32, "top two bytes 0", 15),     # two passes with one digit, a ragged last tile
])
def test_sort_passes_with_a_single_digit(n, key_bits, shape, seed):
    """Passes whose digit is the same for every key keep the order as it is (the kernels copy the
    tile instead of ranking it); the result still equals the oracle's stable sort."""
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    if shape == "top byte 0":
        keys &= np.uint32(0x00FFFFFF)
    elif shape == "low byte 0":
        keys &= np.uint32(0x00FFFF00)
    else:
        keys &= np.uint32(0x0000FFFF)
    vals = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    dk, dv = _run(keys, vals, key_bits)
    ok, ov = oracle.sort_pairs(keys, vals, key_bits)
    assert np.array_equal(dk, ok)
    assert np.array_equal(dv, ov)


def test_sort_with_heavy_ties_keeps_input_order():
    rng = np.random.default_rng(11)
    n = 600_001
    keys = rng.integers(0, 3, n).astype(np.uint32) | (rng.integers(0, 2**20, n).astype(np.uint32) << 12)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = _run(keys, vals, 12)
    ok, ov = oracle.sort_pairs(keys, vals, 12)
    assert np.array_equal(dk, ok) and np.array_equal(dv, ov)
    dk, dv = _run(np.zeros(n, np.uint32), vals, 32)  # all keys equal: the identity
    assert np.array_equal(dv, vals)


def test_sort_large_input_above_l2():
    rng = np.random.default_rng(12)
    n = (1 << 25) + 5  # 268 MB of pairs, twice the L2
    keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = _run(keys, vals, 32)
    ok, ov = oracle.sort_pairs(keys, vals, 32)
    assert np.array_equal(dk, ok) and np.array_equal(dv, ov)


def test_sort_trivial_sizes_and_bad_arguments():
    torch = torch_cuda()
    w = lib_ready()
    from paper_2508_12615_gb300 import _abi

    for n in (0, 1):
        k = torch.arange(n, dtype=torch.int32, device="cuda")
        v = torch.arange(n, dtype=torch.int32, device="cuda")
        w.sort_pairs(k, v, 8)
        assert k.tolist() == list(range(n))
    k = torch.zeros(16, dtype=torch.int32, device="cuda")
    for bits in (0, 33):
        with pytest.raises(_abi.WipesError) as e:
            w.sort_pairs(k, k.clone(), bits)
        assert e.value.status == 1
