"""Pins of the oracle's random block order (Sec. 2.2.2 lists random subset
orders; the reading is a Fisher-Yates shuffle driven by SplitMix64): the
generator against the published reference outputs of SplitMix64, the
shuffle's permutations valid and uniform, one block = acquisition order."""
import collections

import numpy as np
import pytest

import oracle


def test_splitmix64_reference_outputs():
    """Published outputs of the reference SplitMix64: seed 0 gives
    0xE220A8397B1DCDAF first; seed 1234567 gives the five values below."""
    _, v = oracle.splitmix64(0)
    assert v == 0xE220A8397B1DCDAF
    state, out = 1234567, []
    for _ in range(5):
        state, v = oracle.splitmix64(state)
        out.append(v)
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                   16408922859458223821]


def test_block_orders_are_uniform_permutations():
    counts = collections.Counter()
    for seed in range(6000):
        perm = oracle.block_orders(3, 1, "random", seed)[0]
        assert sorted(perm) == [0, 1, 2]
        counts[tuple(perm)] += 1
    assert len(counts) == 6
    # 1000 expected per permutation; 5 sigma ~ 5 * sqrt(1000 * 5/6)
    assert all(abs(c - 1000) < 150 for c in counts.values()), counts
    many = oracle.block_orders(36, 4, "random", 5)
    assert all(sorted(p) == list(range(36)) for p in many)
    assert len({tuple(p) for p in many}) == 4  # the stream moves on between iterations


def test_one_block_and_sequential_order():
    assert oracle.block_orders(1, 3, "random", 9) == [[0], [0], [0]]
    assert oracle.block_orders(4, 2, "sequential", 9) == [[0, 1, 2, 3]] * 2
    with pytest.raises(ValueError):
        oracle.block_orders(4, 1, "shuffled")
