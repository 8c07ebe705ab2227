"""Pins for the oracle's Philox4x64-10 against numpy's library implementation.

numpy.random.Philox increments its 256-bit counter before generating a block,
so the oracle's block for counter c equals numpy's first block when numpy is
seeded with counter c - 1 (256-bit arithmetic, word 0 least significant).
"""

import numpy as np
import pytest

from oracle.philox import philox4x64_10

MASK64 = (1 << 64) - 1


def numpy_block(counter, key):
    c = sum(int(w) << (64 * i) for i, w in enumerate(counter))
    c = (c - 1) % (1 << 256)
    prev = [(c >> (64 * i)) & MASK64 for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    return tuple(int(x) for x in bg.random_raw(4))


@pytest.mark.parametrize("case", range(40))
def test_philox_matches_numpy(case):
    rng = np.random.default_rng(1234 + case)
    counter = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
    if case % 4 == 0:
        counter = [case, case * 7, 0, 0]          # the small counters the relabel kernel uses
    if case == 1:
        counter = [0, 5, 0, 0]                    # borrow across word 0 in the numpy conversion
    key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
    assert philox4x64_10(counter, key) == numpy_block(counter, key)


def test_philox_output_words_differ_across_counters():
    outs = {philox4x64_10((s, b, 0, 0), (7, 0)) for s in range(4) for b in range(64)}
    assert len(outs) == 256
