"""Philox4x64-10, written out from its published definition.

Test infrastructure only (see ``oracle/__init__``).

The relabelling step of the CRL update draws its random numbers from a
counter-based generator so that the CPU oracle and the GPU kernels can draw
the *same* numbers independently.  Philox4x64-10 is defined in
J. Salmon, M. Moraes, R. Dror, D. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11: a 4-word (64-bit) counter and a 2-word key; each of the ten
rounds multiplies words 0 and 2 by two fixed odd constants, keeps the 128-bit
products' high and low halves, XORs the high halves with the other counter
words and the round key, and permutes; the key is bumped by two Weyl
constants (the golden ratio and sqrt(3) - 1, scaled to 2^64) between rounds.

Pinned in ``tests/test_oracle_philox.py`` against ``numpy.random.Philox``
(an independent library implementation of the same generator).
"""

MASK64 = (1 << 64) - 1

# Round multipliers and Weyl key increments of Philox4x64 (Salmon et al. 2011).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(counter, key):
    """Return the four 64-bit output words for ``counter`` (4 ints) under ``key`` (2 ints)."""
    x0, x1, x2, x3 = (int(c) & MASK64 for c in counter)
    k0, k1 = (int(k) & MASK64 for k in key)
    for _ in range(10):
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK64
        k1 = (k1 + PHILOX_W1) & MASK64
    return x0, x1, x2, x3
