"""Pins for the oracle's logit statistics (a diagnostic of the energy matrix):
pure-Python enumeration of the pairs on B <= 4, constant and diagonal matrices,
B = 1, and the decomposition of the full sum into positives and negatives."""

import math

import numpy as np
import pytest

from oracle import critic


def brute(F):
    B = len(F)
    pos = [F[i][i] for i in range(B)]
    neg = [F[i][j] for i in range(B) for j in range(B) if i != j]
    return sum(pos) / len(pos), (sum(neg) / len(neg) if neg else math.nan)


@pytest.mark.parametrize("B", [2, 3, 4])
def test_brute_force(B):
    F = np.random.default_rng(B).standard_normal((B, B))
    d, o = critic.logit_stats(F)
    bd, bo = brute(F.tolist())
    assert d == pytest.approx(bd, rel=1e-14, abs=1e-15)
    assert o == pytest.approx(bo, rel=1e-14, abs=1e-15)


def test_constant_and_diagonal_matrices():
    assert critic.logit_stats(np.full((5, 5), -2.5)) == (pytest.approx(-2.5), pytest.approx(-2.5))
    d, o = critic.logit_stats(np.diag([1.0, 2.0, 3.0]))
    assert d == pytest.approx(2.0) and o == 0.0


def test_single_sample_has_no_negatives():
    d, o = critic.logit_stats(np.array([[0.75]]))
    assert d == 0.75 and math.isnan(o)


def test_sum_decomposes_into_positives_and_negatives():
    B = 7
    F = np.random.default_rng(9).standard_normal((B, B)) * 3.0
    d, o = critic.logit_stats(F)
    assert B * d + B * (B - 1) * o == pytest.approx(F.sum(), rel=1e-13)


def test_energy_matrix_of_equal_representations():
    """All phi_i = psi_j: L2 gives F = 0 everywhere, dot gives |x|^2 / tau everywhere."""
    x = np.random.default_rng(4).standard_normal(6)
    phi = np.tile(x, (4, 1))
    assert critic.logit_stats(critic.energy_matrix(phi, phi, "l2")) == (0.0, 0.0)
    d, o = critic.logit_stats(critic.energy_matrix(phi, phi, "dot", 2.0))
    assert d == pytest.approx(x @ x / 2.0) and o == pytest.approx(x @ x / 2.0)
