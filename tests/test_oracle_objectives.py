"""Pins for the oracle's objectives outside the InfoNCE family (App. A.2, §5.2;
readings C8-C12): FlatNCE, Monte Carlo forward-backward, DPO, IPO, SPPO and
NCE-binary.

Independent checks: scikit-learn's log-loss and mean squared error, pure-Python
enumeration of every pair on B <= 4, closed forms at F = 0 and at the optima the
paper describes, shift invariances, the FlatNCE / InfoNCE gradient identity, and
central finite differences of pure-Python losses in FP64.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import critic

OTHER = ("flatnce_fwd", "flatnce_bwd", "fb", "dpo", "ipo", "sppo", "nce_binary")


def energies(B, seed, scale=1.0):
    return np.random.default_rng(seed).standard_normal((B, B)) * scale


def sig(x):
    return 1.0 / (1.0 + math.exp(-x))


def brute(F, loss):
    """Every term of the objective enumerated in pure Python (no numpy arithmetic)."""
    B = len(F)
    pairs = list(itertools.product(range(B), range(B)))
    if loss == "flatnce_fwd":        # the surrogate mean_i log S_i whose gradient reading C8 takes
        return sum(math.log(sum(math.exp(F[i][j] - F[i][i]) for j in range(B))) for i in range(B)) / B
    if loss == "flatnce_bwd":
        return sum(math.log(sum(math.exp(F[j][i] - F[i][i]) for j in range(B))) for i in range(B)) / B
    if loss == "fb":
        tot = 0.0
        for i in range(B):
            tot += -math.exp(F[i][i]) + sum(math.exp(F[i][j]) ** 2 for j in range(B) if j != i) / (2 * (B - 1))
        return tot / B
    if loss == "dpo":
        return sum(-math.log(sig(F[i][i] - F[i][j])) for i, j in pairs) / B ** 2
    if loss == "ipo":
        return sum(((F[i][i] - F[i][j]) - 1.0) ** 2 for i, j in pairs) / B ** 2
    if loss == "sppo":
        return sum((F[i][i] - 1.0) ** 2 + (F[i][j] + 1.0) ** 2 for i, j in pairs) / B ** 2
    if loss == "nce_binary":
        tot = 0.0
        for i, j in pairs:
            p = sig(F[i][j])
            tot += -math.log(p) if i == j else -math.log(1.0 - p)
        return tot / B ** 2
    raise ValueError(loss)


@pytest.mark.parametrize("B", [1, 2, 3, 4])
@pytest.mark.parametrize("loss", ["fb", "dpo", "ipo", "sppo", "nce_binary"])
def test_values_brute_force(B, loss):
    if loss == "fb" and B == 1:
        with pytest.raises(ValueError):
            critic.objective_value(energies(1, 0), "fb")
        return
    F = energies(B, B)
    assert critic.objective_value(F, loss) == pytest.approx(brute(F.tolist(), loss), rel=1e-13, abs=1e-15)


def test_flatnce_value_is_zero():
    F = energies(5, 1, 3.0)
    assert critic.objective_value(F, "flatnce_fwd") == 0.0
    assert critic.objective_value(F, "flatnce_bwd") == 0.0


def test_values_against_scikit_learn():
    metrics = pytest.importorskip("sklearn.metrics")
    B = 9
    F = energies(B, 2, 1.5)
    p = 1.0 / (1.0 + np.exp(-F))
    eye = np.eye(B)
    assert critic.objective_value(F, "nce_binary") == pytest.approx(
        metrics.log_loss(eye.ravel(), p.ravel(), labels=[0, 1]), rel=1e-12)
    delta = np.diagonal(F)[:, None] - F
    pd = 1.0 / (1.0 + np.exp(-delta))
    assert critic.objective_value(F, "dpo") == pytest.approx(
        metrics.log_loss(np.ones(B * B), pd.ravel(), labels=[0, 1]), rel=1e-12)
    assert critic.objective_value(F, "ipo") == pytest.approx(
        metrics.mean_squared_error(np.ones(B * B), delta.ravel()), rel=1e-12)
    pos = np.repeat(np.diagonal(F), B)
    assert critic.objective_value(F, "sppo") == pytest.approx(
        metrics.mean_squared_error(np.ones(B * B), pos) + metrics.mean_squared_error(-np.ones(B * B), F.ravel()),
        rel=1e-12)


@pytest.mark.parametrize("B", [2, 5])
def test_closed_forms_at_zero_energy(B):
    F = np.zeros((B, B))
    assert critic.objective_value(F, "fb") == pytest.approx(-0.5, abs=1e-15)
    assert critic.objective_value(F, "dpo") == pytest.approx(math.log(2.0), rel=1e-15)
    assert critic.objective_value(F, "ipo") == pytest.approx(1.0, rel=1e-15)
    assert critic.objective_value(F, "sppo") == pytest.approx(2.0, rel=1e-15)
    assert critic.objective_value(F, "nce_binary") == pytest.approx(math.log(2.0), rel=1e-15)


@pytest.mark.parametrize("B", [2, 6])
def test_optima_the_paper_describes(B):
    """App. A.2: IPO wants a gap of one between positive and negative scores, SPPO
    scores of +1 and -1.  At those points only the j = i terms remain, and the
    gradient vanishes for IPO (SPPO keeps the pull of (F_ii + 1)^2 on F_ii)."""
    eye = np.eye(B)
    F = eye.copy()                                   # F_ii - F_ij = 1 for j != i
    assert critic.objective_value(F, "ipo") == pytest.approx(1.0 / B, rel=1e-15)
    np.testing.assert_allclose(critic.objective_grad_F(F, "ipo"), 0.0, atol=1e-16)
    F = 2.0 * eye - 1.0                              # +1 on the diagonal, -1 elsewhere
    assert critic.objective_value(F, "sppo") == pytest.approx(4.0 / B, rel=1e-15)
    G = critic.objective_grad_F(F, "sppo")
    np.testing.assert_allclose(G * (1.0 - eye), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.diagonal(G), 4.0 / B ** 2, rtol=1e-14)


def test_dpo_and_nce_binary_limits():
    """Large margins: DPO keeps only log 2 / B from the j = i pairs; NCE-binary goes to 0."""
    B = 4
    F = 60.0 * (2.0 * np.eye(B) - 1.0)
    assert critic.objective_value(F, "dpo") == pytest.approx(math.log(2.0) / B, rel=1e-12)
    assert critic.objective_value(F, "nce_binary") < 1e-20


def central_fd(f, F, h=1e-6):
    G = np.zeros_like(F)
    for i, j in itertools.product(range(F.shape[0]), repeat=2):
        Fp, Fm = F.copy(), F.copy()
        Fp[i, j] += h
        Fm[i, j] -= h
        G[i, j] = (f(Fp.tolist()) - f(Fm.tolist())) / (2 * h)
    return G


@pytest.mark.parametrize("loss", OTHER)
@pytest.mark.parametrize("B", [2, 4])
def test_gradients_against_finite_differences(loss, B):
    F = energies(B, 10 + B, 0.8)
    G = critic.objective_grad_F(F, loss)
    np.testing.assert_allclose(G, central_fd(lambda x: brute(x, loss), F), rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("direction", ["fwd", "bwd"])
def test_flatnce_gradient_is_infonce_gradient(direction):
    """With j = i inside S_i the constant term exp(0) carries no gradient, so the
    FlatNCE gradient of reading C8 is InfoNCE's of the same direction exactly."""
    F = energies(7, 3, 2.0)
    np.testing.assert_allclose(critic.objective_grad_F(F, "flatnce_" + direction),
                               critic.infonce_grad_F(F, direction, "mean", 0.0), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("loss", ["dpo", "ipo", "flatnce_fwd"])
def test_row_shift_invariance(loss):
    """DPO, IPO and FlatNCE-fwd depend on F_ij - F_ii only: adding a constant to a
    row changes nothing, so every row of the gradient sums to zero."""
    F = energies(6, 4)
    G = critic.objective_grad_F(F, loss)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-15)
    F2 = F + np.arange(6.0)[:, None]
    assert critic.objective_value(F2, loss) == pytest.approx(critic.objective_value(F, loss), rel=1e-13, abs=1e-15)
    np.testing.assert_allclose(critic.objective_grad_F(F2, "flatnce_bwd").sum(axis=0) if loss == "flatnce_fwd"
                               else G.sum(axis=1), 0.0, atol=1e-15)


@pytest.mark.parametrize("loss", OTHER)
def test_penalty_is_added_to_every_objective(loss):
    """Reading C12: total = objective + beta * mean r^2, and the gradient adds the
    penalty's (InfoNCE with beta minus InfoNCE without it)."""
    F = energies(5, 8)
    parts = critic.critic_loss(F, loss, "mean", 0.1, "row")
    ref = critic.infonce_loss(F, "fwd", "mean", 0.1, "row")
    assert parts["penalty"] == pytest.approx(ref["penalty"], rel=1e-15)
    assert parts["total"] == pytest.approx(critic.objective_value(F, loss) + ref["penalty"], rel=1e-14)
    assert parts["fwd"] == ref["fwd"] and parts["bwd"] == ref["bwd"]
    pen = critic.infonce_grad_F(F, "fwd", "mean", 0.1, "row") - critic.infonce_grad_F(F, "fwd", "mean", 0.0, "row")
    np.testing.assert_allclose(critic.critic_grad_F(F, loss, "mean", 0.1, "row"),
                               critic.objective_grad_F(F, loss) + pen, rtol=1e-12, atol=1e-15)
