"""Pins for the oracle's energies, InfoNCE objectives, penalty and gradients.

Independent checks: library routines (scipy cdist, scipy logsumexp), pure
Python enumeration of the softmax terms on B <= 4, closed forms (log B at
equal representations), the fwd/bwd transpose identity, and central finite
differences in FP64.
"""

import itertools
import math

import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.special import logsumexp as sp_lse

from oracle import critic


def reps(B, R, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, R)), rng.standard_normal((B, R))


@pytest.mark.parametrize("tau", [1.0, 0.5])
def test_energies_against_scipy(tau):
    phi, psi = reps(7, 5, 0)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "l2", tau), -cdist(phi, psi) / tau, rtol=1e-13)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "l2sq", tau), -cdist(phi, psi, "sqeuclidean") / tau,
                               rtol=1e-12)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "l1", tau), -cdist(phi, psi, "cityblock") / tau,
                               rtol=1e-13)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "cos", tau), (1.0 - cdist(phi, psi, "cosine")) / tau,
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "dot", tau),
                               np.einsum("ir,jr->ij", phi, psi) / tau, rtol=1e-13)
    for e in critic.ENERGIES:
        np.testing.assert_allclose(critic.energy_diagonal(phi, psi, e, tau),
                                   np.diagonal(critic.energy_matrix(phi, psi, e, tau)), rtol=1e-13)


def test_logsumexp_against_scipy():
    x = np.random.default_rng(1).standard_normal((6, 9)) * 30
    for ax in (0, 1):
        np.testing.assert_allclose(critic.logsumexp(x, ax), sp_lse(x, axis=ax), rtol=1e-14)


def brute_force_loss(F, loss, red, beta, axis):
    """Pure-Python enumeration of every softmax term (no numpy arithmetic)."""
    B = len(F)
    fwd_terms, bwd_terms, rows, cols = [], [], [], []
    for i in range(B):
        row = sum(math.exp(F[i][j]) for j in range(B))
        col = sum(math.exp(F[j][i]) for j in range(B))
        fwd_terms.append(-math.log(math.exp(F[i][i]) / row))
        bwd_terms.append(-math.log(math.exp(F[i][i]) / col))
        rows.append(math.log(row))
        cols.append(math.log(col))
    l_fwd = sum(fwd_terms) / B
    l_bwd = sum(bwd_terms) / B
    w = {"fwd": (1, 0), "bwd": (0, 1), "sym": (0.5, 0.5) if red == "mean" else (1, 1)}[loss]
    p = {"row": (1, 0), "col": (0, 1), "both": (0.5, 0.5)}[axis]
    pen = beta * (p[0] * sum(r * r for r in rows) / B + p[1] * sum(c * c for c in cols) / B)
    return w[0] * l_fwd + w[1] * l_bwd + pen, l_fwd, l_bwd, pen


@pytest.mark.parametrize("B", [1, 2, 3, 4])
@pytest.mark.parametrize("loss,red", [("fwd", "mean"), ("bwd", "mean"), ("sym", "mean"), ("sym", "sum")])
@pytest.mark.parametrize("axis", ["row", "col", "both"])
def test_infonce_brute_force(B, loss, red, axis):
    rng = np.random.default_rng(B * 31 + len(loss))
    F = rng.standard_normal((B, B)) * 2
    out = critic.infonce_loss(F, loss, red, 0.1, axis)
    total, l_fwd, l_bwd, pen = brute_force_loss(F.tolist(), loss, red, 0.1, axis)
    assert out["total"] == pytest.approx(total, rel=1e-13, abs=1e-14)
    assert out["fwd"] == pytest.approx(l_fwd, rel=1e-13, abs=1e-14)
    assert out["bwd"] == pytest.approx(l_bwd, rel=1e-13, abs=1e-14)
    assert out["penalty"] == pytest.approx(pen, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("B", [2, 16, 256])
@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l1", "l2sq"])
def test_equal_representations_give_log_B(B, energy):
    x = np.random.default_rng(B).standard_normal(8)
    phi = np.tile(x, (B, 1))
    F = critic.energy_matrix(phi, phi, energy, 1.0)
    for loss in ("fwd", "bwd", "sym"):
        out = critic.infonce_loss(F, loss, "mean", 0.1, "row")
        assert out["contrastive"] == pytest.approx(math.log(B), rel=1e-12)
    out = critic.infonce_loss(F, "sym", "sum", 0.1, "row")
    assert out["contrastive"] == pytest.approx(2 * math.log(B), rel=1e-12)
    if energy in ("l2", "l1", "l2sq"):          # F == 0 exactly
        assert out["penalty"] == pytest.approx(0.1 * math.log(B) ** 2, rel=1e-12)


def test_backward_is_forward_of_transpose_and_sym_identities():
    F = np.random.default_rng(3).standard_normal((9, 9)) * 3
    a = critic.infonce_loss(F, "bwd", "mean", 0.0)
    b = critic.infonce_loss(F.T, "fwd", "mean", 0.0)
    assert a["total"] == pytest.approx(b["total"], rel=1e-14)
    s_mean = critic.infonce_loss(F, "sym", "mean", 0.0)["total"]
    s_sum = critic.infonce_loss(F, "sym", "sum", 0.0)["total"]
    assert s_sum == pytest.approx(2 * s_mean, rel=1e-14)
    assert s_sum == pytest.approx(a["fwd"] + a["bwd"], rel=1e-14)


def central_fd(f, x, idx, h):
    x = x.copy()
    x0 = x[idx]
    x[idx] = x0 + h
    fp = f(x)
    x[idx] = x0 - h
    fm = f(x)
    return (fp - fm) / (2 * h)


@pytest.mark.parametrize("loss,red", [("fwd", "mean"), ("bwd", "mean"), ("sym", "mean"), ("sym", "sum")])
@pytest.mark.parametrize("axis", ["row", "col", "both"])
def test_grad_F_against_finite_differences(loss, red, axis):
    F = np.random.default_rng(4).standard_normal((5, 5)) * 2
    G = critic.infonce_grad_F(F, loss, red, 0.1, axis)
    f = lambda X: critic.infonce_loss(X, loss, red, 0.1, axis)["total"]
    for idx in itertools.product(range(5), range(5)):
        assert G[idx] == pytest.approx(central_fd(f, F, idx, 1e-6), rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l1", "l2sq"])
@pytest.mark.parametrize("tau", [1.0, 0.7])
def test_energy_backward_against_finite_differences(energy, tau):
    phi, psi = reps(6, 4, 5)
    G = np.random.default_rng(6).standard_normal((6, 6))
    dphi, dpsi = critic.energy_backward(phi, psi, G, energy, tau)
    for which, d in (("phi", dphi), ("psi", dpsi)):
        def f(X):
            p, q = (X, psi) if which == "phi" else (phi, X)
            return float((G * critic.energy_matrix(p, q, energy, tau)).sum())
        base = phi if which == "phi" else psi
        for idx in itertools.product(range(6), range(4)):
            assert d[idx] == pytest.approx(central_fd(f, base, idx, 1e-6), rel=1e-6, abs=1e-8)
    gd = np.random.default_rng(7).standard_normal(6)
    dphi, dpsi = critic.energy_diagonal_backward(phi, psi, gd, energy, tau)
    full_phi, full_psi = critic.energy_backward(phi, psi, np.diag(gd), energy, tau)
    np.testing.assert_allclose(dphi, full_phi, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(dpsi, full_psi, rtol=1e-12, atol=1e-14)


def test_l2_gradient_zero_at_coincident_points():
    phi = np.zeros((3, 4))
    G = np.ones((3, 3))
    dphi, dpsi = critic.energy_backward(phi, phi.copy(), G, "l2", 1.0)
    assert np.all(dphi == 0) and np.all(dpsi == 0)


def test_row_wise_energies_match_dense_broadcast():
    """The row-at-a-time evaluation equals the dense [i][j][r] broadcast of the definition."""
    phi, psi = reps(9, 6, 11)
    diff = phi[:, None, :] - psi[None, :, :]
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "l2"), -np.sqrt((diff ** 2).sum(2)), rtol=1e-14)
    np.testing.assert_allclose(critic.energy_matrix(phi, psi, "l1"), -np.abs(diff).sum(2), rtol=1e-14)
    G = np.random.default_rng(12).standard_normal((9, 9))
    d = np.sqrt((diff ** 2).sum(2))
    H = G / d
    dphi, dpsi = critic.energy_backward(phi, psi, G, "l2", 1.0)
    np.testing.assert_allclose(dphi, -(H[:, :, None] * diff).sum(1), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(dpsi, (H[:, :, None] * diff).sum(0), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("energy", ["l2", "l2sq", "l1"])
def test_row_blocks_give_the_same_bits_on_any_thread_count(energy, monkeypatch):
    """Several row blocks (B > ROW_BLOCK, ragged last block): one thread and four
    threads give identical bits (the block partition is fixed), and both equal
    the dense [i][j][r] broadcast of the definition."""
    B, R = critic.ROW_BLOCK * 2 + 37, 5
    phi, psi = reps(B, R, 13)
    G = np.random.default_rng(14).standard_normal((B, B))
    out = {}
    for n in ("1", "4"):
        monkeypatch.setenv("OMP_NUM_THREADS", n)
        out[n] = (critic.energy_matrix(phi, psi, energy), *critic.energy_backward(phi, psi, G, energy, 0.8))
    for a, b in zip(out["1"], out["4"]):
        np.testing.assert_array_equal(a, b)
    diff = phi[:, None, :] - psi[None, :, :]
    if energy == "l2":
        dense = -np.sqrt((diff ** 2).sum(2))
        term = (G / (0.8 * -dense))[:, :, None] * diff
    elif energy == "l2sq":
        dense = -(diff ** 2).sum(2)
        term = (2.0 * G / 0.8)[:, :, None] * diff
    else:
        dense = -np.abs(diff).sum(2)
        term = (G / 0.8)[:, :, None] * np.sign(diff)
    np.testing.assert_allclose(out["1"][0], dense, rtol=1e-14)
    np.testing.assert_allclose(out["1"][1], -term.sum(1), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(out["1"][2], term.sum(0), rtol=1e-11, atol=1e-12)
