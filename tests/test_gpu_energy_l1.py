"""The -L1 energy on the fused path (App. A.2: F_ij = -|phi_i - psi_j|_1 / tau),
against the FP64 oracle.

Its tiles run on the FP32 SIMT lanes over the FP32 representations, so the op
(functional.infonce_loss(..., path="fused")) is held to the FP32 bars: loss
parts within 1e-5 relative, each gradient within 1e-4 relative (Frobenius) of
the oracle's.  The sign terms are exact (both sides take sign(x - y) of the same
FP32 values, sign(0) = 0); the error is the FP32 rounding of the sums.

Batches 8 (one partial tile), 136 and 520 (several 64- and 128-row tiles with a
ragged tail) cover the direct-write backward (one segment) and the segmented
one (partials added in order); batch 8192 with repr 256 is the large-batch
workload at full size.  The critic step and a grouped sweep train it too."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, functional

from parity_helpers import FP32_GRAD_RTOL, FP32_LOSS_RTOL, rel_err

pytestmark = pytest.mark.gpu

LOSSES = ["fwd", "bwd", "sym", "flatnce_fwd", "flatnce_bwd", "fb", "dpo", "ipo", "sppo", "nce_binary"]


def representations(B, R, seed, scale=0.08, ties=False):
    """Seeded FP32 phi, psi [B][R] (N(0, scale^2)); ties: psi_i = phi_i on the even
    rows and one column of phi copied into psi, so sign(0) terms occur."""
    rng = np.random.default_rng(seed)
    phi = (rng.standard_normal((B, R)) * scale).astype(np.float32)
    psi = (rng.standard_normal((B, R)) * scale).astype(np.float32)
    if ties:
        psi[::2] = phi[::2]
        psi[:, 3] = phi[:, 3]
    return phi, psi


def fused_l1(phi, psi, loss, sym_reduction="mean", penalty="row", tau=1.0, beta=0.1, dtotal=1.0):
    dev = torch.device("cuda")
    p = torch.from_numpy(phi).to(dev).requires_grad_(True)
    q = torch.from_numpy(psi).to(dev).requires_grad_(True)
    total, parts = functional.infonce_loss(p, q, "l1", loss, sym_reduction, penalty, tau, beta, "fused")
    (total * dtotal).backward()
    torch.cuda.synchronize()
    return parts.cpu().numpy(), p.grad.cpu().numpy(), q.grad.cpu().numpy()


def oracle_l1(phi, psi, loss, sym_reduction="mean", penalty="row", tau=1.0, beta=0.1, dtotal=1.0):
    F = oracle.critic.energy_matrix(phi, psi, "l1", float(np.float32(tau)))
    parts = oracle.critic.critic_loss(F, loss, sym_reduction, float(np.float32(beta)), penalty)
    G = oracle.critic.critic_grad_F(F, loss, sym_reduction, float(np.float32(beta)), penalty) * dtotal
    dphi, dpsi = oracle.critic.energy_backward(phi, psi, G, "l1", float(np.float32(tau)))
    return parts, dphi, dpsi


def check(got, ref, loss_rtol=FP32_LOSS_RTOL, grad_rtol=FP32_GRAD_RTOL):
    parts, gphi, gpsi = got
    rparts, rphi, rpsi = ref
    for i, k in enumerate(("total", "fwd", "bwd", "penalty")):
        assert abs(parts[i] - rparts[k]) <= loss_rtol * abs(rparts[k]) + 1e-7, (k, parts[i], rparts[k])
    for name, g, r in (("dphi", gphi, rphi), ("dpsi", gpsi, rpsi)):
        e = rel_err(g, r)
        assert e <= grad_rtol, f"{name}: relative error {e:.3e}"


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("B,R", [(8, 64), (136, 128), (520, 64)])
def test_fused_l1_matches_oracle(loss, B, R):
    phi, psi = representations(B, R, seed=B + R)
    check(fused_l1(phi, psi, loss), oracle_l1(phi, psi, loss))


@pytest.mark.parametrize("R,B", [(192, 264), (256, 136), (64, 392)])
@pytest.mark.parametrize("penalty", ["row", "col", "both"])
def test_fused_l1_every_repr_width_and_penalty_axis(R, B, penalty):
    phi, psi = representations(B, R, seed=7 * R + B)
    args = dict(loss="sym", sym_reduction="sum", penalty=penalty, tau=0.8, beta=0.25, dtotal=1.7)
    check(fused_l1(phi, psi, **args), oracle_l1(phi, psi, **args))


@pytest.mark.parametrize("loss", ["sym", "dpo", "nce_binary"])
def test_fused_l1_ties_take_sign_zero(loss):
    """Equal coordinates (whole equal rows, one equal column) contribute nothing to
    the sign sums; the anchors F_ii of DPO then sit at 0."""
    phi, psi = representations(136, 64, seed=3, ties=True)
    check(fused_l1(phi, psi, loss), oracle_l1(phi, psi, loss))


def test_fused_l1_equal_representations_give_log_B():
    """phi = psi = one repeated row: every F_ij = 0, so InfoNCE = log B and the gradient is 0."""
    B = 72
    phi = np.tile(np.linspace(-1, 1, 64, dtype=np.float32), (B, 1))
    parts, gphi, gpsi = fused_l1(phi, phi.copy(), "sym", beta=0.0)
    assert abs(parts[1] - np.log(B)) <= 1e-6 * np.log(B)
    assert abs(parts[2] - np.log(B)) <= 1e-6 * np.log(B)
    assert not np.any(gphi) and not np.any(gpsi)


def test_fused_l1_is_deterministic():
    phi, psi = representations(520, 128, seed=11)
    a = fused_l1(phi, psi, "sym")
    b = fused_l1(phi, psi, "sym")
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_fused_l1_full_size_large_batch():
    """Batch 8192, repr 256 (the large-batch workload's shapes), InfoNCE forward
    direction with the row penalty; every output against the oracle."""
    phi, psi = representations(8192, 256, seed=5, scale=0.05)
    check(fused_l1(phi, psi, "fwd"), oracle_l1(phi, psi, "fwd"))


def test_fused_l1_gradients_sum_to_zero_at_full_size():
    """F depends on phi_i - psi_j only, so sum_i dL/dphi_i + sum_j dL/dpsi_j = 0 at
    any size (here the large-batch shapes with the symmetric loss and both penalty
    axes)."""
    phi, psi = representations(8192, 256, seed=9, scale=0.05)
    _, gphi, gpsi = fused_l1(phi, psi, "sym", penalty="both")
    s = gphi.astype(np.float64).sum(0) + gpsi.astype(np.float64).sum(0)
    assert np.abs(s).max() <= 1e-4 * np.abs(gphi).sum(0).max()


def test_fused_l1_rejects_misaligned_rows():
    """The tiles move rows in 16-byte pieces: a view starting 4 bytes in is refused."""
    dev = torch.device("cuda")
    base = torch.randn(16 * 64 + 1, device=dev)
    phi = base[1:].view(16, 64)
    with pytest.raises(api.CRLError) as e:
        functional.infonce_loss(phi, phi, "l1", "sym", "mean", "row", 1.0, 0.1, "fused")
    assert e.value.code == api.E_INVALID_ARG
