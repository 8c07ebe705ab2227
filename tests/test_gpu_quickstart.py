"""The user-facing quick start: a BF16 fused context on the Ant workload, the
collection stub filling the buffer, update steps, and a checkpoint that a fresh
context resumes from."""

import math

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

pytestmark = pytest.mark.gpu


def test_quick_start_runs_and_resumes():
    w = workload.ANT_AUTOGRAD
    ctx = api.CRLContext(w, precision="bf16", path="fused")
    nets = workload.init_agent(w)
    for net, layers in nets.items():
        ctx.load_network(net, layers)
    ctx.collect(1000, episode_length=1000)
    assert ctx.buffer_size() == (w.T, w.T)
    loss = torch.zeros(6, device="cuda")
    for _ in range(3):
        ctx.update_step(loss_out=loss)
    torch.cuda.synchronize()
    parts = loss.cpu().numpy()
    assert np.all(np.isfinite(parts)) and parts[0] > 0.0
    assert ctx.sync_status() == (0, 0)
    state = ctx.save_state()
    saved = {n: {k: ctx.store[n][k].clone() for k in ("params", "grads", "adam_m", "adam_v")}
             for n in ("phi", "psi", "pi")}
    ctx.update_step(loss_out=loss)
    want = loss.cpu().numpy().copy()
    b = api.CRLContext(w, precision="bf16", path="fused")
    for n, d in saved.items():
        for k, v in d.items():
            b.store[n][k].copy_(v)
    b.load_state(state)
    b.update_step(loss_out=loss)
    np.testing.assert_array_equal(loss.cpu().numpy(), want)
    assert not math.isnan(b.get_alpha())


def test_quick_start_autograd_critic_loss():
    """The quick start's autograd lines: the fused critic loss on BF16 kernels
    behind torch.autograd, at batch 8192 and repr 256, gives finite gradients of
    the representations' shapes, and the autotuner report of a context lists
    its problem lists."""
    from paper_2408_11052_gb300 import functional
    torch.manual_seed(0)
    phi = torch.randn(8192, 256, device="cuda", requires_grad=True)
    psi = torch.randn(8192, 256, device="cuda", requires_grad=True)
    total, parts = functional.infonce_loss(phi, psi, energy="l2", loss="fwd", path="fused")
    total.backward()
    torch.cuda.synchronize()
    assert math.isfinite(total.detach().item()) and parts[1].item() > 0.0
    assert phi.grad.shape == phi.shape and psi.grad.shape == psi.shape
    assert torch.isfinite(phi.grad).all() and torch.isfinite(psi.grad).all()
    # the L2 energy depends on phi_i - psi_j only, so shifting every row of both
    # by one vector leaves the loss unchanged: sum_i dphi_i + sum_j dpsi_j = 0,
    # here up to the BF16 rounding of the coefficient tiles
    net = (phi.grad.sum(0) + psi.grad.sum(0)).abs()
    scale = phi.grad.abs().sum(0) + psi.grad.abs().sum(0)
    assert bool((net <= 1e-2 * scale).all())
