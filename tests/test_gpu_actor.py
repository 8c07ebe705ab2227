"""GPU parity of the actor step (tanh-Gaussian policy, DDPG-style objective with entropy,
backward through phi to the action, Adam) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import workload

from parity_helpers import (FP32_GRAD_RTOL, FP32_LOSS_RTOL, FP64_GRAD_RTOL, FP64_LOSS_RTOL, assert_grads_close,
                            assert_scalar_close, hp, pick_step, setup, small)

pytestmark = pytest.mark.gpu

TOL = {"fp32": (FP32_LOSS_RTOL, FP32_GRAD_RTOL), "fp64": (FP64_LOSS_RTOL, FP64_GRAD_RTOL)}


def run_actor(w, precision, start=5, eps_seed=3, nets=None, n=70, mean_len=9.0):
    raw = workload.init_agent(w, perturb=True) if nets is None else nets
    # push one log-std outside the clip range so both branches run
    raw["pi"][-1]["b"][w.A] = np.float32(3.0)
    ctx, nets, buf = setup(w, precision=precision, n=n, mean_len=mean_len, nets=raw)
    eps = workload.actor_noise(w.B, w.A, eps_seed)
    step = pick_step(w, nets, buf, start, eps=eps.astype(np.float64))
    s, a, g, _ = ctx.sample(step=step)
    out = ctx.actor_step(s, g, torch.from_numpy(eps).to(ctx.device), apply_update=False)
    torch.cuda.synchronize()
    s_o, _, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s_o, g_o, eps.astype(np.float64),
                                           w.energy, h["tau"], h["alpha"])
    return ctx, nets, out.cpu().numpy(), ref


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_actor_step_matches_oracle(precision, energy, layernorm):
    w = small(energy=energy, layernorm=layernorm, tau=0.8)
    ctx, _, got, ref = run_actor(w, precision)
    lt, gt = TOL[precision]
    assert_scalar_close(got[0], ref["loss"], lt, "actor loss", atol=1e-7)
    assert_scalar_close(got[1], ref["logpi_mean"], lt, "mean log pi", atol=1e-7)
    assert_grads_close(ctx.network("pi", "grads"), ref["grads"], gt, "pi")
    assert ctx.sync_status() == (0, 0)


def test_actor_full_size_humanoid_config():
    """Batch 1024, 4 x 1024 LayerNorm MLPs, obs 268, action 17, cosine energy (LayerNorm
    shifts raised by 4 to keep every unit off its kink, as in the critic test)."""
    w = workload.HUMANOID_BF16
    nets = workload.init_agent(w, perturb=True)
    for net in ("phi", "psi", "pi"):
        for layer in nets[net][:-1]:
            layer["ln_b"] = layer["ln_b"] + np.float32(4.0)
    ctx, _, got, ref = run_actor(w, "fp32", nets=nets, mean_len=None)
    assert_scalar_close(got[0], ref["loss"], FP32_LOSS_RTOL, "actor loss", atol=1e-7)
    assert_grads_close(ctx.network("pi", "grads"), ref["grads"], FP32_GRAD_RTOL, "pi")


def test_actor_does_not_touch_critic():
    w = small()
    ctx, nets, _, _ = run_actor(w, "fp32")
    before = {n: ctx.store[n]["params"].clone() for n in ("phi", "psi")}
    s, a, g, _ = ctx.sample(step=9)
    ctx.actor_step(s, g, None, apply_update=True)
    torch.cuda.synchronize()
    for n in ("phi", "psi"):
        assert torch.equal(before[n], ctx.store[n]["params"])


def test_actor_philox_noise_matches_oracle_noise():
    """eps = NULL draws Box-Muller noise from Philox at the step of the last sample."""
    w = small(B=40)
    ctx, nets, buf = setup(w, precision="fp64", n=50)
    step = None
    for cand in range(17, 17 + 64):
        eps = oracle.actor.gaussian_noise(w.seed, 0, cand, w.B, w.A)
        try:
            step = pick_step(w, nets, buf, cand, eps=eps, tries=1)
            break
        except AssertionError:
            continue
    assert step is not None
    s, a, g, _ = ctx.sample(step=step)
    out = ctx.actor_step(s, g, None, apply_update=False)
    torch.cuda.synchronize()
    eps = oracle.actor.gaussian_noise(w.seed, 0, step, w.B, w.A)
    s_o, _, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s_o, g_o, eps, w.energy, h["tau"],
                                           h["alpha"])
    assert_scalar_close(out[0].item(), ref["loss"], FP64_LOSS_RTOL, "actor loss", atol=1e-7)
    assert_grads_close(ctx.network("pi", "grads"), ref["grads"], 1e-8, "pi")
