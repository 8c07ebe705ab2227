"""GPU parity of the critic step (encoders, energy, InfoNCE + penalty, backward, Adam)
against the FP64 oracle, through crl_critic_step."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

from parity_helpers import (FP32_GRAD_RTOL, FP32_LOSS_RTOL, FP64_GRAD_RTOL, FP64_LOSS_RTOL, assert_grads_close,
                            assert_scalar_close, hp, pick_step, setup, small)

pytestmark = pytest.mark.gpu

TOL = {"fp32": (FP32_LOSS_RTOL, FP32_GRAD_RTOL), "fp64": (FP64_LOSS_RTOL, FP64_GRAD_RTOL)}


def run_critic(w, precision, start=4, nets=None, penalty_axis=None, n=70, mean_len=9.0, perturb=True):
    kw = {} if penalty_axis is None else {"penalty_axis": penalty_axis}
    ctx, nets, buf = setup(w, precision=precision, n=n, mean_len=mean_len, perturb=perturb, nets=nets, **kw)
    step = pick_step(w, nets, buf, start)
    s, a, g, _ = ctx.sample(step=step)
    loss = ctx.critic_step(s, a, g, apply_update=False)
    torch.cuda.synchronize()
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o, w.energy, h["tau"], w.loss,
                                           w.sym_reduction, h["beta"], penalty_axis or w.penalty_axis)
    return ctx, nets, (s, a, g), loss.cpu().numpy(), ref


def check(ctx, got, ref, precision):
    parts, gphi, gpsi, _, _ = ref
    lt, gt = TOL[precision]
    for i, k in enumerate(("total", "fwd", "bwd", "penalty")):
        assert_scalar_close(got[i], parts[k], lt, k, atol=1e-7 if k == "penalty" else 0.0)
    assert_grads_close(ctx.network("phi", "grads"), gphi, gt, "phi")
    assert_grads_close(ctx.network("psi", "grads"), gpsi, gt, "psi")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
@pytest.mark.parametrize("loss", ["fwd", "bwd", "sym"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_critic_step_matches_oracle(precision, energy, loss, layernorm):
    w = small(energy=energy, loss=loss, layernorm=layernorm, tau=0.7 if energy == "cos" else 1.0)
    ctx, _, _, got, ref = run_critic(w, precision)
    check(ctx, got, ref, precision)
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("sym_reduction,penalty_axis", [("sum", "row"), ("mean", "col"), ("mean", "both")])
def test_critic_reductions_and_penalty_axes(sym_reduction, penalty_axis):
    w = small(sym_reduction=sym_reduction)
    ctx, _, _, got, ref = run_critic(w, "fp32", penalty_axis=penalty_axis)
    check(ctx, got, ref, "fp32")


@pytest.mark.parametrize("B", [1, 2, 63, 65, 129])
def test_critic_ragged_and_degenerate_batches(B):
    w = small(B=B, hidden=33, repr=5)
    ctx, _, _, got, ref = run_critic(w, "fp32")
    if B == 1:
        assert ref[0]["contrastive"] == 0.0       # one sample: the softmax over one entry is 1
    check(ctx, got, ref, "fp32")


OBJECTIVES = ["flatnce_fwd", "flatnce_bwd", "fb", "dpo", "ipo", "sppo", "nce_binary"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("energy", ["l2", "dot"])
@pytest.mark.parametrize("loss", OBJECTIVES)
def test_critic_objectives_match_oracle(precision, energy, loss):
    """The other objectives of App. A.2 / §5.2 with the logsumexp penalty."""
    w = small(energy=energy, loss=loss)
    ctx, _, _, got, ref = run_critic(w, precision)
    check(ctx, got, ref, precision)
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("B,loss", [(2, "fb"), (65, "dpo"), (129, "ipo"), (63, "sppo"), (1, "nce_binary"),
                                    (1, "dpo"), (3, "flatnce_bwd")])
def test_critic_objectives_ragged_and_degenerate_batches(B, loss):
    w = small(B=B, hidden=33, repr=5, loss=loss)
    ctx, _, _, got, ref = run_critic(w, "fp32")
    check(ctx, got, ref, "fp32")


def test_forward_backward_objective_needs_two_samples():
    w = small(B=4, loss="fb")
    ctx, _, _ = setup(w, n=40)
    s, a, g, _ = ctx.sample(step=0)
    with pytest.raises(api.CRLError) as e:
        ctx.critic_step(s[:1], a[:1], g[:1])
    assert e.value.code == api.E_SHAPE


@pytest.mark.parametrize("direction", ["fwd", "bwd"])
def test_flatnce_gradient_is_infonce_gradient_on_gpu(direction):
    """Reading C8: FlatNCE's gradient is InfoNCE's of the same direction (the same
    coefficients, so bit for bit), and its value is 0: total = penalty."""
    out = {}
    for loss in (direction, "flatnce_" + direction):
        w = small(loss=loss)
        ctx, _, _, got, _ = run_critic(w, "fp32")
        out[loss] = (got, {n: ctx.store[n]["grads"].cpu().numpy() for n in ("phi", "psi")})
    a, b = out[direction], out["flatnce_" + direction]
    for n in ("phi", "psi"):
        np.testing.assert_array_equal(a[1][n], b[1][n])
    assert b[0][0] == b[0][3] and b[0][3] == a[0][3]
    np.testing.assert_array_equal(a[0][1:], b[0][1:])


def test_equal_representations_give_log_B_on_gpu():
    """All-zero output weights make phi = psi = const for every sample: InfoNCE = log B."""
    w = small(B=128)
    ctx, _, _ = setup(w, n=60)
    for net in ("phi", "psi"):
        ctx.views(net)[-1]["W"].zero_()
        ctx.views(net)[-1]["b"].fill_(0.25)
    s, a, g, _ = ctx.sample(step=1)
    loss = ctx.critic_step(s, a, g).cpu().numpy()
    assert loss[1] == pytest.approx(np.log(128), rel=1e-6)
    assert loss[2] == pytest.approx(np.log(128), rel=1e-6)
    assert loss[3] == pytest.approx(0.1 * np.log(128) ** 2, rel=1e-6)


def test_critic_adam_update_matches_oracle():
    w = small()
    ctx, nets, (s, a, g), _, _ = run_critic(w, "fp64")
    ctx.critic_step(s, a, g, apply_update=True)
    ctx.critic_step(s, a, g, apply_update=True)
    torch.cuda.synchronize()
    h = hp(w)
    state = oracle.step.AgentState(nets["phi"], nets["psi"], nets["pi"])
    s_o, a_o, g_o = (x.cpu().numpy() for x in (s, a, g))
    for t in (1, 2):
        _, gp, gq, _, _ = oracle.step.critic_loss_and_grad(state.nets["phi"], state.nets["psi"], s_o, a_o, g_o,
                                                           w.energy, h["tau"], w.loss, w.sym_reduction, h["beta"],
                                                           "row")
        for name, gr in (("phi", gp), ("psi", gq)):
            state.nets[name], state.m[name], state.v[name] = oracle.step.adam_net(
                state.nets[name], gr, state.m[name], state.v[name], t, h["lr_critic"], h["adam_beta1"],
                h["adam_beta2"], h["adam_eps"])
    for name in ("phi", "psi"):
        for gl, rl in zip(ctx.network(name), state.nets[name]):
            for k in rl:
                np.testing.assert_allclose(gl[k], rl[k], rtol=1e-10, atol=1e-13)


def test_critic_full_size_ant_config():
    """Batch 256, 2 x 256 MLPs, repr 64, L2 + symmetric InfoNCE (the bench's launch)."""
    w = workload.ANT_AUTOGRAD
    ctx, _, _, got, ref = run_critic(w, "fp32", mean_len=None)
    check(ctx, got, ref, "fp32")


def test_critic_full_size_humanoid_config():
    """Batch 1024, 4 x 1024 MLPs with LayerNorm, obs 268, cosine energy.

    With 8.4M hidden units no batch is free of pre-activations near zero, so the
    LayerNorm shifts are raised by 4 (every unit sits >= ~4 sigma from its kink);
    the small-size tests cover the masked case.
    """
    w = workload.HUMANOID_BF16
    nets = workload.init_agent(w, perturb=True)
    for net in ("phi", "psi"):
        for layer in nets[net][:-1]:
            layer["ln_b"] = layer["ln_b"] + np.float32(4.0)
    ctx, _, _, got, ref = run_critic(w, "fp32", nets=nets, mean_len=None)
    check(ctx, got, ref, "fp32")
