"""The BF16 tensor-core path behind torch.autograd.Function: the encoders on the
tcgen05 GEMMs (functional.encoder(..., precision="bf16")) and the fused energy +
InfoNCE + logsumexp-penalty kernels (functional.infonce_loss(..., path="fused")),
against the FP64 oracle at the BF16 bars: loss relative error <= 2e-2 and
gradient cosine >= 0.999 per parameter tensor.  Batches 8, 136 and 520 are ragged
against the 128-row tiles; batch 8192 with repr 256 is the large-batch workload
(its 268 MB B x B matrix is never written)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, functional, workload

from parity_helpers import hp, setup

pytestmark = pytest.mark.gpu

BF16_LOSS_RTOL = 2e-2
BF16_GRAD_COS = 0.999


def cosine(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def autograd_critic(ctx, w, s, a, g, precision="bf16", path="fused"):
    """Critic loss through the autograd wrappers; returns (loss, parts, phi grads, psi grads) (flat)."""
    pp = ctx.store["phi"]["params"].clone().requires_grad_(True)
    pq = ctx.store["psi"]["params"].clone().requires_grad_(True)
    phi = functional.encoder(pp, s, a, w.D, w.A, w.hidden, w.layers, w.repr, w.layernorm, precision=precision)
    psi = functional.encoder(pq, g, None, w.G, 0, w.hidden, w.layers, w.repr, w.layernorm, precision=precision)
    total, parts = functional.infonce_loss(phi, psi, w.energy, w.loss, w.sym_reduction, w.penalty_axis,
                                           float(np.float32(w.tau)), float(np.float32(w.beta)), path)
    total.backward()
    torch.cuda.synchronize()
    return total.item(), parts.cpu().numpy(), pp.grad, pq.grad


def check_against_oracle(ctx, w, buf, nets, step, loss, parts, gp, gq):
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref, gphi, gpsi, _, _ = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o, w.energy,
                                                             h["tau"], w.loss, w.sym_reduction, h["beta"],
                                                             w.penalty_axis)
    assert abs(loss - ref["total"]) <= BF16_LOSS_RTOL * abs(ref["total"])
    for i, k in enumerate(("total", "fwd", "bwd", "penalty")):
        assert abs(parts[i] - ref[k]) <= BF16_LOSS_RTOL * abs(ref[k]), k
    worst = 1.0
    for net, flat, gref in (("phi", gp, gphi), ("psi", gq, gpsi)):
        for t in ctx.layout[net]:
            n = t["rows"] * t["cols"]
            got = flat[t["offset"]:t["offset"] + n].double().cpu().numpy()
            c = cosine(got, gref[t["layer"]][t["kind"]])
            worst = min(worst, c)
            assert c >= BF16_GRAD_COS, (net, t["layer"], t["kind"], c)
    return worst


@pytest.mark.parametrize("B,R,energy,loss", [(8, 64, "l2", "sym"), (136, 128, "dot", "fwd"),
                                             (520, 64, "cos", "bwd"), (136, 192, "l2sq", "sym"),
                                             (264, 64, "l2", "dpo"), (136, 64, "l2", "nce_binary")])
def test_bf16_autograd_critic_matches_oracle(B, R, energy, loss):
    w = workload.Workload("ag", E=6, T=48, D=29, A=8, G=2, B=B, hidden=96, layers=2, repr=R, energy=energy,
                          loss=loss, tau=0.7 if energy == "cos" else 1.0, seed=41)
    ctx, nets, buf = setup(w, precision="fp32", n=70)
    s, a, g, _ = ctx.sample(step=3)
    check_against_oracle(ctx, w, buf, nets, 3, *autograd_critic(ctx, w, s, a, g))


def test_bf16_autograd_layernorm_humanoid_shapes():
    """4 x 1024 LayerNorm encoders, batch 1024, obs 268 / action 17 / goal 3, cos energy."""
    w = workload.HUMANOID_BF16
    ctx, nets, buf = setup(w, precision="fp32", mean_len=None)
    s, a, g, _ = ctx.sample(step=4)
    check_against_oracle(ctx, w, buf, nets, 4, *autograd_critic(ctx, w, s, a, g))


def test_bf16_autograd_large_batch():
    """Batch 8192, repr 256, 2 x 512 encoders, L2 energy, forward InfoNCE."""
    w = workload.LARGE_BATCH
    ctx, nets, buf = setup(w, precision="fp32", n=40, mean_len=None)
    s, a, g, _ = ctx.sample(step=4)
    check_against_oracle(ctx, w, buf, nets, 4, *autograd_critic(ctx, w, s, a, g))


def test_bf16_autograd_input_gradients_and_two_forwards_before_backward():
    """Each forward keeps its own workspace: two encoder forwards of the same shape
    before either backward give the same gradients as one forward-backward each,
    and the input gradients (x0 and x1) match the FP32 path's within the BF16 bar."""
    dev = torch.device("cuda")
    w = workload.Workload("ag2", E=1, T=1, D=29, A=8, G=2, B=136, hidden=128, layers=2, repr=64, seed=43)
    cnt, _ = api.param_layout(api.make_config(w), "phi")
    torch.manual_seed(1)
    params = (torch.randn(cnt, device=dev) * 0.1).requires_grad_(True)
    xs = [torch.randn(136, 29, device=dev, requires_grad=True) for _ in range(2)]
    xa = [torch.randn(136, 8, device=dev, requires_grad=True) for _ in range(2)]
    dys = [torch.randn(136, 64, device=dev) for _ in range(2)]
    # two forwards, then both backwards
    ys = [functional.encoder(params, xs[i], xa[i], 29, 8, 128, 2, 64, precision="bf16") for i in range(2)]
    (ys[0] * dys[0]).sum().backward(retain_graph=True)
    g_first = [params.grad.clone(), xs[0].grad.clone(), xa[0].grad.clone()]
    params.grad = None
    (ys[1] * dys[1]).sum().backward()
    g_second = [params.grad.clone(), xs[1].grad.clone(), xa[1].grad.clone()]
    for i, want in ((0, g_first), (1, g_second)):
        params.grad = None
        x0 = xs[i].detach().clone().requires_grad_(True)
        x1 = xa[i].detach().clone().requires_grad_(True)
        y = functional.encoder(params, x0, x1, 29, 8, 128, 2, 64, precision="bf16")
        (y * dys[i]).sum().backward()
        for got, ref in zip((params.grad, x0.grad, x1.grad), want):
            torch.testing.assert_close(got, ref, rtol=0, atol=0)
        # the FP32 plain kernels on the same inputs
        params32 = params.detach().clone().requires_grad_(True)
        x0f = xs[i].detach().clone().requires_grad_(True)
        x1f = xa[i].detach().clone().requires_grad_(True)
        (functional.encoder(params32, x0f, x1f, 29, 8, 128, 2, 64) * dys[i]).sum().backward()
        for got, ref in ((params.grad, params32.grad), (x0.grad, x0f.grad), (x1.grad, x1f.grad)):
            assert cosine(got.cpu().numpy(), ref.cpu().numpy()) >= BF16_GRAD_COS


def test_bf16_fused_op_rejects_what_it_does_not_take():
    dev = torch.device("cuda")
    phi = torch.randn(12, 64, device=dev, requires_grad=True)       # B not a multiple of 8
    with pytest.raises(api.CRLError) as e:
        functional.infonce_loss(phi, phi, "l2", "sym", "mean", "row", 1.0, 0.1, "fused")
    assert e.value.code == api.E_UNSUPPORTED
    phi = torch.randn(16, 48, device=dev, requires_grad=True)       # repr not in {64, 128, 192, 256}
    with pytest.raises(api.CRLError) as e:
        functional.infonce_loss(phi, phi, "l2", "sym", "mean", "row", 1.0, 0.1, "fused")
    assert e.value.code == api.E_UNSUPPORTED
    phi = torch.randn(16, 64, device=dev, dtype=torch.float64, requires_grad=True)
    with pytest.raises(TypeError):
        functional.infonce_loss(phi, phi, "l2", "sym", "mean", "row", 1.0, 0.1, "fused")
