"""FP64 GPU check path: the hand-written critic gradient against central finite
differences (h = 1e-6, FP64) on 64 random parameter coordinates, Ant-shaped
(obs 29, goal 2, action 8, batch 256, 2 x 256 MLPs, repr 64), dot and L2 energy,
forward / backward / symmetric InfoNCE; and the autograd.Function wrappers."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import functional, workload

from parity_helpers import pick_step, setup

pytestmark = pytest.mark.gpu


def fd_loss_fn(ctx, w, s, a, g, penalty_axis="row"):
    """Critic loss in FP64 on the GPU through the op-level kernels (autograd.Function forward)."""
    def loss():
        pp, pq = ctx.store["phi"]["params"], ctx.store["psi"]["params"]
        phi = functional.encoder(pp, s, a, w.D, w.A, w.hidden, w.layers, w.repr, w.layernorm)
        psi = functional.encoder(pq, g, None, w.G, 0, w.hidden, w.layers, w.repr, w.layernorm)
        total, _ = functional.infonce_loss(phi, psi, w.energy, w.loss, w.sym_reduction, penalty_axis, w.tau, w.beta)
        return total.item()
    return loss


@pytest.mark.parametrize("energy,loss", [(e, l) for e in ("dot", "l2", "l1") for l in ("fwd", "bwd", "sym")] +
                         [("l2", l) for l in ("fb", "dpo", "ipo", "sppo", "nce_binary")] + [("dot", "dpo")])
def test_fp64_gradient_against_central_differences(energy, loss):
    w = workload.ANT_AUTOGRAD.with_(energy=energy, loss=loss)
    ctx, _, _ = setup(w, precision="fp64", n=60)
    s, a, g, _ = ctx.sample(step=2)
    ctx.critic_step(s, a, g, apply_update=False)
    grads = {n: ctx.store[n]["grads"].cpu().numpy() for n in ("phi", "psi")}
    f = fd_loss_fn(ctx, w, s, a, g)
    L0 = f()
    rng = np.random.default_rng(7)
    h = 1e-6
    checked = 0
    for net in ("phi", "psi"):
        p = ctx.store[net]["params"]
        live = [t for t in ctx.layout[net]]
        coords = []
        for t in live:
            n = t["rows"] * t["cols"]
            coords += [t["offset"] + i for i in range(n)]
        for idx in rng.choice(coords, size=64, replace=False):
            x0 = p[idx].item()
            vals = []
            for step in (h, h / 2):
                p[idx] = x0 + step
                fp = f()
                p[idx] = x0 - step
                fm = f()
                vals.append((fp - fm) / (2 * step))
            p[idx] = x0
            # roundoff of a central difference of an FP64 loss L: about 2 eps |L| / h
            atol = 4 * np.finfo(np.float64).eps * max(abs(L0), 1.0) / (h / 2)
            if abs(vals[0] - vals[1]) > 1e-5 * abs(grads[net][idx]) + 2 * atol:
                continue                                  # a ReLU kink within +-h
            assert grads[net][idx] == pytest.approx(vals[0], rel=1e-5, abs=atol), (net, idx)
            checked += 1
    assert checked >= 0.9 * 128


def test_autograd_functions_gradcheck_fp64():
    torch.manual_seed(0)
    dev = torch.device("cuda")
    w = workload.Workload("gc", E=1, T=1, D=4, A=2, G=2, B=5, hidden=6, layers=2, repr=3, layernorm=True, seed=1)
    n = sum(int(np.prod(v.shape)) for layer in workload.init_network(w, "phi", 0) for v in layer.values())
    from paper_2408_11052_gb300 import api
    cnt, _ = api.param_layout(api.make_config(w), "phi")
    params = torch.randn(cnt, dtype=torch.float64, device=dev, requires_grad=True)
    x0 = torch.randn(5, 4, device=dev)
    x1 = torch.randn(5, 2, device=dev)
    fn = lambda p: functional.encoder(p, x0, x1, 4, 2, 6, 2, 3, True)
    assert torch.autograd.gradcheck(fn, (params,), eps=1e-6, atol=1e-7, rtol=1e-5)
    assert n <= cnt
    phi = torch.randn(6, 3, dtype=torch.float64, device=dev, requires_grad=True)
    psi = torch.randn(6, 3, dtype=torch.float64, device=dev, requires_grad=True)
    for energy in ("l2", "dot", "cos", "l2sq"):
        for loss in ("fwd", "bwd", "sym"):
            fl = lambda a, b: functional.infonce_loss(a, b, energy, loss, "mean", "both", 0.9, 0.1)[0]
            assert torch.autograd.gradcheck(fl, (phi, psi), eps=1e-6, atol=1e-8, rtol=1e-6)
    # the other objectives (FlatNCE has the constant value 0, so finite differences do not see its gradient)
    for energy in ("l2", "dot"):
        for loss in ("fb", "dpo", "ipo", "sppo", "nce_binary"):
            fl = lambda a, b: functional.infonce_loss(a, b, energy, loss, "mean", "row", 0.9, 0.1)[0]
            assert torch.autograd.gradcheck(fl, (phi, psi), eps=1e-6, atol=1e-8, rtol=1e-6), (energy, loss)


def test_autograd_functions_fp32_match_oracle():
    w = workload.ANT_AUTOGRAD
    ctx, nets, buf = setup(w, precision="fp32", n=60)
    step = pick_step(w, nets, buf, 4)
    s, a, g, _ = ctx.sample(step=step)
    pp = ctx.store["phi"]["params"].clone().requires_grad_(True)
    pq = ctx.store["psi"]["params"].clone().requires_grad_(True)
    phi = functional.encoder(pp, s, a, w.D, w.A, w.hidden, w.layers, w.repr)
    psi = functional.encoder(pq, g, None, w.G, 0, w.hidden, w.layers, w.repr)
    total, parts = functional.infonce_loss(phi, psi)
    total.backward()
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    ref, gphi, gpsi, _, _ = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o)
    assert total.item() == pytest.approx(ref["total"], rel=1e-5)
    for net, flat, gref in (("phi", pp.grad, gphi), ("psi", pq.grad, gpsi)):
        for t in ctx.layout[net]:
            n = t["rows"] * t["cols"]
            got = flat[t["offset"]:t["offset"] + n].double().cpu().numpy()
            want = gref[t["layer"]][t["kind"]].ravel()
            assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want), (net, t)
