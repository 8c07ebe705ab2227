"""Pins for the oracle's MLPs, actor objective, Adam and full critic gradient.

Independent checks: torch's CPU fp64 library ops (linear, layer_norm, relu,
TanhTransform log-density, autograd, optim.Adam), the one-step Adam closed
form, and central finite differences (h = 1e-6, FP64) on 64 random parameter
coordinates, skipping coordinates whose +-h perturbation flips a ReLU.
"""

import numpy as np
import pytest
import torch

from oracle import actor, adam, critic, mlp, step
from paper_2408_11052_gb300 import workload


def small(layernorm, **kw):
    return workload.Workload("t", E=4, T=20, D=6, A=3, G=2, B=12, hidden=16, layers=2, repr=5,
                             layernorm=layernorm, seed=9, **kw)


def as64(net):
    return [{k: v.astype(np.float64) for k, v in layer.items()} for layer in net]


def torch_mlp(net, x):
    h = x
    for layer in net[:-1]:
        z = torch.nn.functional.linear(h, layer["W"], layer["b"])
        if "ln_g" in layer:
            z = torch.nn.functional.layer_norm(z, (z.shape[1],), layer["ln_g"], layer["ln_b"], eps=1e-6)
        h = torch.relu(z)
    return torch.nn.functional.linear(h, net[-1]["W"], net[-1]["b"])


def to_torch(net):
    return [{k: torch.tensor(v, requires_grad=True) for k, v in layer.items()} for layer in net]


@pytest.mark.parametrize("layernorm", [False, True])
def test_mlp_forward_backward_against_torch(layernorm):
    w = small(layernorm)
    net = as64(workload.init_network(w, "phi", 3, perturb=True))
    x = np.random.default_rng(0).standard_normal((w.B, w.D + w.A))
    out, cache = mlp.forward(net, x)
    tnet = to_torch(net)
    tx = torch.tensor(x, requires_grad=True)
    tout = torch_mlp(tnet, tx)
    np.testing.assert_allclose(out, tout.detach().numpy(), rtol=1e-12, atol=1e-13)
    dout = np.random.default_rng(1).standard_normal(out.shape)
    grads, dx = mlp.backward(net, cache, dout)
    tout.backward(torch.tensor(dout))
    np.testing.assert_allclose(dx, tx.grad.numpy(), rtol=1e-10, atol=1e-12)
    for layer, tl in zip(grads, tnet):
        assert set(layer) == set(tl)
        for k in layer:
            np.testing.assert_allclose(layer[k], tl[k].grad.numpy(), rtol=1e-10, atol=1e-12)


def test_policy_log_density_against_torch_distributions():
    rng = np.random.default_rng(2)
    B, A = 50, 4
    out = rng.standard_normal((B, 2 * A)) * 0.7
    out[:3, A:] = [-9.0, 5.0, 1.0, -4.99]           # clipped and unclipped log-stds
    out[3:6, :A] = 9.0                               # saturated tanh
    eps = rng.standard_normal((B, A))
    a_new, logpi, h = actor.policy_head(out, eps)
    mu = torch.tensor(out[:, :A])
    std = torch.tensor(np.exp(np.clip(out[:, A:], -5, 2)))
    dist = torch.distributions.TransformedDistribution(torch.distributions.Normal(mu, std),
                                                       [torch.distributions.transforms.TanhTransform()])
    ref = dist.log_prob(torch.tensor(a_new)).sum(dim=1).numpy()
    # torch recovers u = atanh(a), ill-conditioned once tanh saturates: compare unsaturated rows only
    ok = np.abs(h["u"]).max(axis=1) < 3.0
    assert ok.sum() > 20
    np.testing.assert_allclose(logpi[ok], ref[ok], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(a_new, np.tanh(h["u"]), rtol=0, atol=0)
    # every row against the density evaluated with 50 significant digits
    import mpmath
    mpmath.mp.dps = 50
    for i in range(B):
        tot = mpmath.mpf(0)
        for d in range(A):
            u = mpmath.mpf(h["u"][i, d])
            sd = mpmath.exp(mpmath.mpf(float(np.clip(out[i, A + d], -5, 2))))
            z = (u - mpmath.mpf(out[i, d])) / sd
            tot += -z * z / 2 - mpmath.log(sd) - mpmath.log(2 * mpmath.pi) / 2 - mpmath.log(1 - mpmath.tanh(u) ** 2)
        assert logpi[i] == pytest.approx(float(tot), rel=1e-11, abs=1e-11)


def test_adam_one_step_closed_form():
    g = np.array([1e-3, -2.0, 0.0, 5e-9, -7.5])
    p = np.arange(5.0)
    new_p, m, v = adam.adam_update(p, g, np.zeros(5), np.zeros(5), 1, lr=3e-4)
    # after one step from zero moments, m_hat = g and v_hat = g^2
    np.testing.assert_allclose(new_p, p - 3e-4 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)


def test_adam_matches_torch_optim_over_steps():
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(11)
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=6e-4, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(11), np.zeros(11)
    for t in range(1, 6):
        g = rng.standard_normal(11)
        p, m, v = adam.adam_update(p, g, m, v, t, lr=6e-4)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


def flat_coords(net, rng, n):
    keys = [(li, k, idx) for li, layer in enumerate(net) for k in layer for idx in np.ndindex(layer[k].shape)]
    pick = rng.choice(len(keys), size=min(n, len(keys)), replace=False)
    return [keys[i] for i in pick]


def relu_masks(net, x):
    _, cache = mlp.forward(net, x)
    return [c["u"] > 0 for c in cache[:-1]]


def fd_check(loss_fn, nets, grads, inputs_for_masks, rng, n=64, h=1e-6, rtol=2e-5, atol=1e-8):
    """Central FD on n random coordinates of each network in ``nets`` (dict name -> net)."""
    checked = 0
    for name, net in nets.items():
        for li, k, idx in flat_coords(net, rng, n):
            x0 = net[li][k][idx]
            net[li][k][idx] = x0 + h
            fp, mp = loss_fn(), [relu_masks(nn, inputs_for_masks[nm]()) for nm, nn in nets.items()]
            net[li][k][idx] = x0 - h
            fm, mm = loss_fn(), [relu_masks(nn, inputs_for_masks[nm]()) for nm, nn in nets.items()]
            net[li][k][idx] = x0
            if any((a != b).any() for A_, B_ in zip(mp, mm) for a, b in zip(A_, B_)):
                continue                                  # a ReLU kink lies within +-h
            fd = (fp - fm) / (2 * h)
            assert grads[name][li][k][idx] == pytest.approx(fd, rel=rtol, abs=atol), (name, li, k, idx)
            checked += 1
    assert checked >= 0.9 * n * len(nets)


@pytest.mark.parametrize("energy", ["l2", "dot", "cos"])
@pytest.mark.parametrize("loss", ["fwd", "bwd", "sym"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_critic_gradient_finite_differences(energy, loss, layernorm):
    w = small(layernorm)
    nets = {n: as64(workload.init_network(w, n, 20 + i, perturb=True)) for i, n in enumerate(("phi", "psi"))}
    rng = np.random.default_rng(30)
    s, a, g = rng.standard_normal((w.B, w.D)), rng.uniform(-1, 1, (w.B, w.A)), rng.standard_normal((w.B, w.G))
    kw = dict(energy=energy, tau=0.8, loss=loss, sym_reduction="mean", beta=0.1, penalty_axis="row")
    _, gphi, gpsi, _, _ = step.critic_loss_and_grad(nets["phi"], nets["psi"], s, a, g, **kw)

    def loss_fn():
        return step.critic_loss_and_grad(nets["phi"], nets["psi"], s, a, g, **kw)[0]["total"]

    inputs = {"phi": lambda: np.concatenate([s, a], axis=1), "psi": lambda: g}
    fd_check(loss_fn, nets, {"phi": gphi, "psi": gpsi}, inputs, rng)


@pytest.mark.parametrize("energy", ["l2", "dot", "cos"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_actor_gradient_finite_differences(energy, layernorm):
    w = small(layernorm)
    nets = {n: as64(workload.init_network(w, n, 40 + i, perturb=True)) for i, n in enumerate(("phi", "psi", "pi"))}
    rng = np.random.default_rng(50)
    s, g = rng.standard_normal((w.B, w.D)), rng.standard_normal((w.B, w.G))
    eps = rng.standard_normal((w.B, w.A))
    # push a few log-stds outside the clip range so both branches are exercised
    nets["pi"][-1]["b"][w.A:w.A + 1] = 3.0
    out = actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s, g, eps, energy, 0.8, 0.1)

    def loss_fn():
        return actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s, g, eps, energy, 0.8, 0.1)["loss"]

    def phi_in():
        o, _ = mlp.forward(nets["pi"], np.concatenate([s, g], axis=1))
        return np.concatenate([s, actor.policy_head(o, eps)[0]], axis=1)

    inputs = {"pi": lambda: np.concatenate([s, g], axis=1), "phi": phi_in}
    fd_check(loss_fn, {"pi": nets["pi"]}, {"pi": out["grads"]}, inputs, rng)


def test_actor_gradient_against_torch_autograd():
    w = small(True)
    nets = {n: as64(workload.init_network(w, n, 60 + i, perturb=True)) for i, n in enumerate(("phi", "psi", "pi"))}
    rng = np.random.default_rng(70)
    s, g, eps = rng.standard_normal((w.B, w.D)), rng.standard_normal((w.B, w.G)), rng.standard_normal((w.B, w.A))
    out = actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s, g, eps, "l2", 1.0, 0.2)
    tpi = to_torch(nets["pi"])
    tphi = [{k: torch.tensor(v) for k, v in l.items()} for l in nets["phi"]]
    tpsi = [{k: torch.tensor(v) for k, v in l.items()} for l in nets["psi"]]
    ts, tg, te = torch.tensor(s), torch.tensor(g), torch.tensor(eps)
    o = torch_mlp(tpi, torch.cat([ts, tg], 1))
    mu, ls = o[:, :w.A], torch.clamp(o[:, w.A:], -5, 2)
    dist = torch.distributions.TransformedDistribution(torch.distributions.Normal(mu, ls.exp()),
                                                       [torch.distributions.transforms.TanhTransform()])
    u = mu + ls.exp() * te
    a_new = torch.tanh(u)
    logpi = torch.distributions.Normal(mu, ls.exp()).log_prob(u).sum(1) - torch.log1p(-a_new ** 2).sum(1)
    f = -torch.linalg.vector_norm(torch_mlp(tphi, torch.cat([ts, a_new], 1)) - torch_mlp(tpsi, tg), dim=1)
    loss = (0.2 * logpi - f).mean()
    loss.backward()
    assert out["loss"] == pytest.approx(loss.item(), rel=1e-10)
    for layer, tl in zip(out["grads"], tpi):
        for k in layer:
            np.testing.assert_allclose(layer[k], tl[k].grad.numpy(), rtol=1e-7, atol=1e-10)
    del dist


def test_update_step_runs_and_orders_critic_before_actor():
    from oracle import relabel
    w = small(False)
    nets = {n: as64(workload.init_network(w, n, 80 + i)) for i, n in enumerate(("phi", "psi", "pi"))}
    buf = relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    obs, act, done = workload.buffer_contents(w, n=25, mean_len=6.0)
    buf.insert(obs, act, done)
    st = step.AgentState(nets["phi"], nets["psi"], nets["pi"])
    cfg = dict(seed=1, agent=0, B=w.B, goal_idx=(0, 1), gamma=0.99, energy="l2", tau=1.0, loss="sym",
               sym_reduction="mean", beta=0.1, penalty_axis="row", alpha=0.1, lr_critic=3e-4, lr_actor=6e-4)
    eps = workload.actor_noise(w.B, w.A, 5).astype(np.float64)
    out = step.update_step(st, buf, cfg, step=0, eps=eps)
    assert st.t_critic == 1 and st.t_actor == 1
    # the actor loss uses the updated critic
    s, a, g, idx = relabel.sample_relabel(buf, 1, 0, 0, w.B, (0, 1), 0.99)
    ref = actor.actor_loss_and_grad(nets["pi"], st.nets["phi"], st.nets["psi"], s, g, eps, "l2", 1.0, 0.1)
    assert out["actor_loss"] == pytest.approx(ref["loss"], rel=1e-14)
    np.testing.assert_array_equal(out["idx"], idx)
    assert np.isfinite(out["critic"]["total"])
    assert critic.infonce_loss  # module used above


def test_gaussian_noise_is_standard_normal():
    """Box-Muller draws from Philox: moments and a Kolmogorov-Smirnov test against N(0, 1)."""
    from scipy import stats
    eps = actor.gaussian_noise(3, 0, 5, 600, 7).ravel()
    assert abs(eps.mean()) < 5 / np.sqrt(eps.size)
    assert abs(eps.std() - 1.0) < 0.05
    assert stats.kstest(eps, "norm").pvalue > 1e-3
    again = actor.gaussian_noise(3, 0, 5, 4, 7)
    np.testing.assert_array_equal(again, eps.reshape(600, 7)[:4])
    assert (actor.gaussian_noise(3, 0, 6, 4, 7) != again).all()


# ---- entropy-coefficient auto-tuning (reading P5) -------------------------------

def test_alpha_first_adam_step_moves_log_alpha_by_lr_against_the_entropy_gap():
    """First Adam step: m_hat = g, v_hat = g^2, so log alpha moves by -lr sign(g)
    (up to eps): up when the policy's entropy -mean(log pi) is below the target
    H_target = -A, down when above."""
    from oracle.actor import alpha_loss_grad
    from oracle.adam import adam_update
    lr, A = 6e-4, 8
    for logpi_mean, expect_up in ((-2.0, False), (12.0, True)):   # entropy 2 > -8: down; entropy -12 < -8: up
        g = alpha_loss_grad(logpi_mean, -A)
        la, m, v = adam_update(np.log(0.1), g, 0.0, 0.0, 1, lr)
        step = float(la) - np.log(0.1)
        assert np.isclose(abs(step), lr, rtol=1e-6)
        assert (step > 0) == expect_up


def test_alpha_update_matches_torch_adam_on_the_scalar_loss():
    """Three steps of the oracle's log-alpha update against torch.optim.Adam minimising
    -log_alpha * (mean log pi + H_target) (log pi held fixed)."""
    import torch
    from oracle.actor import alpha_loss_grad
    from oracle.adam import adam_update
    H = -17.0
    logpis = [-3.0, -25.0, -10.5]
    la, m, v = np.log(0.1), 0.0, 0.0
    p = torch.tensor(np.log(0.1), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for t, lp in enumerate(logpis, start=1):
        la, m, v = adam_update(la, alpha_loss_grad(lp, H), m, v, t, 3e-3)
        opt.zero_grad()
        loss = -p * (lp + H)
        loss.backward()
        opt.step()
        assert np.isclose(float(la), p.item(), rtol=0, atol=1e-12)


def test_update_step_uses_alpha_before_its_update():
    """With auto-tuning the step's actor loss equals the actor loss at the pre-update
    alpha, and the returned next alpha is one Adam step on log alpha from it."""
    from paper_2408_11052_gb300 import workload
    from oracle.actor import actor_loss_and_grad, alpha_loss_grad, gaussian_noise
    from oracle.adam import adam_update
    from oracle.relabel import ReplayBuffer, sample_relabel
    from oracle.step import AgentState, update_step
    w = workload.SMALL_FP32.with_(E=4, T=30, B=8, hidden=16, repr=8)
    nets = {k: [{kk: vv.astype(np.float64) for kk, vv in l.items()} for l in v]
            for k, v in workload.init_agent(w).items()}
    obs, act, done = workload.buffer_contents(w, n=30, mean_len=6.0)
    buf = ReplayBuffer(w.E, w.T, w.D, w.A)
    buf.insert(obs, act, done)
    cfg = dict(seed=w.seed, agent=0, B=w.B, goal_idx=w.goals(), gamma=w.gamma, energy=w.energy, tau=w.tau,
               loss=w.loss, sym_reduction=w.sym_reduction, beta=w.beta, penalty_axis=w.penalty_axis, alpha=0.1,
               lr_critic=w.lr_critic, lr_actor=w.lr_actor, alpha_autotune=True, target_entropy=-float(w.A),
               lr_alpha=6e-4)
    state = AgentState(nets["phi"], nets["psi"], nets["pi"])
    alphas = []
    for step in range(2):
        eps = gaussian_noise(w.seed, 0, step, w.B, w.A)
        before = AgentState(state.nets["phi"], state.nets["psi"], state.nets["pi"])   # a deep copy
        out = update_step(state, buf, cfg, step, eps)
        alphas.append((out["alpha"], out["alpha_next"]))
        if step == 0:
            # the step's actor loss is the one at the initial alpha
            s, _, g, _ = sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
            ref = actor_loss_and_grad(before.nets["pi"], state.nets["phi"], state.nets["psi"], s, g, eps,
                                      w.energy, w.tau, 0.1)
            assert np.isclose(out["actor_loss"], ref["loss"], rtol=0, atol=1e-12)
            la_next, _, _ = adam_update(np.log(0.1), alpha_loss_grad(out["logpi_mean"], cfg["target_entropy"]),
                                        0.0, 0.0, 1, 6e-4)
            assert np.isclose(out["alpha"], 0.1)
            assert np.isclose(np.log(out["alpha_next"]), float(la_next), rtol=0, atol=1e-12)
    assert np.isclose(alphas[1][0], alphas[0][1])          # step 2 uses the alpha step 1 produced
    assert alphas[0][1] != alphas[0][0]
