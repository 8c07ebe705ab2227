"""One CRL update step (the body of the update loop of Algorithm 1, App. F).

Test infrastructure only (see ``oracle/__init__``).

Order (Algorithm 1): sample a relabelled batch with discount, update the
critic (phi, psi) on L_critic + beta * L_logsumexp, then update the policy on
L_actor with the critic as just updated.
"""

import copy

import numpy as np

from . import actor, adam, critic, mlp, relabel


def critic_loss_and_grad(phi_net, psi_net, s, a, g, energy="l2", tau=1.0, loss="sym",
                         sym_reduction="mean", beta=0.1, penalty_axis="row"):
    """Critic loss parts and gradients (§3.1 critic objective, App. A.2, Algorithm 1).

    Returns (parts, grads_phi, grads_psi, phi [B][R], psi [B][R]).
    """
    x = np.concatenate([np.asarray(s, dtype=np.float64), np.asarray(a, dtype=np.float64)], axis=1)
    phi, cphi = mlp.forward(phi_net, x)
    psi, cpsi = mlp.forward(psi_net, np.asarray(g, dtype=np.float64))
    F = critic.energy_matrix(phi, psi, energy, tau)
    parts = critic.critic_loss(F, loss, sym_reduction, beta, penalty_axis)
    G = critic.critic_grad_F(F, loss, sym_reduction, beta, penalty_axis)
    dphi, dpsi = critic.energy_backward(phi, psi, G, energy, tau)
    gphi, _ = mlp.backward(phi_net, cphi, dphi)
    gpsi, _ = mlp.backward(psi_net, cpsi, dpsi)
    return parts, gphi, gpsi, phi, psi


def zeros_like_net(net):
    return [{k: np.zeros_like(v, dtype=np.float64) for k, v in layer.items()} for layer in net]


def adam_net(net, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Apply ``adam.adam_update`` to every tensor of a network; returns new (net, m, v)."""
    new_net, new_m, new_v = [], [], []
    for layer, gl, ml, vl in zip(net, grads, m, v):
        nl, nm, nv = {}, {}, {}
        for k in layer:
            nl[k], nm[k], nv[k] = adam.adam_update(layer[k], gl[k], ml[k], vl[k], t, lr, beta1, beta2, eps)
        new_net.append(nl)
        new_m.append(nm)
        new_v.append(nv)
    return new_net, new_m, new_v


class AgentState:
    """Parameters and Adam moments of phi, psi and pi, plus the Adam step counters."""

    def __init__(self, phi_net, psi_net, pi_net):
        self.nets = {"phi": copy.deepcopy(phi_net), "psi": copy.deepcopy(psi_net),
                     "pi": copy.deepcopy(pi_net)}
        self.m = {k: zeros_like_net(n) for k, n in self.nets.items()}
        self.v = {k: zeros_like_net(n) for k, n in self.nets.items()}
        self.t_critic = 0
        self.t_actor = 0
        # entropy-coefficient auto-tuning (reading P5): log alpha and its Adam moments,
        # initialised from cfg["alpha"] on the first tuned step
        self.log_alpha = None
        self.m_alpha = 0.0
        self.v_alpha = 0.0


def update_step(state, buf, cfg, step, eps):
    """One full update step in place on ``state``; returns a dict of loss parts.

    cfg keys: seed, agent, B, goal_idx, gamma, offset_min, energy, tau, loss,
    sym_reduction, beta, penalty_axis, alpha, lr_critic, lr_actor, and optionally
    adam_beta1, adam_beta2, adam_eps (textbook defaults) and alpha_autotune,
    target_entropy, lr_alpha (reading P5 of the actor module; the returned dict
    then carries the alpha used and the updated one) and alpha_rg (the
    random-goal actor mix, reading P6; 0 by default).
    eps [B][A]: the actor's Gaussian noise, drawn by the caller.
    """
    s, a, g, idx = relabel.sample_relabel(buf, cfg["seed"], cfg.get("agent", 0), step, cfg["B"],
                                          cfg["goal_idx"], cfg["gamma"], cfg.get("offset_min", 1))
    parts, gphi, gpsi, _, _ = critic_loss_and_grad(
        state.nets["phi"], state.nets["psi"], s, a, g, cfg["energy"], cfg["tau"], cfg["loss"],
        cfg["sym_reduction"], cfg["beta"], cfg["penalty_axis"])
    betas = (cfg.get("adam_beta1", 0.9), cfg.get("adam_beta2", 0.999), cfg.get("adam_eps", 1e-8))
    state.t_critic += 1
    for name, grads in (("phi", gphi), ("psi", gpsi)):
        state.nets[name], state.m[name], state.v[name] = adam_net(
            state.nets[name], grads, state.m[name], state.v[name], state.t_critic, cfg["lr_critic"], *betas)
    g_actor = g
    if cfg.get("alpha_rg", 0.0) > 0.0:
        g_actor, _ = relabel.actor_goal_mix(cfg["seed"], cfg.get("agent", 0), step, g, cfg["alpha_rg"])
    tune = bool(cfg.get("alpha_autotune", False))
    if tune and state.log_alpha is None:
        state.log_alpha = float(np.log(cfg["alpha"]))
    alpha = float(np.exp(state.log_alpha)) if tune else cfg["alpha"]
    act = actor.actor_loss_and_grad(state.nets["pi"], state.nets["phi"], state.nets["psi"], s, g_actor, eps,
                                    cfg["energy"], cfg["tau"], alpha)
    state.t_actor += 1
    state.nets["pi"], state.m["pi"], state.v["pi"] = adam_net(
        state.nets["pi"], act["grads"], state.m["pi"], state.v["pi"], state.t_actor, cfg["lr_actor"], *betas)
    out = {"critic": parts, "actor_loss": act["loss"], "logpi_mean": act["logpi_mean"], "idx": idx, "alpha": alpha}
    if tune:
        ga = actor.alpha_loss_grad(act["logpi_mean"], cfg["target_entropy"])
        la, state.m_alpha, state.v_alpha = adam.adam_update(state.log_alpha, ga, state.m_alpha, state.v_alpha,
                                                        state.t_actor, cfg["lr_alpha"], *betas)
        state.log_alpha = float(la)
        out["alpha_next"] = float(np.exp(state.log_alpha))
    return out
