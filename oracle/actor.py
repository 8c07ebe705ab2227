"""Actor objective (DDPG-style policy extraction with an entropy term) and its gradient.

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes
--------------------
* Eq. 3 (§3.2): the goal-conditioned policy pi_theta(a | s, g) maximises
  E[f(s, a', g)] with a' ~ pi_theta(. | s, g), (s, a) uniform from the buffer
  and g from the future of the same trajectory (random-goal weight 0, App. C).
* §5.1: the methods use "a tuneable entropy coefficient".
* Algorithm 1: the policy update follows the critic update of the same step,
  so the critic parameters are the freshly updated ones; the critic is not
  changed by the actor loss.

Readings where the paper is silent
----------------------------------
P1  The policy is a tanh-squashed diagonal Gaussian: the MLP on concat(s, g)
    outputs (mu, l) of width 2A, l is clipped to [-5, 2], sigma = exp(l),
    u = mu + sigma * eps with eps ~ N(0, I) (passed in), a' = tanh(u).
P2  log pi(a'|s, g) = sum_d [ -eps_d^2 / 2 - log(2 pi) / 2 - l_d
                              - 2 (log 2 - u_d - softplus(-2 u_d)) ],
    the Gaussian log-density minus log|det da'/du| = sum log(1 - tanh(u)^2),
    written in the overflow-free form.
P3  L_actor = mean_i [ alpha * log pi_i - F_ii ], F_ii = f(phi(s_i, a'_i), psi(g_i)) / tau
    with the critic's energy and temperature; alpha is given.
P4  The clip passes the gradient only strictly inside (-5, 2).
P5  Entropy-coefficient auto-tuning (§5.1, "a tuneable entropy coefficient";
    the paper gives no rule): alpha = exp(log_alpha), log_alpha learned by
    Adam on  L(log_alpha) = -log_alpha * (mean_i log pi_i + H_target)  with
    log pi held fixed and H_target = -A (the action dimension).  The actor
    loss of a step uses alpha before that step's update; the configured alpha
    is the initial value.
P6  Random-goal actor mix (App. D, weight alpha_rg; the paper recommends and
    uses 0): sample b's actor goal is, with probability alpha_rg, the
    relabelled goal of sample (b + 1) mod B of the same batch (another,
    independently drawn transition, so a draw from the buffer's goal
    marginal), else its own relabelled goal.  The choice uses the top 32 bits
    of word 2 of sample b's relabel Philox block (step, b, 0, 0): a random goal
    iff (w2 >> 32) < floor(alpha_rg * 2^32) (alpha_rg a float32, so the
    threshold is exact).  The per-sample mixture is an unbiased estimate of
    App. D's weighted sum of the two expectations.  See
    ``relabel.actor_goal_mix``.
"""

import numpy as np

from . import critic, mlp

LOG_STD_MIN = -5.0
LOG_STD_MAX = 2.0


def gaussian_noise(seed, agent, step, B, A, word=1):
    """eps [B][A] ~ N(0, 1) drawn from Philox4x64-10 by the Box-Muller transform.

    Used when the update step draws its own actor noise (reading P1; ``word`` 1,
    the collection stub's draws use 2 to 5).  For row b
    and element d: block (step, b, word, d // 4) under key (seed, agent); words
    2q and 2q+1 (q = (d % 4) // 2) give u1, u2 = (top 53 bits + 1/2) / 2^53,
    and the element is sqrt(-2 ln u1) * (cos 2 pi u2 if d is even else sin 2 pi u2)
    (Box & Muller, 1958).
    """
    from .philox import philox4x64_10
    eps = np.zeros((B, A))
    for b in range(B):
        for d in range(A):
            w = philox4x64_10((step, b, word, d // 4), (seed, agent))
            q = (d % 4) // 2
            u1 = ((w[2 * q] >> 11) + 0.5) / 2.0 ** 53
            u2 = ((w[2 * q + 1] >> 11) + 0.5) / 2.0 ** 53
            rad = np.sqrt(-2.0 * np.log(u1))
            eps[b, d] = rad * (np.cos(2.0 * np.pi * u2) if d % 2 == 0 else np.sin(2.0 * np.pi * u2))
    return eps


def softplus(x):
    return np.logaddexp(0.0, x)


def policy_head(out, eps):
    """Reading P1 / P2: (a', log pi, intermediates) from the MLP output [B][2A]."""
    A = out.shape[1] // 2
    mu, l_raw = out[:, :A], out[:, A:]
    ell = np.clip(l_raw, LOG_STD_MIN, LOG_STD_MAX)
    sigma = np.exp(ell)
    u = mu + sigma * eps
    a_new = np.tanh(u)
    logpi = (-0.5 * eps ** 2 - 0.5 * np.log(2.0 * np.pi) - ell
             - 2.0 * (np.log(2.0) - u - softplus(-2.0 * u))).sum(axis=1)
    return a_new, logpi, {"l_raw": l_raw, "sigma": sigma, "u": u, "a": a_new}


def actor_loss_and_grad(pi_net, phi_net, psi_net, s, g, eps, energy="l2", tau=1.0, alpha=0.1):
    """L_actor (reading P3) and its gradient with respect to the actor parameters.

    Returns dict: loss, logpi_mean, f_mean, grads (like ``pi_net``), a_new.
    """
    s = np.asarray(s, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    B, D = s.shape
    out, pi_cache = mlp.forward(pi_net, np.concatenate([s, g], axis=1))
    a_new, logpi, hc = policy_head(out, eps)
    phi, phi_cache = mlp.forward(phi_net, np.concatenate([s, a_new], axis=1))
    psi, _ = mlp.forward(psi_net, g)
    f = critic.energy_diagonal(phi, psi, energy, tau)
    loss = np.mean(alpha * logpi - f)

    # d loss / d f_i = -1/B ; through phi only (psi does not depend on theta).
    dphi, _ = critic.energy_diagonal_backward(phi, psi, -np.ones(B) / B, energy, tau)
    _, dx = mlp.backward(phi_net, phi_cache, dphi)
    da = dx[:, D:]
    u, sigma, a = hc["u"], hc["sigma"], hc["a"]
    # d logpi / du = 2 tanh(u); d logpi / dl = -1 (plus the u path)
    du = da * (1.0 - a ** 2) + (alpha / B) * 2.0 * a
    dmu = du
    dl = du * sigma * eps - (alpha / B)
    inside = (hc["l_raw"] > LOG_STD_MIN) & (hc["l_raw"] < LOG_STD_MAX)
    dl_raw = np.where(inside, dl, 0.0)
    grads, _ = mlp.backward(pi_net, pi_cache, np.concatenate([dmu, dl_raw], axis=1))
    return {"loss": loss, "logpi_mean": float(np.mean(logpi)), "f_mean": float(np.mean(f)),
            "grads": grads, "a_new": a_new, "logpi": logpi}


def alpha_loss_grad(logpi_mean, target_entropy):
    """dL/d(log alpha) of  L = -log_alpha * (logpi_mean + target_entropy)  (reading P5)."""
    return -(float(logpi_mean) + float(target_entropy))
