"""Pins for the random-goal actor mix (App. D; reading P6 of the oracle's actor
module): the extreme weights, the choice bit recomputed from numpy's own Philox,
the rate of random goals against the binomial law, and the update step's use of
the mixed goals for the actor only."""

import math

import numpy as np
import pytest

from oracle import relabel, step
from oracle.relabel import actor_goal_mix

from test_oracle_philox import numpy_block


def goals(B, G=3, seed=0):
    return np.random.default_rng(seed).standard_normal((B, G))


def test_weight_zero_keeps_every_goal():
    g = goals(17)
    out, rnd = actor_goal_mix(5, 1, 9, g, 0.0)
    np.testing.assert_array_equal(out, g)
    assert not rnd.any()


def test_weight_one_takes_the_next_sample_goal():
    g = goals(17)
    out, rnd = actor_goal_mix(5, 1, 9, g, 1.0)
    assert rnd.all()
    np.testing.assert_array_equal(out, np.roll(g, -1, axis=0))


@pytest.mark.parametrize("alpha_rg", [0.25, 0.5, 0.8])
def test_choice_bit_from_numpy_philox(alpha_rg):
    """Word 2 of numpy's Philox4x64-10 block (step, b, 0, 0) keyed (seed, agent)."""
    seed, agent, st, B = 11, 3, 123456, 64
    g = goals(B, seed=2)
    out, rnd = actor_goal_mix(seed, agent, st, g, alpha_rg)
    thr = math.floor(float(np.float32(alpha_rg)) * 2.0 ** 32)
    for b in range(B):
        w = numpy_block([st, b, 0, 0], [seed, agent])
        assert rnd[b] == ((w[2] >> 32) < thr)
        np.testing.assert_array_equal(out[b], g[(b + 1) % B] if rnd[b] else g[b])


def test_rate_of_random_goals_is_binomial():
    B, a = 4096, 0.3
    _, rnd = actor_goal_mix(7, 0, 42, goals(B), a)
    sd = math.sqrt(B * a * (1 - a))
    assert abs(rnd.sum() - B * a) < 4 * sd


def test_update_step_uses_mixed_goals_for_the_actor_only():
    """The critic parts do not depend on alpha_rg; the actor loss equals the actor
    loss evaluated on the mixed goals."""
    from oracle import actor, mlp  # noqa: F401
    rng = np.random.default_rng(3)
    E, T, D, A, G, B = 4, 30, 6, 2, 2, 12

    def net(sizes):
        return [{"W": rng.standard_normal((o, i)) / math.sqrt(i), "b": rng.standard_normal(o) * 0.1}
                for i, o in zip(sizes[:-1], sizes[1:])]

    phi, psi, pi = net([D + A, 8, 4]), net([G, 8, 4]), net([D + G, 8, 2 * A])
    buf = relabel.ReplayBuffer(E, T, D, A)
    buf.insert(rng.standard_normal((20, E, D)), rng.uniform(-1, 1, (20, E, A)), np.zeros((20, E), dtype=np.uint8))
    cfg = dict(seed=1, agent=0, B=B, goal_idx=[0, 1], gamma=0.9, energy="l2", tau=1.0, loss="sym",
               sym_reduction="mean", beta=0.1, penalty_axis="row", alpha=0.1, lr_critic=0.0, lr_actor=0.0)
    eps = actor.gaussian_noise(1, 0, 5, B, A)
    outs = {}
    for a_rg in (0.0, 0.6):
        st = step.AgentState(phi, psi, pi)
        outs[a_rg] = step.update_step(st, buf, dict(cfg, alpha_rg=a_rg), 5, eps)
    assert outs[0.0]["critic"]["total"] == outs[0.6]["critic"]["total"]
    s, _, g, _ = relabel.sample_relabel(buf, 1, 0, 5, B, [0, 1], 0.9)
    g_mix, rnd = actor_goal_mix(1, 0, 5, g, 0.6)
    assert rnd.any() and not rnd.all()
    ref = actor.actor_loss_and_grad(pi, phi, psi, s, g_mix, eps, "l2", 1.0, 0.1)
    assert outs[0.6]["actor_loss"] == pytest.approx(ref["loss"], rel=1e-14)
    assert outs[0.6]["actor_loss"] != outs[0.0]["actor_loss"]
