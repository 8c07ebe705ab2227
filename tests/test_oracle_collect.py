"""Pins for the oracle's collection stub (its own synthetic dynamics, not the
paper's; readings S1-S4 of ``oracle.collect``): episode boundaries, the zero
policy's closed form, the dynamics residuals and the reset states against the
normal law, and float32 storage."""

import math

import numpy as np
import pytest

from oracle import actor, collect


def zero_policy(D, G, A, hidden=5):
    return [{"W": np.zeros((hidden, D + G)), "b": np.zeros(hidden)},
            {"W": np.zeros((2 * A, hidden)), "b": np.zeros(2 * A)}]


def random_policy(D, G, A, hidden=7, seed=0):
    rng = np.random.default_rng(seed)
    return [{"W": rng.standard_normal((hidden, D + G)) / math.sqrt(D + G), "b": rng.standard_normal(hidden) * 0.1},
            {"W": rng.standard_normal((2 * A, hidden)) / math.sqrt(hidden), "b": rng.standard_normal(2 * A) * 0.1}]


@pytest.mark.parametrize("L", [1, 3, 7])
def test_done_flags_close_every_episode_after_L_steps(L):
    E, D, G, A = 5, 4, 2, 3
    envs = collect.initial_envs(1, 0, E, D, G)
    _, _, done, (_, _, t) = collect.collect(zero_policy(D, G, A), envs, 0, 20, L, 1, 0, A)
    expect = np.array([(k % L) == L - 1 for k in range(20)], dtype=np.uint8)
    for e in range(E):
        np.testing.assert_array_equal(done[:, e], expect)
    assert (t == 20 % L).all()


def test_zero_policy_acts_with_tanh_of_the_collection_noise():
    """mu = 0 and log sigma = 0: a = tanh(eps), eps the word-2 draws of each step."""
    E, D, G, A = 6, 5, 2, 3
    envs = collect.initial_envs(4, 2, E, D, G)
    _, act, _, _ = collect.collect(zero_policy(D, G, A), envs, 10, 4, 100, 4, 2, A)
    for i in range(4):
        eps = actor.gaussian_noise(4, 2, 10 + i, E, A, word=2)
        np.testing.assert_allclose(act[i], np.tanh(eps).astype(np.float32), rtol=1e-7, atol=1e-7)


def test_dynamics_residuals_and_resets_are_standard_normal():
    E, D, G, A, L, n = 64, 8, 2, 4, 5, 40
    envs = collect.initial_envs(7, 0, E, D, G)
    obs, act, done, _ = collect.collect(random_policy(D, G, A), envs, 0, n, L, 7, 0, A)
    cols = np.arange(D) % A
    res, fresh = [], []
    for i in range(n - 1):
        moving = done[i] == 0
        r = (obs[i + 1].astype(np.float64) - obs[i] - 0.05 * act[i][:, cols].astype(np.float64)) / 0.1
        res.append(r[moving])
        fresh.append(obs[i + 1][~moving].astype(np.float64))
    res = np.concatenate(res).ravel()
    fresh = np.concatenate(fresh).ravel()
    for x in (res, fresh):
        n_x = x.size
        assert abs(x.mean()) < 4 / math.sqrt(n_x)
        assert abs(x.var() - 1.0) < 4 * math.sqrt(2.0 / n_x)
    # the first states are the initial N(0, I) draws
    assert abs(obs[0].mean()) < 4 / math.sqrt(obs[0].size)


def test_states_are_stored_as_float32():
    E, D, G, A = 3, 4, 2, 2
    obs, act, done, (s, g, _) = collect.collect(random_policy(D, G, A), collect.initial_envs(0, 0, E, D, G), 0, 3,
                                                2, 0, 0, A)
    assert obs.dtype == np.float32 and act.dtype == np.float32 and s.dtype == np.float32 and g.dtype == np.float32
