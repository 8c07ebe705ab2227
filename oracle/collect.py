"""Collection stub: Algorithm 1's loop over environments with synthetic dynamics.

Test infrastructure only (see ``oracle/__init__``).

Algorithm 1 (App. F) alternates collection (each environment acts with the
policy, steps, and stores its trajectory) with ``num_updates`` update steps;
§5.6 studies the ratio of the two.  The simulators are outside this project, so
the library's collection stub runs dynamics of its own definition.  This module
restates that definition, written plainly:

S1  E environments; environment e holds a state s_e [D], a commanded goal g_e [G]
    and its step t_e within the episode.  The first states and goals are
    N(0, I) draws (Philox words 4 and 5 at the counter value 2^64 - 1).
S2  Collection step k (k = 0, 1, ...): (mu, l) = pi(concat(s, g)) and
    a = tanh(mu + exp(clip(l)) eps), eps ~ N(0, I) from word 2 at counter k (the
    policy head of the actor, reading P1).
S3  The slice (s, a, done) is appended to the buffer, done = [t_e = L - 1] for
    the episode length L.
S4  s' = s + 0.1 xi + 0.05 a[d mod A], xi ~ N(0, I) from word 3 at counter k;
    after an episode's last step instead s' ~ N(0, I) (word 4) and
    g' ~ N(0, I) (word 5) at counter k, and t' = 0; else t' = t + 1.
All draws: ``actor.gaussian_noise`` (Box-Muller on Philox4x64-10 blocks
(counter, env, word, d // 4) keyed (seed, agent)).  The state is float32, like
the buffer that stores it.
"""

import numpy as np

from . import actor, mlp

INIT_STEP = (1 << 64) - 1


def initial_envs(seed, agent, E, D, G):
    """(s [E][D], g [E][G], t [E]) before the first collection step (S1)."""
    s = actor.gaussian_noise(seed, agent, INIT_STEP, E, D, word=4).astype(np.float32)
    g = actor.gaussian_noise(seed, agent, INIT_STEP, E, G, word=5).astype(np.float32)
    return s, g, np.zeros(E, dtype=np.int64)


def collect(pi_net, envs, step0, n, episode_length, seed, agent, A):
    """n collection steps from ``envs`` = (s, g, t) at counter step0 (S2-S4).

    Returns (obs [n][E][D] f32, act [n][E][A] f32, done [n][E] u8, new envs).
    """
    s, g, t = (x.copy() for x in envs)
    E, D = s.shape
    G = g.shape[1]
    obs = np.zeros((n, E, D), dtype=np.float32)
    act = np.zeros((n, E, A), dtype=np.float32)
    done = np.zeros((n, E), dtype=np.uint8)
    for i in range(n):
        k = step0 + i
        out, _ = mlp.forward(pi_net, np.concatenate([s, g], axis=1).astype(np.float64))
        eps = actor.gaussian_noise(seed, agent, k, E, A, word=2)
        a, _, _ = actor.policy_head(out, eps)
        last = t >= episode_length - 1
        obs[i] = s
        act[i] = a.astype(np.float32)
        done[i] = last.astype(np.uint8)
        xi = actor.gaussian_noise(seed, agent, k, E, D, word=3)
        cols = np.arange(D) % A
        moved = s.astype(np.float64) + 0.1 * xi + 0.05 * a[:, cols]
        fresh_s = actor.gaussian_noise(seed, agent, k, E, D, word=4)
        fresh_g = actor.gaussian_noise(seed, agent, k, E, G, word=5)
        s = np.where(last[:, None], fresh_s, moved).astype(np.float32)
        g = np.where(last[:, None], fresh_g, g).astype(np.float32)
        t = np.where(last, 0, t + 1)
    return obs, act, done, (s, g, t)
