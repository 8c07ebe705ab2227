"""Replay buffer model and hindsight future-goal relabelling, written plainly.

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes
--------------------
* §3 (Preliminaries): the discounted state-visitation distribution is the
  distribution of the state T steps in the future with T ~ Geom(1 - gamma);
  App. D.1 shows it equals the goal-conditioned Q-function.
* §3.1 and §3.2: each batch element (s_i, a_i, g_i) takes (s, a) uniformly
  from the buffer and the goal g_i from the future of the same trajectory.
* Algorithm 1 (App. F): trajectories are stored per environment; the update
  samples "with discount" a batch of state-action pairs and future goals.
* App. B.3 (Table "Hyperparameters"): ``max_replay_size`` transitions per
  environment, ``discounting`` = 0.99.

Readings where the paper is silent
----------------------------------
R1  The transition (e, t) is uniform over all E * size stored steps.
R2  The offset k has support {1..L} with P(k) proportional to gamma^(k-1)
    (strict future; ``offset_min = 1``), renormalised over what is left of the
    episode: L = (last step of the episode) - t, and for an episode that is
    still open, L = (newest stored step) - t.  When L = 0 the goal is the
    state itself (k = 0).  ``offset_min = 0`` gives support {0..L} with
    P(k) proportional to gamma^k.
R3  The goal is a fixed subset ``goal_idx`` of the state dimensions.
R4  Random numbers: Philox4x64-10 keyed by (seed, agent) and countered by
    (step, b, 0, 0) for batch element b.  Output word 0 picks the transition
    through a 64x64 -> high-64 multiply (idx = floor(w0 * n / 2^64)); the top
    32 bits of word 1 drive the offset.
R5  The inverse CDF of the truncated geometric is evaluated in integer
    arithmetic on a fixed-point table of gamma^k (``geometric_table``), so that
    two independent implementations take the same decision for every draw:
    k is the smallest k in the support with
        v * (G[0] - G[L + 1 - m]) < (G[0] - G[k + 1 - m]) * 2^32,  m = offset_min,
    i.e. v / 2^32 < CDF(k).  This is the exact inverse CDF of the truncated
    geometric up to the <= 2^-32 per-step flooring of the table.
R6  A stored step's ``done`` flag marks its observation as the last of its
    episode (the terminal s' of Algorithm 1); the next stored step starts a
    new episode.
"""

import numpy as np

from .philox import philox4x64_10

TWO32 = 1 << 32
TWO64 = 1 << 64


def gamma_fixed_point(gamma):
    """gq = round(gamma * 2^32), computed exactly (gamma is a float32 value).

    gamma * 2^32 is exact in binary64 for any float32 gamma, so adding 1/2 and
    flooring rounds half up without any rounding error.
    """
    if not (0.0 <= gamma < 1.0):
        raise ValueError("gamma must lie in [0, 1)")
    return int(np.floor(float(np.float32(gamma)) * float(TWO32) + 0.5))


def geometric_table(gamma, n):
    """G[0] = 2^32, G[k] = floor(G[k-1] * gq / 2^32) for k = 1..n (reading R5).

    G[k] approximates gamma^k * 2^32 from below; integers only.
    """
    gq = gamma_fixed_point(gamma)
    table = [TWO32]
    for _ in range(n):
        table.append((table[-1] * gq) >> 32)
    return table


def truncated_geometric_offset(v, L, table, offset_min=1):
    """Smallest offset k whose CDF exceeds v / 2^32 (reading R2 and R5).

    v: 32-bit uniform integer.  L: steps left in the episode after t.
    Scans k upward, which is the definition of the inverse CDF; Python
    integers never overflow.
    """
    if offset_min not in (0, 1):
        raise ValueError("offset_min must be 0 or 1")
    if L == 0 and offset_min == 1:
        return 0
    m = offset_min
    total = table[0] - table[L + 1 - m]
    for k in range(m, L + 1):
        if v * total < (table[0] - table[k + 1 - m]) * TWO32:
            return k
    raise AssertionError("inverse CDF did not terminate; gamma must be < 1")


class ReplayBuffer:
    """Per-environment trajectory storage (Algorithm 1; App. B.3 capacity).

    Keeps, per environment, the newest ``T`` steps in chronological order:
    obs[e][t], act[e][t], done[e][t] with t = 0 the oldest stored step.
    All environments insert in lockstep (one time slice per call row).
    """

    def __init__(self, E, T, D, A):
        self.E, self.T, self.D, self.A = E, T, D, A
        self.obs = np.zeros((E, 0, D), dtype=np.float64)
        self.act = np.zeros((E, 0, A), dtype=np.float64)
        self.done = np.zeros((E, 0), dtype=bool)

    @property
    def size(self):
        return self.obs.shape[1]

    def insert(self, obs, act, done):
        """Append n time slices: obs [n][E][D], act [n][E][A], done [n][E]."""
        obs = np.asarray(obs, dtype=np.float64)
        act = np.asarray(act, dtype=np.float64)
        done = np.asarray(done).astype(bool)
        self.obs = np.concatenate([self.obs, obs.transpose(1, 0, 2)], axis=1)[:, -self.T:]
        self.act = np.concatenate([self.act, act.transpose(1, 0, 2)], axis=1)[:, -self.T:]
        self.done = np.concatenate([self.done, done.T], axis=1)[:, -self.T:]

    def horizon(self, e, t):
        """L = steps from t to the end of its episode, truncated at the newest step (R2, R6)."""
        for tau in range(t, self.size):
            if self.done[e, tau]:
                return tau - t
        return self.size - 1 - t


def draw_indices(seed, agent, step, b, E, size):
    """(e, t, v) for batch element b (readings R1 and R4)."""
    w = philox4x64_10((step, b, 0, 0), (seed, agent))
    n = E * size
    idx = (w[0] * n) >> 64
    e, t = divmod(idx, size)
    v = w[1] >> 32
    return e, t, v


def actor_goal_mix(seed, agent, step, g, alpha_rg):
    """Actor goals of the random-goal mix (App. D; reading P6 of the actor module).

    g [B][G]: the relabelled goals of the batch drawn at ``step``.  Returns
    (g_actor [B][G], random [B] bool).
    """
    g = np.asarray(g, dtype=np.float64)
    B = g.shape[0]
    thr = min(int(np.floor(float(np.float32(alpha_rg)) * TWO32)), TWO32)
    out = g.copy()
    rnd = np.zeros(B, dtype=bool)
    for b in range(B):
        w = philox4x64_10((step, b, 0, 0), (seed, agent))
        if (w[2] >> 32) < thr:
            rnd[b] = True
            out[b] = g[(b + 1) % B]
    return out, rnd


def sample_relabel(buf, seed, agent, step, B, goal_idx, gamma, offset_min=1):
    """Sample a relabelled batch (Algorithm 1, "sample with discount").

    Returns s [B][D], a [B][A], g [B][G] (float64) and idx [B][3] = (e, t, k)
    (int64), t chronological from the oldest stored step.
    """
    if buf.size == 0:
        raise ValueError("empty buffer")
    table = geometric_table(gamma, buf.T + 1)
    goal_idx = list(goal_idx)
    s = np.zeros((B, buf.D))
    a = np.zeros((B, buf.A))
    g = np.zeros((B, len(goal_idx)))
    idx = np.zeros((B, 3), dtype=np.int64)
    for b in range(B):
        e, t, v = draw_indices(seed, agent, step, b, buf.E, buf.size)
        L = buf.horizon(e, t)
        k = truncated_geometric_offset(v, L, table, offset_min)
        s[b] = buf.obs[e, t]
        a[b] = buf.act[e, t]
        g[b] = buf.obs[e, t + k, goal_idx]
        idx[b] = (e, t, k)
    return s, a, g, idx

