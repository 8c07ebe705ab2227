"""Pins for the oracle's replay buffer and future-goal relabelling.

They check the oracle against what the paper and probability fix, not against
itself: the exact truncated-geometric pmf computed from gamma^k directly, the
closed-form mean, uniformity of (e, t), the episode structure, and special
cases (gamma = 0, L = 0, L = 1).
"""

from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import relabel
from oracle.philox import philox4x64_10
from paper_2408_11052_gb300 import workload


def exact_cdf(gamma, L, k, offset_min=1):
    """P(offset <= k) for the truncated geometric on {m..L}, P(j) ~ gamma^(j-m)."""
    m = offset_min
    g = float(np.float32(gamma))
    return (1.0 - g ** (k - m + 1)) / (1.0 - g ** (L - m + 1))


def test_gamma_fixed_point_is_rounded_scaled_gamma():
    for gamma in (0.0, 0.5, 0.9, 0.97, 0.99, 0.999, 1.0 - 2.0 ** -24):
        gq = relabel.gamma_fixed_point(gamma)
        exact = Fraction(float(np.float32(gamma))) * 2 ** 32
        assert abs(Fraction(gq) - exact) <= Fraction(1, 2)
    with pytest.raises(ValueError):
        relabel.gamma_fixed_point(1.0)


@pytest.mark.parametrize("gamma", [0.0, 0.5, 0.99, 0.999])
def test_geometric_table_tracks_exact_powers(gamma):
    table = relabel.geometric_table(gamma, 1001)
    gq = relabel.gamma_fixed_point(gamma)
    assert table[0] == 2 ** 32
    for k in (1, 2, 3, 10, 100, 500, 1001):
        exact = Fraction(gq ** k, 2 ** (32 * (k - 1)))   # (gq / 2^32)^k * 2^32
        assert exact - k <= table[k] <= exact
    assert all(table[k] >= table[k + 1] for k in range(1001))


@pytest.mark.parametrize("gamma,L,offset_min", [(0.99, 1, 1), (0.99, 2, 1), (0.99, 5, 1), (0.9, 100, 1),
                                                (0.99, 100, 1), (0.99, 999, 1), (0.99, 7, 0), (0.5, 40, 0)])
def test_offset_inverse_cdf_on_grid(gamma, L, offset_min):
    """A deterministic uniform grid of v reproduces the exact CDF within 1/N."""
    table = relabel.geometric_table(gamma, L + 2)
    N = 4096 if L < 500 else 1024
    ks = np.array([relabel.truncated_geometric_offset(int((i + 0.5) * 2 ** 32 / N), L, table, offset_min)
                   for i in range(N)])
    assert ks.min() >= offset_min and ks.max() <= L
    for k in range(offset_min, L + 1):
        emp = np.mean(ks <= k)
        assert abs(emp - exact_cdf(gamma, L, k, offset_min)) <= 1.0 / N + 1e-6, k


def test_offset_special_cases():
    t99 = relabel.geometric_table(0.99, 20)
    t0 = relabel.geometric_table(0.0, 20)
    for v in (0, 1, 2 ** 31, 2 ** 32 - 1):
        assert relabel.truncated_geometric_offset(v, 0, t99) == 0          # no future step: the state itself
        assert relabel.truncated_geometric_offset(v, 1, t99) == 1          # only one future step
        assert relabel.truncated_geometric_offset(v, 17, t0) == 1          # gamma = 0: next step
        assert relabel.truncated_geometric_offset(v, 17, t0, 0) == 0       # gamma = 0, k >= 0: now
        assert relabel.truncated_geometric_offset(v, 0, t99, 0) == 0
    # v = 0 always picks the first support point, v = 2^32 - 1 the last for short horizons
    assert relabel.truncated_geometric_offset(0, 10, t99) == 1
    assert relabel.truncated_geometric_offset(2 ** 32 - 1, 10, t99) == 10


@pytest.mark.parametrize("L", [5, 100, 999])
def test_offset_distribution_with_philox_draws(L):
    """Chi-square and the closed-form mean E[k] = 1/(1-g) - L g^L / (1-g^L) on Philox draws."""
    gamma = 0.99
    g = float(np.float32(gamma))
    table = relabel.geometric_table(gamma, L + 2)
    n = 20000
    ks = np.array([relabel.truncated_geometric_offset(philox4x64_10((L, i, 0, 0), (99, 0))[1] >> 32, L, table)
                   for i in range(n)])
    mean = 1.0 / (1.0 - g) - L * g ** L / (1.0 - g ** L)
    pk = np.array([g ** (k - 1) for k in range(1, L + 1)])
    pk /= pk.sum()
    var = float(np.sum(pk * (np.arange(1, L + 1) - mean) ** 2))
    assert abs(ks.mean() - mean) < 5.0 * np.sqrt(var / n)
    # chi-square on bins with expected count >= 20
    counts = np.bincount(ks, minlength=L + 1)[1:]
    exp = pk * n
    edges, obs_b, exp_b, acc_o, acc_e = [], [], [], 0, 0.0
    for c, e_ in zip(counts, exp):
        acc_o += c
        acc_e += e_
        if acc_e >= 20:
            obs_b.append(acc_o)
            exp_b.append(acc_e)
            acc_o, acc_e = 0, 0.0
    obs_b[-1] += acc_o
    exp_b[-1] += acc_e
    p = stats.chisquare(obs_b, exp_b).pvalue
    assert p > 1e-3


def small_buffer(E=4, T=50, D=5, A=3, n=80, mean_len=8.0, seed=5):
    w = workload.Workload("t", E=E, T=T, D=D, A=A, G=2, B=64, hidden=8, layers=1, repr=4, seed=seed)
    obs, act, done = workload.buffer_contents(w, n=n, mean_len=mean_len)
    buf = relabel.ReplayBuffer(E, T, D, A)
    buf.insert(obs[: n // 2], act[: n // 2], done[: n // 2])
    buf.insert(obs[n // 2:], act[n // 2:], done[n // 2:])
    return buf, (obs, act, done)


def test_ring_keeps_newest_steps():
    buf, (obs, act, done) = small_buffer()
    assert buf.size == 50
    np.testing.assert_array_equal(buf.obs, obs[-50:].transpose(1, 0, 2))
    np.testing.assert_array_equal(buf.act, act[-50:].transpose(1, 0, 2))
    np.testing.assert_array_equal(buf.done, done[-50:].T.astype(bool))


def test_horizon_matches_episode_ids():
    buf, _ = small_buffer()
    for e in range(buf.E):
        # episode id of step t = number of done flags strictly before t
        ep = np.concatenate([[0], np.cumsum(buf.done[e].astype(int))[:-1]])
        for t in range(buf.size):
            L = buf.horizon(e, t)
            assert ep[t + L] == ep[t]
            assert t + L == buf.size - 1 or buf.done[e, t + L]
            assert not buf.done[e, t:t + L].any()


def test_relabel_goals_stay_in_episode_future():
    buf, _ = small_buffer()
    goal_idx = (3, 1)
    s, a, g, idx = relabel.sample_relabel(buf, seed=11, agent=2, step=7, B=400, goal_idx=goal_idx, gamma=0.9)
    for b in range(400):
        e, t, k = idx[b]
        L = buf.horizon(e, t)
        assert (k == 0) == (L == 0)
        assert 1 <= k <= L or L == 0
        np.testing.assert_array_equal(s[b], buf.obs[e, t])
        np.testing.assert_array_equal(a[b], buf.act[e, t])
        np.testing.assert_array_equal(g[b], buf.obs[e, t + k, list(goal_idx)])


def test_relabel_transitions_uniform():
    E, size = 4, 16
    n = 16000
    cells = np.zeros(E * size, dtype=int)
    for b in range(n):
        e, t, _ = relabel.draw_indices(3, 0, 1, b, E, size)
        assert 0 <= e < E and 0 <= t < size
        cells[e * size + t] += 1
    assert stats.chisquare(cells).pvalue > 1e-3


def test_relabel_is_a_function_of_seed_step_agent():
    buf, _ = small_buffer()
    r1 = relabel.sample_relabel(buf, 1, 0, 3, 32, (0, 1), 0.99)[3]
    r2 = relabel.sample_relabel(buf, 1, 0, 3, 32, (0, 1), 0.99)[3]
    r3 = relabel.sample_relabel(buf, 1, 0, 4, 32, (0, 1), 0.99)[3]
    r4 = relabel.sample_relabel(buf, 1, 1, 3, 32, (0, 1), 0.99)[3]
    np.testing.assert_array_equal(r1, r2)
    assert (r1 != r3).any() and (r1 != r4).any()
