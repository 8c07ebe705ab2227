"""Seeded synthetic inputs for the CRL update step.

This module only draws numbers; it holds none of the method's arithmetic.  It
serves both the CUDA path (tests, ``bench.py``) and the CPU oracle, which
receive the same arrays.

Workloads stand in for the paper's Brax environments (not available here):
shapes follow the environment table and the hyperparameter table of the
paper (Ant: obs 29, action 8, goal 2; Humanoid: obs 268, action 17, goal 3;
1024 environments, episodes of 1000 steps, batch 256, discount 0.99).

Recipe
------
* States: per environment s_0 ~ N(0, I_D), s_{t+1} = s_t + 0.1 xi_t with
  xi_t ~ N(0, I_D); a new episode restarts from a fresh N(0, I_D) draw.
* Actions: i.i.d. U[-1, 1]^A.
* Episodes: fixed length (``episode_len``) or geometric lengths with a given
  mean (>= 1) to exercise short and zero horizons.  ``done`` marks the last
  step of each episode.
* Weights: W ~ N(0, 1/fan_in), stored [out][in]; biases 0, LayerNorm gain 1
  and bias 0; with ``perturb`` the biases, gains and shifts get small seeded
  noise so that every parameter tensor carries signal in parity tests.
* Actor noise: eps ~ N(0, I_A).
"""

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    """Shapes and hyperparameters of one CRL update-step workload."""
    name: str
    E: int            # parallel environments (buffer rows)
    T: int            # stored steps per environment (ring capacity)
    D: int            # observation dim
    A: int            # action dim
    G: int            # goal dim (goal = obs[goal_idx])
    B: int            # batch size
    hidden: int       # hidden width
    layers: int       # hidden layers
    repr: int         # representation dim R
    layernorm: bool = False
    energy: str = "l2"
    loss: str = "sym"
    sym_reduction: str = "mean"
    penalty_axis: str = "row"
    beta: float = 0.1
    tau: float = 1.0
    gamma: float = 0.99
    alpha: float = 0.1
    lr_critic: float = 3e-4
    lr_actor: float = 6e-4
    episode_len: int = 1000
    seed: int = 0
    goal_idx: tuple = field(default=None)
    alpha_autotune: bool = False     # learn log(alpha) (reading P5); target entropy -A, lr = lr_actor
    target_entropy: float = None
    lr_alpha: float = None
    alpha_rg: float = 0.0            # random-goal actor mix (reading P6)

    def goals(self):
        return tuple(range(self.G)) if self.goal_idx is None else tuple(self.goal_idx)

    def with_(self, **kw):
        return replace(self, **kw)


# The five workloads of the measurement plan, by what they are.
SMALL_FP32 = Workload("small_fp32_critic_E64xT1000_D29_B256", E=64, T=1000, D=29, A=8, G=2, B=256,
                      hidden=256, layers=2, repr=64, energy="l2", loss="sym", seed=0)
ANT_AUTOGRAD = Workload("ant_E1024xT1000_D29_A8_G2_B256_2x256_R64", E=1024, T=1000, D=29, A=8, G=2,
                        B=256, hidden=256, layers=2, repr=64, energy="l2", loss="sym", seed=1)
HUMANOID_BF16 = Workload("humanoid_E1024xT1000_D268_A17_G3_B1024_4x1024LN_R64_cos", E=1024, T=1000,
                         D=268, A=17, G=3, B=1024, hidden=1024, layers=4, repr=64, layernorm=True,
                         energy="cos", loss="sym", tau=1.0, seed=2)
LARGE_BATCH = Workload("large_batch_E4096xT500_D64_A16_G8_B8192_2x512_R256", E=4096, T=500, D=64,
                       A=16, G=8, B=8192, hidden=512, layers=2, repr=256, energy="l2", loss="fwd",
                       episode_len=500, seed=3)
WORKLOADS = {w.name: w for w in (SMALL_FP32, ANT_AUTOGRAD, HUMANOID_BF16, LARGE_BATCH)}


def sweep_agents(n_agents=32, seed=4):
    """The batched-sweep workload: independent agents with uneven shapes.

    Batch sizes uniform over {256, 512, 1024, 2048}, obs dims over {29, 64, 268}
    (goal/action dims tied to the obs dim: 29 -> (2, 8), 64 -> (8, 16),
    268 -> (3, 17)), repr dims over {64, 128}; 512 envs x 1000 steps each.
    """
    rng = np.random.default_rng(seed)
    ga = {29: (2, 8), 64: (8, 16), 268: (3, 17)}
    out = []
    for i in range(n_agents):
        D = int(rng.choice([29, 64, 268]))
        G, A = ga[D]
        out.append(Workload(f"sweep_agent{i}", E=512, T=1000, D=D, A=A, G=G,
                            B=int(rng.choice([256, 512, 1024, 2048])), hidden=256, layers=2,
                            repr=int(rng.choice([64, 128])), seed=1000 + i))
    return out


def episode_done_flags(n, E, episode_len=None, mean_len=None, rng=None, start=0):
    """done [n][E] (uint8): fixed episode length, or geometric lengths with mean ``mean_len``."""
    done = np.zeros((n, E), dtype=np.uint8)
    if mean_len is None:
        steps = np.arange(start, start + n)
        done[(steps + 1) % episode_len == 0, :] = 1
        return done
    p = 1.0 / float(mean_len)
    for e in range(E):
        t = -1
        while True:
            t += int(rng.geometric(p))
            if t >= n:
                break
            done[t, e] = 1
    return done


def random_walk(E, n, D, A, done, seed, scale=0.1, dtype=np.float32):
    """obs [n][E][D], act [n][E][A]: random-walk states restarting after each ``done``."""
    rng = np.random.default_rng(seed)
    obs = np.empty((n, E, D), dtype=dtype)
    act = rng.uniform(-1.0, 1.0, size=(n, E, A)).astype(dtype)
    s = rng.standard_normal((E, D)).astype(dtype)
    for t in range(n):
        obs[t] = s
        step = (scale * rng.standard_normal((E, D))).astype(dtype)
        fresh = rng.standard_normal((E, D)).astype(dtype)
        s = np.where(done[t][:, None].astype(bool), fresh, s + step)
    return obs, act


def buffer_contents(w, n=None, mean_len=None, seed_offset=0):
    """(obs, act, done) time-major for ``n`` inserted steps of workload ``w``."""
    n = w.T if n is None else n
    rng = np.random.default_rng(w.seed * 7919 + 17 + seed_offset)
    done = episode_done_flags(n, w.E, w.episode_len, mean_len, rng)
    obs, act = random_walk(w.E, n, w.D, w.A, done, seed=w.seed * 7919 + 23 + seed_offset)
    return obs, act, done


def buffer_contents_device(w, n=None, seed_offset=0, device="cuda"):
    """The recipe of ``buffer_contents`` with fixed-length episodes, drawn on the
    device with a seeded torch generator (a different random stream from the
    numpy one; used to fill large buffers quickly, e.g. the 32-agent sweep).
    Returns device tensors obs [n][E][D], act [n][E][A], done [n][E] (uint8)."""
    import torch
    n = w.T if n is None else n
    g = torch.Generator(device=device)
    g.manual_seed(w.seed * 7919 + 29 + seed_offset)
    t = torch.arange(n, device=device)
    done = ((t + 1) % w.episode_len == 0).to(torch.uint8)[:, None].expand(n, w.E).contiguous()
    act = torch.rand((n, w.E, w.A), generator=g, device=device) * 2.0 - 1.0
    obs = torch.empty((n, w.E, w.D), device=device)
    for e0 in range(0, n, w.episode_len):
        e1 = min(n, e0 + w.episode_len)
        start = torch.randn((1, w.E, w.D), generator=g, device=device)
        steps = 0.1 * torch.randn((e1 - e0, w.E, w.D), generator=g, device=device)
        steps[0] = 0.0
        obs[e0:e1] = start + torch.cumsum(steps, dim=0)
    return obs, act, done


def network_shapes(w, net):
    """(in_dim, [hidden]*layers, out_dim) of phi, psi or pi."""
    ins = {"phi": w.D + w.A, "psi": w.G, "pi": w.D + w.G}[net]
    out = {"phi": w.repr, "psi": w.repr, "pi": 2 * w.A}[net]
    return ins, out


def init_network(w, net, seed, perturb=False, dtype=np.float32):
    """List of layer dicts {W [out][in], b[, ln_g, ln_b]}, hidden layers first."""
    rng = np.random.default_rng(seed)
    ins, out = network_shapes(w, net)
    dims = [ins] + [w.hidden] * w.layers + [out]
    layers = []
    for li in range(len(dims) - 1):
        fan_in, fan_out = dims[li], dims[li + 1]
        layer = {"W": (rng.standard_normal((fan_out, fan_in)) / np.sqrt(fan_in)).astype(dtype),
                 "b": np.zeros(fan_out, dtype=dtype)}
        if perturb:
            layer["b"] = (0.1 * rng.standard_normal(fan_out)).astype(dtype)
        if w.layernorm and li < len(dims) - 2:
            layer["ln_g"] = np.ones(fan_out, dtype=dtype)
            layer["ln_b"] = np.zeros(fan_out, dtype=dtype)
            if perturb:
                layer["ln_g"] = (1.0 + 0.1 * rng.standard_normal(fan_out)).astype(dtype)
                layer["ln_b"] = (0.1 * rng.standard_normal(fan_out)).astype(dtype)
        layers.append(layer)
    return layers


def init_agent(w, perturb=False):
    """Seeded phi, psi, pi networks of workload ``w``."""
    base = w.seed * 101
    return {net: init_network(w, net, base + i, perturb) for i, net in enumerate(("phi", "psi", "pi"))}


def actor_noise(B, A, seed):
    """eps [B][A] ~ N(0, I)."""
    return np.random.default_rng(seed).standard_normal((B, A)).astype(np.float32)


def representations(B, R, seed, dtype=np.float32):
    """phi, psi [B][R] ~ N(0, I) for tests of the energy / loss stage alone."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, R)).astype(dtype), rng.standard_normal((B, R)).astype(dtype)
