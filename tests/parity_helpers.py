"""Shared setup for the GPU parity tests: the same seeded inputs go to the CUDA
path (through the C ABI) and to the FP64 oracle.

Two rules keep the comparisons meaningful:

* Hyperparameters reach the library as float32 (crl_config); the oracle gets
  those same float32 values (``hp``), so the FP64 path can be compared at
  ~1e-12 and not at the 1e-8 of a rounded 0.999.
* A ReLU mask is an integer decision taken by floating point.  A unit whose
  pre-activation lies within the FP32 rounding of zero may fall on either
  side in FP32 and in FP64, and one such flip moves a gradient tensor by
  ~1/sqrt(B H) -- far above 1e-4.  ``pick_step`` therefore picks the relabel
  step whose batch keeps every pre-activation at least 1e-5 (relative to the
  layer's RMS) away from zero, using the oracle's forward pass only.
"""

import numpy as np
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

# Tolerances of the parity contract (FP32 path vs the FP64 oracle):
# loss relative error <= 1e-5, gradient relative L2 error per tensor <= 1e-4.
FP32_LOSS_RTOL = 1e-5
FP32_GRAD_RTOL = 1e-4
# The FP64 GPU path differs from the oracle only by summation order; its loss
# leaves the C ABI as float32 (relative rounding <= 6e-8).
FP64_LOSS_RTOL = 1.2e-7
FP64_GRAD_RTOL = 1e-9
KINK_MARGIN = 1e-5


def f32(x):
    return float(np.float32(x))


def hp(w):
    """Hyperparameters exactly as the library holds them (float32)."""
    return {"tau": f32(w.tau), "beta": f32(w.beta), "alpha": f32(w.alpha), "gamma": f32(w.gamma),
            "lr_critic": f32(w.lr_critic), "lr_actor": f32(w.lr_actor),
            "adam_beta1": f32(0.9), "adam_beta2": f32(0.999), "adam_eps": f32(1e-8),
            "target_entropy": f32(-w.A if w.target_entropy is None else w.target_entropy),
            "lr_alpha": f32(w.lr_actor if w.lr_alpha is None else w.lr_alpha)}


def small(**kw):
    """A small workload whose sizes are ragged against the 64-wide GEMM tiles."""
    base = dict(E=6, T=48, D=29, A=8, G=2, B=96, hidden=80, layers=2, repr=24, seed=21)
    base.update(kw)
    return workload.Workload("parity", **base)


def to64(nets):
    return {k: [{kk: vv.astype(np.float64) for kk, vv in l.items()} for l in v] for k, v in nets.items()}


def setup(w, precision="fp32", n=None, mean_len=9.0, agent=0, offset_min=1, perturb=True, nets=None, path="plain",
          **over):
    """Context with seeded networks and buffer; the oracle's buffer and networks alongside."""
    ctx = api.CRLContext(w, precision=precision, path=path, agent=agent, offset_min=offset_min, **over)
    nets = workload.init_agent(w, perturb=perturb) if nets is None else nets
    for k, v in nets.items():
        ctx.load_network(k, v)
    obs, act, done = workload.buffer_contents(w, n=n, mean_len=mean_len)
    dev = ctx.device
    ctx.insert(torch.from_numpy(obs).to(dev), torch.from_numpy(act).to(dev), torch.from_numpy(done).to(dev))
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    buf.insert(obs, act, done)
    return ctx, to64(nets), buf


def kink_margin(net, x):
    """min over hidden units of |pre-activation| / RMS of its layer (oracle forward)."""
    _, cache = oracle.mlp.forward(net, x)
    m = np.inf
    for c in cache[:-1]:
        u = c["u"]
        m = min(m, float(np.abs(u).min() / np.sqrt((u ** 2).mean())))
    return m


def batch_margin(w, nets, s, a, g, eps=None):
    m = min(kink_margin(nets["phi"], np.concatenate([s, a], 1)), kink_margin(nets["psi"], g))
    if eps is not None:
        out, _ = oracle.mlp.forward(nets["pi"], np.concatenate([s, g], 1))
        a_new, _, _ = oracle.actor.policy_head(out, eps)
        m = min(m, kink_margin(nets["pi"], np.concatenate([s, g], 1)),
                kink_margin(nets["phi"], np.concatenate([s, a_new], 1)))
    return m


def pick_step(w, nets, buf, start=0, eps=None, tries=64, offset_min=1):
    """First relabel step >= start whose batch is kink-free (see the module docstring)."""
    best, best_m = start, -1.0
    for step in range(start, start + tries):
        s, a, g, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma, offset_min)
        m = batch_margin(w, nets, s, a, g, eps)
        if m >= KINK_MARGIN:
            return step
        if m > best_m:
            best, best_m = step, m
    raise AssertionError(f"no kink-free batch in {tries} steps (best margin {best_m:.2e} at step {best})")


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def assert_grads_close(got_net, ref_net, rtol, label=""):
    worst = 0.0
    for li, (g, r) in enumerate(zip(got_net, ref_net)):
        assert set(g) == set(r)
        for k in r:
            e = rel_err(g[k], r[k])
            worst = max(worst, e)
            assert e <= rtol, f"{label} layer {li} {k}: relative error {e:.3e} > {rtol:.1e}"
    return worst


def assert_scalar_close(got, ref, rtol, label="", atol=0.0):
    err = abs(float(got) - float(ref))
    assert err <= rtol * abs(float(ref)) + atol, f"{label}: {got} vs {ref} (abs error {err:.3e})"
    return err
