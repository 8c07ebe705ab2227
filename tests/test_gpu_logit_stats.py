"""GPU parity of the logit statistics (crl_set_logit_stats / crl_get_logit_stats):
the mean positive and negative logits of a critic step against the oracle's
energy matrix of the same batch, on every precision and path; the update step
and a sweep agent against the same step taken one call at a time; off by
default."""

import math

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

from parity_helpers import hp, pick_step, setup, small

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-6, "fp32": 1e-5, "bf16": 2e-2}


def oracle_stats(w, nets, buf, step):
    s, a, g, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    _, _, _, phi, psi = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s, a, g, w.energy, h["tau"],
                                                         w.loss, w.sym_reduction, h["beta"], w.penalty_axis)
    F = oracle.critic.energy_matrix(phi, psi, w.energy, h["tau"])
    return oracle.critic.logit_stats(F), float(np.mean(np.abs(F)))


@pytest.mark.parametrize("precision,path", [("fp64", "plain"), ("fp32", "plain"), ("bf16", "plain"),
                                            ("bf16", "fused")])
@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
def test_critic_step_logit_stats_match_oracle(precision, path, energy):
    w = small(B=72, repr=64, energy=energy, tau=0.7 if energy == "cos" else 1.0)
    ctx, nets, buf = setup(w, precision=precision, path=path, n=60)
    assert all(math.isnan(v) for v in ctx.logit_stats())
    ctx.set_logit_stats(True)
    step = pick_step(w, nets, buf, 4)
    s, a, g, _ = ctx.sample(step=step)
    ctx.critic_step(s, a, g, apply_update=False)
    got = ctx.logit_stats()
    (d, o), scale = oracle_stats(w, nets, buf, step)
    tol = TOL[precision] * scale
    assert abs(got[0] - d) <= tol, (got, d)
    assert abs(got[1] - o) <= tol, (got, o)
    assert ctx.sync_status() == (0, 0)


def test_single_sample_has_no_negatives():
    w = small(B=1, hidden=33, repr=5)
    ctx, nets, buf = setup(w, precision="fp32", n=60)
    ctx.set_logit_stats(True)
    s, a, g, _ = ctx.sample(step=3, B=1)
    ctx.critic_step(s, a, g)
    d, o = ctx.logit_stats()
    assert math.isfinite(d) and math.isnan(o)


@pytest.mark.parametrize("precision,path", [("fp32", "plain"), ("bf16", "fused")])
def test_update_step_logit_stats_equal_separate_calls(precision, path):
    """Stats switched on after the update step was captured (the graph is rebuilt),
    then compared with sample + crl_critic_step on the same batch."""
    w = small(B=64, repr=64)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=7)
    got = []
    for fused in (True, False):
        ctx, _, _ = setup(w, precision=precision, path=path, n=60)
        hist = []
        for i in range(3):
            ins = [torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra]
            if i == 1:
                ctx.set_logit_stats(True)
            if fused:
                ctx.update_step(*ins, loss_out=torch.zeros(6, device=ctx.device))
            else:
                ctx.insert(*ins)
                s, a, g, _ = ctx.sample(step=i, B=w.B)
                ctx.critic_step(s, a, g, apply_update=True)
                ctx.actor_step(s, g, apply_update=True)
            hist.append(ctx.logit_stats())
        got.append(hist)
    assert all(math.isnan(v) for v in got[0][0])
    np.testing.assert_array_equal(np.array(got[0][1:]), np.array(got[1][1:]))
    assert got[0][1] != got[0][2]


def test_sweep_agent_logit_stats_equal_single_agent():
    ws = [workload.Workload(f"stats{i}", E=12, T=60, D=D, A=A, G=G, B=B, hidden=64, layers=2, repr=R, seed=40 + i)
          for i, (B, D, A, G, R) in enumerate([(64, 29, 8, 2, 64), (136, 64, 16, 8, 128)])]
    sw = api.CRLSweep(ws, "bf16", "fused", grouped=True)
    single = api.CRLContext(ws[1], "bf16", "fused", agent=1)
    for i, w in enumerate(ws):
        nets = workload.init_agent(w, perturb=True)
        obs, act, done = workload.buffer_contents(w, n=w.T, mean_len=9.0)
        for ctx in ([sw.agents[i], single] if i == 1 else [sw.agents[i]]):
            for k, v in nets.items():
                ctx.load_network(k, v)
            ctx.insert(*(torch.from_numpy(x).to(ctx.device) for x in (obs, act, done)))
    sw.agents[1].set_logit_stats(True)
    single.set_logit_stats(True)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        sw.update_step(loss_out=torch.zeros(2, 6, device="cuda"))
        single.update_step(loss_out=torch.zeros(6, device="cuda"))
    torch.cuda.synchronize()
    assert sw.agents[1].logit_stats() == single.logit_stats()
    assert all(math.isnan(v) for v in sw.agents[0].logit_stats())
    sw.close()
