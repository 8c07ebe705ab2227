"""Batched sweep: each agent of a sweep (one launch per kernel over all agents,
or the agents' steps one after another) matches the same agent run alone
through crl_update_step, bit for bit, over several steps -- the first eager,
the later ones replayed from the captured graph."""

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

pytestmark = pytest.mark.gpu


def uneven_agents(n_buffer_steps=60):
    """Agents with uneven batch, obs / action / goal dims and repr; shared hidden width and depth."""
    specs = [(64, 29, 8, 2, 64), (136, 64, 16, 8, 128), (32, 268, 17, 3, 64), (256, 29, 8, 2, 128)]
    return [workload.Workload(f"sweep_test{i}", E=12, T=n_buffer_steps, D=D, A=A, G=G, B=B, hidden=64, layers=2,
                              repr=R, seed=40 + i)
            for i, (B, D, A, G, R) in enumerate(specs)]


def fill(ctx, w, n, seed_offset):
    obs, act, done = workload.buffer_contents(w, n=n, mean_len=9.0, seed_offset=seed_offset)
    ctx.insert(*(torch.from_numpy(x).to(ctx.device) for x in (obs, act, done)))


def run_and_compare(ws, precision, path, grouped, steps=4, check=None, pinned=False):
    sw = api.CRLSweep(ws, precision, path, grouped=grouped)
    check = range(len(ws)) if check is None else check
    singles = {i: api.CRLContext(ws[i], precision, path, agent=i) for i in check}
    for i, w in enumerate(ws):
        nets = workload.init_agent(w, perturb=True)
        for k, v in nets.items():
            sw.agents[i].load_network(k, v)
            if i in singles:
                singles[i].load_network(k, v)
        fill(sw.agents[i], w, w.T, 0)
        if i in singles:
            fill(singles[i], w, w.T, 0)
    extra = [workload.buffer_contents(w, n=steps, mean_len=9.0, seed_offset=7) for w in ws]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    loss_sw = torch.zeros(len(ws), 6, dtype=torch.float32, device="cuda")
    loss_1 = torch.zeros(6, dtype=torch.float32, device="cuda")
    hist_sw, hist_1 = [], {i: [] for i in singles}
    with torch.cuda.stream(stream):
        for t in range(steps):
            ins = [[torch.from_numpy(np.ascontiguousarray(x[t:t + 1])).pin_memory() if pinned
                    else torch.from_numpy(x[t:t + 1]).cuda() for x in extra[i]] for i in range(len(ws))]
            sw.update_step([a[0] for a in ins], [a[1] for a in ins], [a[2] for a in ins], loss_out=loss_sw)
            hist_sw.append(loss_sw.cpu().numpy().copy())
        for i, ctx in singles.items():
            for t in range(steps):
                ctx.update_step(*(torch.from_numpy(x[t:t + 1]).cuda() for x in extra[i]), loss_out=loss_1)
                hist_1[i].append(loss_1.cpu().numpy().copy())
    torch.cuda.synchronize()
    assert sw.sync_status() == (0, 0)
    for i, ctx in singles.items():
        assert ctx.sync_status() == (0, 0)
        got = np.array([h[i] for h in hist_sw])
        assert np.all(np.isfinite(got))
        np.testing.assert_array_equal(got, np.array(hist_1[i]), err_msg=f"agent {i} losses")
        for net in ("phi", "psi", "pi"):
            for which in ("params", "adam_m", "adam_v"):
                a = sw.agents[i].store[net][which].cpu().numpy()
                b = ctx.store[net][which].cpu().numpy()
                np.testing.assert_array_equal(a, b, err_msg=f"agent {i} {net} {which}")
        assert sw.agents[i].get_step() == ctx.get_step() == steps
        assert sw.agents[i].get_alpha() == ctx.get_alpha()
    sw.close()


def test_grouped_sweep_matches_single_agents():
    run_and_compare(uneven_agents(), "bf16", "fused", grouped=True)


def test_grouped_sweep_with_pinned_host_inputs_matches_single_agents():
    """Pinned host inputs of every agent, read in place by the grouped insert."""
    run_and_compare(uneven_agents(), "bf16", "fused", grouped=True, steps=3, pinned=True)


def test_sequential_sweep_matches_single_agents_fp32():
    run_and_compare(uneven_agents(), "fp32", "plain", grouped=False, steps=3)


def test_sequential_bf16_sweep_matches_single_agents():
    run_and_compare(uneven_agents()[:2], "bf16", "fused", grouped=False, steps=3)


def test_grouped_sweep_with_alpha_autotune():
    """Agents that tune their entropy coefficient (one of them with a fixed one)."""
    ws = [w.with_(alpha_autotune=(i != 2), lr_alpha=0.05, target_entropy=-2.0 - i) for i, w in enumerate(uneven_agents())]
    run_and_compare(ws, "bf16", "fused", grouped=True, steps=3)


def test_grouped_sweep_with_mixed_objectives():
    """An objective sweep (§5.2) in one grouped sweep: the backward runs one launch
    per objective kind over its agents."""
    ws = [w.with_(loss=l) for w, l in zip(uneven_agents(), ("dpo", "sym", "fb", "ipo"))]
    run_and_compare(ws, "bf16", "fused", grouped=True, steps=3)


def test_grouped_sweep_with_random_goal_mix():
    """Agents whose actors take another sample's goal with probability alpha_rg (the
    random-goal actor mix, App. D) beside agents without it: each matches its own
    single-agent run."""
    ws = [w.with_(alpha_rg=a) for w, a in zip(uneven_agents(), (0.5, 0.0, 1.0, 0.25))]
    run_and_compare(ws, "bf16", "fused", grouped=True, steps=3)


def test_grouped_sweep_with_l1_agents():
    """-L1 agents (their own SIMT energy launches) beside tcgen05 ones in one grouped sweep."""
    ws = [w.with_(energy=e, loss=l) for w, e, l in zip(uneven_agents(), ("l1", "l2", "l1", "cos"),
                                                       ("sym", "fwd", "dpo", "sym"))]
    run_and_compare(ws, "bf16", "fused", grouped=True, steps=3)


def test_grouped_sweep_of_32_agents_sampled():
    """The 32-agent sweep workload's shapes (batch 256..2048, obs 29 / 64 / 268,
    repr 64 / 128, 512 envs), short buffers; agents 0, 13 and 31 checked."""
    ws = [w.with_(T=80) for w in workload.sweep_agents(32)]
    run_and_compare(ws, "bf16", "fused", grouped=True, steps=3, check=[0, 13, 31])


def test_sweep_rejects_mismatched_agents():
    ws = uneven_agents()[:2]
    bad = [ws[0], ws[1].with_(hidden=128)]
    with pytest.raises(api.CRLError) as e:
        api.CRLSweep(bad, "bf16", "fused", grouped=True)
    assert e.value.code == api.E_INVALID_ARG
    with pytest.raises(api.CRLError) as e:
        api.CRLSweep(ws, "fp32", "plain", grouped=True)
    assert e.value.code == api.E_UNSUPPORTED

