"""The user-facing quick start: a BF16 fused context on the Ant workload, the
collection stub filling the buffer, update steps, and a checkpoint that a fresh
context resumes from."""

import math

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

pytestmark = pytest.mark.gpu


def test_quick_start_runs_and_resumes():
    w = workload.ANT_AUTOGRAD
    ctx = api.CRLContext(w, precision="bf16", path="fused")
    nets = workload.init_agent(w)
    for net, layers in nets.items():
        ctx.load_network(net, layers)
    ctx.collect(1000, episode_length=1000)
    assert ctx.buffer_size() == (w.T, w.T)
    loss = torch.zeros(6, device="cuda")
    for _ in range(3):
        ctx.update_step(loss_out=loss)
    torch.cuda.synchronize()
    parts = loss.cpu().numpy()
    assert np.all(np.isfinite(parts)) and parts[0] > 0.0
    assert ctx.sync_status() == (0, 0)
    state = ctx.save_state()
    saved = {n: {k: ctx.store[n][k].clone() for k in ("params", "grads", "adam_m", "adam_v")}
             for n in ("phi", "psi", "pi")}
    ctx.update_step(loss_out=loss)
    want = loss.cpu().numpy().copy()
    b = api.CRLContext(w, precision="bf16", path="fused")
    for n, d in saved.items():
        for k, v in d.items():
            b.store[n][k].copy_(v)
    b.load_state(state)
    b.update_step(loss_out=loss)
    np.testing.assert_array_equal(loss.cpu().numpy(), want)
    assert not math.isnan(b.get_alpha())
