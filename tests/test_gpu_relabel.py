"""GPU parity of buffer insert + sample/relabel against the oracle: bit-exact (e, t, k),
exact s, a, g; ring wrap-around, short episodes, offset_min, gamma edge cases, full sizes."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

from parity_helpers import setup, small

pytestmark = pytest.mark.gpu


def compare(ctx, buf, w, step, B, offset_min=1, agent=0, sample_rows=None):
    s, a, g, idx = ctx.sample(step=step, B=B)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    s, a, g = s.cpu().numpy(), a.cpu().numpy(), g.cpu().numpy()
    rows = range(B) if sample_rows is None else sample_rows
    table = oracle.relabel.geometric_table(w.gamma, w.T + 2)
    for b in rows:
        e, t, v = oracle.relabel.draw_indices(w.seed, agent, step, b, w.E, buf.size)
        k = oracle.relabel.truncated_geometric_offset(v, buf.horizon(e, t), table, offset_min)
        assert tuple(idx[b]) == (e, t, k), (b, tuple(idx[b]), (e, t, k))
        np.testing.assert_array_equal(s[b], buf.obs[e, t].astype(np.float32))
        np.testing.assert_array_equal(a[b], buf.act[e, t].astype(np.float32))
        np.testing.assert_array_equal(g[b], buf.obs[e, t + k, list(w.goals())].astype(np.float32))
    return idx


@pytest.mark.parametrize("gamma", [0.0, 0.9, 0.99])
@pytest.mark.parametrize("offset_min", [1, 0])
def test_relabel_bit_exact_small(gamma, offset_min):
    w = small(gamma=gamma, B=200, G=3, goal_idx=(5, 0, 28))
    ctx, _, buf = setup(w, n=130, mean_len=7.0, offset_min=offset_min)   # 130 > T = 48: the ring wraps
    assert ctx.buffer_size() == (48, 130)
    for step in (0, 1, 12345, 2 ** 40 + 3):
        compare(ctx, buf, w, step, 200, offset_min)
    assert ctx.sync_status() == (0, 0)


def test_relabel_insert_in_chunks_and_single_steps():
    w = small(B=150)
    obs, act, done = workload.buffer_contents(w, n=75, mean_len=5.0)
    ctx = api.CRLContext(w)
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    dev = ctx.device
    for lo, hi in ((0, 1), (1, 30), (30, 31), (31, 75)):
        ctx.insert(torch.from_numpy(obs[lo:hi]).to(dev), torch.from_numpy(act[lo:hi]).to(dev),
                   torch.from_numpy(done[lo:hi]).to(dev))
        buf.insert(obs[lo:hi], act[lo:hi], done[lo:hi])
        compare(ctx, buf, w, hi, 150)


def test_relabel_host_pointer_insert_matches_device_insert():
    w = small(B=64)
    obs, act, done = workload.buffer_contents(w, n=60, mean_len=6.0)
    ctx = api.CRLContext(w)
    ctx.insert(obs, act, done)                       # numpy arrays: host pointers, staged by the library
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    buf.insert(obs, act, done)
    compare(ctx, buf, w, 9, 64)


def test_auto_step_counter():
    w = small(B=32)
    ctx, _, buf = setup(w, n=40)
    ctx.set_step(100)
    _, _, _, i1 = ctx.sample(step=api.STEP_AUTO, B=32)
    _, _, _, i2 = ctx.sample(step=api.STEP_AUTO, B=32)
    _, _, _, r1 = ctx.sample(step=100, B=32)
    _, _, _, r2 = ctx.sample(step=101, B=32)
    torch.cuda.synchronize()
    assert torch.equal(i1, r1) and torch.equal(i2, r2)
    assert ctx.get_step() == 102


def test_relabel_errors():
    w = small(B=32)
    ctx = api.CRLContext(w)
    with pytest.raises(api.CRLError) as e:
        ctx.sample(step=0, B=32)
    assert e.value.code == api.E_BUFFER_EMPTY
    ctx, _, _ = setup(w, n=10)
    one = [torch.empty(1, n, dtype=torch.float32, device=ctx.device) for n in (w.D, w.A, w.G)]
    with pytest.raises(api.CRLError) as e:
        ctx.sample(step=0, B=0, out=(*one, None))
    assert e.value.code == api.E_SHAPE


def test_relabel_full_size_ant_config():
    """1024 envs x 1000 steps, batch 256: every sample of the launch bench.py times."""
    w = workload.ANT_AUTOGRAD
    ctx, _, buf = setup(w, perturb=False, mean_len=None)
    for step in (0, 7):
        compare(ctx, buf, w, step, w.B)


def test_relabel_full_size_large_batch_sampled_rows():
    """4096 envs x 500 steps, episodes of 500, batch 8192: 1024 sampled rows of the launch."""
    w = workload.LARGE_BATCH
    ctx, _, buf = setup(w, perturb=False, mean_len=None)
    rows = list(range(0, w.B, 8))
    compare(ctx, buf, w, 3, w.B, sample_rows=rows)


def test_relabel_batch_larger_than_config():
    """A standalone sample may exceed the configured batch (the outputs are the
    caller's): 5000 samples on a context built for 32, every row checked."""
    w = small(B=32)
    ctx, _, buf = setup(w, n=90, mean_len=6.0)
    compare(ctx, buf, w, 77, 5000)
    assert ctx.sync_status() == (0, 0)


def test_relabel_throughput_shapes_sampled():
    """The relabel throughput measurement's launch: Humanoid-shaped rows (obs 268,
    action 17, goal 3), 1024 envs x 1000 steps, 2^20 samples; 2000 rows checked."""
    w = workload.Workload("relabel", E=1024, T=1000, D=268, A=17, G=3, B=256, hidden=64, layers=1, repr=64,
                          seed=5)
    ctx, _, buf = setup(w, perturb=False, mean_len=None)
    rows = np.random.default_rng(3).choice(1 << 20, 2000, replace=False)
    compare(ctx, buf, w, 4242, 1 << 20, sample_rows=rows)
    assert ctx.sync_status() == (0, 0)
