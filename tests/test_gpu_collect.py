"""GPU parity of the collection stub (crl_collect) against the oracle's restatement
of its synthetic dynamics: the slices it inserts, episode boundaries exactly, the
buffer it fills (relabel bit-exact on those slices), and the argument checks."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

from parity_helpers import small, to64

pytestmark = pytest.mark.gpu


def run(w, precision, n, L, calls=1):
    ctx = api.CRLContext(w, precision=precision, path="plain")
    nets = workload.init_agent(w, perturb=True)
    for k, v in nets.items():
        ctx.load_network(k, v)
    dev = ctx.device
    outs = []
    for _ in range(calls):
        o = (torch.zeros(n, w.E, w.D, device=dev), torch.zeros(n, w.E, w.A, device=dev),
             torch.zeros(n, w.E, dtype=torch.uint8, device=dev))
        ctx.collect(n, L, out=o)
        outs.append(o)
    torch.cuda.synchronize()
    obs = np.concatenate([o[0].cpu().numpy() for o in outs])
    act = np.concatenate([o[1].cpu().numpy() for o in outs])
    done = np.concatenate([o[2].cpu().numpy() for o in outs])
    return ctx, to64(nets), obs, act, done


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_collect_matches_oracle(precision):
    w = small(E=6, T=48, B=32)
    n, L = 25, 7
    ctx, nets, obs, act, done = run(w, precision, n, L)
    envs = oracle.collect.initial_envs(w.seed, 0, w.E, w.D, w.G)
    o_obs, o_act, o_done, _ = oracle.collect.collect(nets["pi"], envs, 0, n, L, w.seed, 0, w.A)
    np.testing.assert_array_equal(done, o_done)
    tol = 2e-6 if precision == "fp64" else 2e-5
    np.testing.assert_allclose(act, o_act, rtol=tol, atol=tol)
    np.testing.assert_allclose(obs, o_obs, rtol=tol, atol=tol)
    assert ctx.buffer_size() == (min(n, w.T), n)
    assert ctx.sync_status() == (0, 0)


def test_collect_in_several_calls_continues_the_same_stream():
    w = small(E=4, T=40, B=16)
    _, _, obs1, act1, done1 = run(w, "fp32", 12, 5, calls=1)
    _, _, obs2, act2, done2 = run(w, "fp32", 4, 5, calls=3)
    np.testing.assert_array_equal(obs1, obs2)
    np.testing.assert_array_equal(act1, act2)
    np.testing.assert_array_equal(done1, done2)


def test_collected_buffer_relabels_bit_exactly():
    """Relabel from the collected buffer against the oracle's relabel of the same
    slices: indices bit-exact and truncated at the stub's episode ends."""
    w = small(E=5, T=30, B=200)
    n, L = 45, 6                     # the ring wraps; every episode is 6 steps
    ctx, _, obs, act, done = run(w, "fp32", n, L)
    buf = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
    buf.insert(obs, act, done)
    table = oracle.relabel.geometric_table(w.gamma, w.T + 2)
    s, a, g, idx = ctx.sample(step=3, B=w.B)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    for b in range(w.B):
        e, t, v = oracle.relabel.draw_indices(w.seed, 0, 3, b, w.E, buf.size)
        k = oracle.relabel.truncated_geometric_offset(v, buf.horizon(e, t), table, 1)
        assert tuple(idx[b]) == (e, t, k)
        assert buf.horizon(e, t) <= L - 1
    np.testing.assert_array_equal(s.cpu().numpy(), buf.obs[idx[:, 0], idx[:, 1]])


def test_collect_errors():
    w = small(E=4, T=20, B=16)
    ctx = api.CRLContext(w)
    for k, v in workload.init_agent(w).items():
        ctx.load_network(k, v)
    with pytest.raises(api.CRLError) as e:
        ctx.collect(0, 5)
    assert e.value.code == api.E_INVALID_ARG
    with pytest.raises(api.CRLError) as e:
        ctx.collect(2, 0)
    assert e.value.code == api.E_INVALID_ARG
    host = np.zeros((2, w.E, w.D), dtype=np.float32)
    with pytest.raises(api.CRLError) as e:
        ctx.collect(2, 5, out=(host, None, None))
    assert e.value.code == api.E_INVALID_ARG
