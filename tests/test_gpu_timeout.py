"""Failure detection without a GPU fault: the bounded device waits of the
tensor-core kernels (grouped GEMMs: one-tile, persistent and CTA-pair; the
fused energy stage).  A wait limit of one nanosecond makes the waits run out on
purpose: the step must return, crl_sync_status must report CRL_E_TIMEOUT, and
after the limit is restored the same context must give exactly the results of
a step that never timed out (the kernels drained their own copies and MMAs,
freed their tensor memory and left every ticket consistent)."""

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

from parity_helpers import setup, small

pytestmark = pytest.mark.gpu

STATUS_TIMEOUT = 4     # CRL_STATUS_TIMEOUT


def critic_and_actor(ctx, s, a, g, eps):
    lc = ctx.critic_step(s, a, g, apply_update=False)
    la = ctx.actor_step(s, g, eps, apply_update=False)
    torch.cuda.synchronize()
    grads = {n: ctx.store[n]["grads"].cpu().numpy().copy() for n in ("phi", "psi", "pi")}
    return lc.cpu().numpy().copy(), la.cpu().numpy().copy(), grads


@pytest.mark.parametrize("kernel", ["one_tile", "persistent", "cta_pair"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_waits_run_out_and_the_context_stays_usable(kernel, layernorm):
    w = small(B=256, hidden=256, repr=64, E=8, T=200, layernorm=layernorm)
    prev_kernel = api.set_gemm_kernel(kernel)
    prev_tune = api.set_autotune(False)
    try:
        ctx, _, _ = setup(w, precision="bf16", path="fused", n=150, mean_len=30.0)
        s, a, g, _ = ctx.sample(step=3)
        eps = torch.from_numpy(workload.actor_noise(w.B, w.A, 5)).to(ctx.device)
        ref = critic_and_actor(ctx, s, a, g, eps)
        assert ctx.sync_status() == (0, 0)

        ctx.set_wait_limit_ns(1)
        critic_and_actor(ctx, s, a, g, eps)            # returns: every wait is bounded
        rc, status = ctx.sync_status()
        assert rc == api.E_TIMEOUT and status & STATUS_TIMEOUT
        assert "wait" in api.lib().crl_last_error(ctx.handle).decode()

        ctx.set_wait_limit_ns(0)
        for _ in range(2):                             # the same context, the default limit
            got = critic_and_actor(ctx, s, a, g, eps)
            assert ctx.sync_status() == (0, 0)
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])
            for n in ("phi", "psi", "pi"):
                np.testing.assert_array_equal(got[2][n], ref[2][n], err_msg=n)
    finally:
        api.set_gemm_kernel(prev_kernel)
        api.set_autotune(prev_tune)


def test_update_step_graph_sees_the_limit_on_replay():
    """The limit lives in device memory next to the status word: a captured
    update step replays with the new limit, and with the default again after it."""
    w = small(B=128, hidden=128, repr=64, E=8, T=200)
    ctx, _, _ = setup(w, precision="bf16", path="fused", n=150, mean_len=30.0)
    loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    extra = workload.buffer_contents(w, n=6, mean_len=9.0, seed_offset=3)
    stream = torch.cuda.Stream(device=ctx.device)
    with torch.cuda.stream(stream):
        for i in range(2):                              # the second call captures the graph
            ctx.update_step(*(torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra), loss_out=loss,
                            stream=stream)
    stream.synchronize()
    assert ctx.sync_status(stream) == (0, 0)
    ctx.set_wait_limit_ns(1)
    with torch.cuda.stream(stream):
        ctx.update_step(*(torch.from_numpy(x[2:3]).to(ctx.device) for x in extra), loss_out=loss, stream=stream)
    rc, status = ctx.sync_status(stream)
    assert rc == api.E_TIMEOUT and status & STATUS_TIMEOUT
    ctx.set_wait_limit_ns(0)
    with torch.cuda.stream(stream):
        ctx.update_step(*(torch.from_numpy(x[3:4]).to(ctx.device) for x in extra), loss_out=loss, stream=stream)
    assert ctx.sync_status(stream) == (0, 0)
