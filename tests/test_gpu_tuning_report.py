"""The tile autotuner's report (crl_gemm_tuning_report): after one critic and
one actor step with autotuning on, every grouped GEMM problem list the context
launched has one record; each record's pick is among its timed candidates and
is the fastest of them; the report is the same when read twice, and a buffer
shorter than the report is refused without being written.  And the pick never
changes an output: a tuned context and one on the fixed rule agree bit for bit."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2408_11052_gb300 import api, workload

from parity_helpers import setup, small

pytestmark = pytest.mark.gpu


def test_report_lists_every_tuned_problem_list_with_its_fastest_candidate():
    w = small(B=256, hidden=256, repr=64, E=8, T=200)
    prev = api.set_autotune(True)
    try:
        ctx, _, _ = setup(w, precision="bf16", path="fused", n=150, mean_len=30.0)
        s, a, g, _ = ctx.sample(step=3)
        eps = torch.from_numpy(workload.actor_noise(w.B, w.A, 5)).to(ctx.device)
        ctx.critic_step(s, a, g, apply_update=False)
        ctx.actor_step(s, g, eps, apply_update=False)
        torch.cuda.synchronize()
        assert ctx.sync_status() == (0, 0)
        rep = api.gemm_tuning_report(ctx.handle)
        assert len(rep) >= 4          # forward layers, input gradients, weight gradients at least
        for r in rep:
            assert r["problems"] >= 1 and r["gflop"] > 0 and len(r["first_mnk"]) == 3
            timed = {k: v for k, v in r["us"].items() if v >= 0}
            assert r["picked"] in timed
            assert timed[r["picked"]] == min(timed.values())
        assert api.gemm_tuning_report(ctx.handle) == rep

        need = ctypes.c_size_t()
        api.check(api.lib().crl_gemm_tuning_report(ctx.handle, None, 0, ctypes.byref(need)), ctx.handle)
        short = ctypes.create_string_buffer(b"x" * 7, need.value - 1)
        rc = api.lib().crl_gemm_tuning_report(ctx.handle, short, need.value - 1, ctypes.byref(need))
        assert rc == api.E_SHAPE and short.raw[:7] == b"x" * 7
    finally:
        api.set_autotune(prev)


def test_outputs_do_not_depend_on_the_tuners_pick():
    """At batch 4096 the weight gradients split the batch over several CTAs.
    The split follows from the problem's shape alone and such a launch is tuned
    over the one-tile kernel only, so a context that autotunes and one that runs
    the fixed rule give the same bits: critic and actor gradients, and the
    parameters after two update steps."""
    w = small(B=4096, hidden=256, repr=64, E=8, T=400)
    prev = api.set_autotune(True)
    try:
        results = []
        for tune in (True, False):
            api.set_autotune(tune)
            ctx, _, _ = setup(w, precision="bf16", path="fused", n=300, mean_len=60.0)
            s, a, g, _ = ctx.sample(step=3)
            eps = torch.from_numpy(workload.actor_noise(w.B, w.A, 5)).to(ctx.device)
            ctx.critic_step(s, a, g, apply_update=False)
            ctx.actor_step(s, g, eps, apply_update=False)
            torch.cuda.synchronize()
            grads = {n: ctx.store[n]["grads"].cpu().numpy().copy() for n in ("phi", "psi", "pi")}
            loss = torch.zeros(6, device=ctx.device)
            for _ in range(2):
                ctx.update_step(loss_out=loss)
            torch.cuda.synchronize()
            assert ctx.sync_status() == (0, 0)
            params = {n: ctx.store[n]["params"].cpu().numpy().copy() for n in ("phi", "psi", "pi")}
            splits = [r for r in api.gemm_tuning_report(ctx.handle) if r["first_mnk"][2] == w.B]
            results.append((grads, params, loss.cpu().numpy().copy(), splits))
        (g_t, p_t, l_t, rep), (g_f, p_f, l_f, _) = results
        assert rep and all(r["picked"].startswith("one_tile") for r in rep)   # the weight-gradient lists
        for n in ("phi", "psi", "pi"):
            np.testing.assert_array_equal(g_t[n], g_f[n], err_msg=n)
            np.testing.assert_array_equal(p_t[n], p_f[n], err_msg=n)
        np.testing.assert_array_equal(l_t, l_f)
    finally:
        api.set_autotune(prev)
