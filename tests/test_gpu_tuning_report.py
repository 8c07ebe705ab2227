"""The tile autotuner's report (crl_gemm_tuning_report): after one critic and
one actor step with autotuning on, every grouped GEMM problem list the context
launched has one record; each record's pick is among its timed candidates and
is the fastest of them; the report is the same when read twice, and a buffer
shorter than the report is refused without being written."""

import ctypes

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
