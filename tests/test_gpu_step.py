"""Full update steps (insert -> relabel -> critic + Adam -> actor + Adam) through
crl_update_step against the oracle's update step, and the status / error paths."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import api, workload

from parity_helpers import KINK_MARGIN, batch_margin, hp, setup, small

pytestmark = pytest.mark.gpu


def oracle_steps(w, nets, buf, n_steps, start_step, inserts, check_kinks=False):
    """Run the oracle's update step n_steps times; with check_kinks, None if a batch is near a kink."""
    h = hp(w)
    state = oracle.step.AgentState(nets["phi"], nets["psi"], nets["pi"])
    cfg = dict(seed=w.seed, agent=0, B=w.B, goal_idx=w.goals(), gamma=w.gamma, energy=w.energy, tau=h["tau"],
               loss=w.loss, sym_reduction=w.sym_reduction, beta=h["beta"], penalty_axis=w.penalty_axis,
               alpha=h["alpha"], lr_critic=h["lr_critic"], lr_actor=h["lr_actor"], adam_beta1=h["adam_beta1"],
               adam_beta2=h["adam_beta2"], adam_eps=h["adam_eps"], alpha_autotune=w.alpha_autotune,
               target_entropy=h["target_entropy"], lr_alpha=h["lr_alpha"], alpha_rg=float(np.float32(w.alpha_rg)))
    outs = []
    for i in range(n_steps):
        buf.insert(*inserts[i])
        eps = oracle.actor.gaussian_noise(w.seed, 0, start_step + i, w.B, w.A)
        if check_kinks:
            s, a, g, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, start_step + i, w.B, w.goals(), w.gamma)
            pre = {"phi": state.nets["phi"], "psi": state.nets["psi"], "pi": state.nets["pi"]}
            if batch_margin(w, pre, s, a, g, eps) < KINK_MARGIN:
                return None
        outs.append(oracle.step.update_step(state, buf, cfg, start_step + i, eps))
    return state, outs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("host_inputs", [False, True])
def test_update_steps_match_oracle(precision, host_inputs):
    w = small(B=64)
    ctx, nets, buf = setup(w, precision=precision, n=60)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=99)
    inserts = [tuple(x[i:i + 1] for x in extra) for i in range(3)]
    start = None
    for cand in range(0, 48):
        trial = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
        trial.obs, trial.act, trial.done = buf.obs.copy(), buf.act.copy(), buf.done.copy()
        if oracle_steps(w, nets, trial, 3, cand, inserts, check_kinks=True) is not None:
            start = cand
            break
    assert start is not None
    ctx.set_step(start)
    kw = dict(dtype=torch.float32)
    loss_out = torch.zeros(6, **kw) if host_inputs else torch.zeros(6, device=ctx.device, **kw)
    losses = []
    for obs, act, done in inserts:
        if host_inputs:
            ctx.update_step(obs, act, done, loss_out=loss_out)
        else:
            d = ctx.device
            ctx.update_step(torch.from_numpy(obs).to(d), torch.from_numpy(act).to(d), torch.from_numpy(done).to(d),
                            loss_out=loss_out)
        torch.cuda.synchronize()
        losses.append(loss_out.cpu().numpy().astype(np.float64).copy())
    state, outs = oracle_steps(w, nets, buf, 3, start, inserts)
    rtol = 1.2e-7 if precision == "fp64" else 2e-4
    for got, ref in zip(losses, outs):
        c = ref["critic"]
        np.testing.assert_allclose(got[:4], [c["total"], c["fwd"], c["bwd"], c["penalty"]], rtol=rtol, atol=1e-7)
        np.testing.assert_allclose(got[4:6], [ref["actor_loss"], ref["logpi_mean"]], rtol=rtol, atol=1e-6)
    # Parameters after three Adam steps.  FP32: Adam's first steps move every weight by
    # about lr * sign(g), so coordinates whose true gradient is near zero may move the
    # other way; allow 2 lr there and 1e-3 lr elsewhere.
    for net in ("phi", "psi", "pi"):
        lr = w.lr_actor if net == "pi" else w.lr_critic
        for gl, rl in zip(ctx.network(net), state.nets[net]):
            for k in rl:
                if precision == "fp64":
                    np.testing.assert_allclose(gl[k], rl[k], rtol=1e-9, atol=1e-12)
                else:
                    err = np.abs(gl[k] - rl[k])
                    assert np.mean(err <= 1e-3 * lr + 1e-7) > 0.98, (net, k)
                    assert err.max() <= 6 * lr + 1e-6, (net, k)
    assert ctx.sync_status() == (0, 0)
    assert ctx.get_step() == start + 3


@pytest.mark.parametrize("loss", ["dpo", "fb", "flatnce_bwd"])
def test_update_steps_with_other_objectives_match_oracle(loss):
    """Three full FP64 update steps with an objective outside InfoNCE."""
    w = small(B=48, loss=loss)
    ctx, nets, buf = setup(w, precision="fp64", n=60)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=5)
    inserts = [tuple(x[i:i + 1] for x in extra) for i in range(3)]
    start = None
    for cand in range(0, 48):
        trial = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
        trial.obs, trial.act, trial.done = buf.obs.copy(), buf.act.copy(), buf.done.copy()
        if oracle_steps(w, nets, trial, 3, cand, inserts, check_kinks=True) is not None:
            start = cand
            break
    assert start is not None
    ctx.set_step(start)
    loss_out = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    got = []
    for ins in inserts:
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in ins), loss_out=loss_out)
        got.append(loss_out.cpu().numpy().astype(np.float64).copy())
    state, outs = oracle_steps(w, nets, buf, 3, start, inserts)
    for g, ref in zip(got, outs):
        c = ref["critic"]
        np.testing.assert_allclose(g[:4], [c["total"], c["fwd"], c["bwd"], c["penalty"]], rtol=1.2e-7, atol=1e-7)
        np.testing.assert_allclose(g[4:6], [ref["actor_loss"], ref["logpi_mean"]], rtol=1.2e-7, atol=1e-6)
    for net in ("phi", "psi", "pi"):
        for gl, rl in zip(ctx.network(net), state.nets[net]):
            for k in rl:
                np.testing.assert_allclose(gl[k], rl[k], rtol=1e-9, atol=1e-12)
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("precision,path", [("fp64", "plain"), ("fp32", "plain"), ("bf16", "plain"),
                                            ("bf16", "fused")])
@pytest.mark.parametrize("alpha_rg", [0.5, 1.0])
def test_random_goal_mix_matches_oracle(precision, path, alpha_rg):
    """Random-goal actor mix (App. D): three update steps against the oracle's; the
    critic parts keep the relabelled goals, the actor takes the mixed ones."""
    w = small(B=64, repr=64, alpha_rg=alpha_rg)
    ctx, nets, buf = setup(w, precision=precision, path=path, n=60)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=11)
    inserts = [tuple(x[i:i + 1] for x in extra) for i in range(3)]
    start = 0
    if precision != "bf16":
        start = None
        for cand in range(0, 48):
            trial = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
            trial.obs, trial.act, trial.done = buf.obs.copy(), buf.act.copy(), buf.done.copy()
            if oracle_steps(w, nets, trial, 3, cand, inserts, check_kinks=True) is not None:
                start = cand
                break
        assert start is not None
    ctx.set_step(start)
    loss_out = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    got = []
    for ins in inserts:
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in ins), loss_out=loss_out)
        got.append(loss_out.cpu().numpy().astype(np.float64).copy())
    _, outs = oracle_steps(w, nets, buf, 3, start, inserts)
    rtol = {"fp64": 1.2e-7, "fp32": 2e-4, "bf16": 2e-2}[precision]
    for g, ref in zip(got, outs):
        np.testing.assert_allclose(g[0], ref["critic"]["total"], rtol=rtol)
        np.testing.assert_allclose(g[4:6], [ref["actor_loss"], ref["logpi_mean"]], rtol=rtol, atol=1e-6)
    assert ctx.sync_status() == (0, 0)


def test_random_goal_mix_changes_only_the_actor():
    """Same seeds with and without the mix: identical critic losses, different actor loss."""
    out = {}
    for a_rg in (0.0, 0.7):
        w = small(B=64, alpha_rg=a_rg)
        ctx, _, _ = setup(w, n=60)
        loss_out = torch.zeros(6, dtype=torch.float32, device=ctx.device)
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in workload.buffer_contents(w, n=1, seed_offset=3)),
                        loss_out=loss_out)
        out[a_rg] = loss_out.cpu().numpy()
    np.testing.assert_array_equal(out[0.0][:4], out[0.7][:4])
    assert out[0.0][4] != out[0.7][4]


@pytest.mark.parametrize("precision,path", [("fp64", "plain"), ("fp32", "plain"), ("bf16", "plain"),
                                            ("bf16", "fused")])
def test_alpha_autotune_matches_oracle(precision, path):
    """Entropy-coefficient auto-tuning: the alpha each actor loss uses, the alpha after
    each step, the losses and the policy after four steps against the oracle's step.
    lr_alpha 0.05 moves alpha by about 5 % a step, so a wrong alpha shows in the loss."""
    w = small(B=64, repr=64, alpha_autotune=True, target_entropy=-3.0, lr_alpha=0.05)
    ctx, nets, buf = setup(w, precision=precision, path=path, n=60)
    n_steps = 4
    extra = workload.buffer_contents(w, n=n_steps, mean_len=9.0, seed_offset=99)
    inserts = [tuple(x[i:i + 1] for x in extra) for i in range(n_steps)]
    start = 0
    if precision != "bf16":
        start = None
        for cand in range(0, 48):
            trial = oracle.relabel.ReplayBuffer(w.E, w.T, w.D, w.A)
            trial.obs, trial.act, trial.done = buf.obs.copy(), buf.act.copy(), buf.done.copy()
            if oracle_steps(w, nets, trial, n_steps, cand, inserts, check_kinks=True) is not None:
                start = cand
                break
        assert start is not None
    ctx.set_step(start)
    assert ctx.get_alpha() == pytest.approx(w.alpha, rel=1e-7)
    loss_out = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    losses, alphas = [], []
    for obs, act, done in inserts:
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in (obs, act, done)), loss_out=loss_out)
        torch.cuda.synchronize()
        losses.append(loss_out.cpu().numpy().astype(np.float64).copy())
        alphas.append(ctx.get_alpha())
    state, outs = oracle_steps(w, nets, buf, n_steps, start, inserts)
    assert len({round(o["alpha"], 6) for o in outs}) == n_steps          # alpha really moves
    rtol = {"fp64": 1e-7, "fp32": 2e-4, "bf16": 2e-2}[precision]
    arel = {"fp64": 1e-7, "fp32": 1e-5, "bf16": 1e-3}[precision]
    for got, ref, a in zip(losses, outs, alphas):
        np.testing.assert_allclose(got[4:6], [ref["actor_loss"], ref["logpi_mean"]], rtol=rtol, atol=1e-6 + rtol * 1e-2)
        assert a == pytest.approx(ref["alpha_next"], rel=arel)
    if precision != "bf16":
        for gl, rl in zip(ctx.network("pi"), state.nets["pi"]):
            for k in rl:
                if precision == "fp64":
                    np.testing.assert_allclose(gl[k], rl[k], rtol=1e-9, atol=1e-12)
                else:
                    err = np.abs(gl[k] - rl[k])
                    assert np.mean(err <= 1e-3 * w.lr_actor + 1e-7) > 0.98, k
    assert ctx.sync_status() == (0, 0)
    ctx.rebind()                 # binding the parameters again resets the tuned coefficient
    assert ctx.get_alpha() == pytest.approx(w.alpha, rel=1e-7)


def test_alpha_is_fixed_without_autotune():
    w = small(B=32)
    ctx, _, _ = setup(w, n=40)
    for _ in range(2):
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in workload.buffer_contents(w, n=1, seed_offset=3)))
    assert ctx.get_alpha() == np.float32(w.alpha)


def test_nonfinite_loss_sets_status():
    w = small(B=32)
    ctx, _, _ = setup(w, n=40)
    ctx.views("phi")[-1]["b"][0] = float("nan")
    s, a, g, _ = ctx.sample(step=0)
    ctx.critic_step(s, a, g)
    rc, status = ctx.sync_status()
    assert rc == api.E_NONFINITE and status & api.STATUS_NONFINITE
    assert ctx.sync_status() == (0, 0)          # cleared by the read


def test_bad_sizes_and_configs_are_rejected():
    w = small(B=32)
    ctx, _, _ = setup(w, n=40)
    big = [torch.zeros(33, n, device=ctx.device) for n in (w.D, w.A, w.G)]
    with pytest.raises(api.CRLError) as e:
        ctx.critic_step(*big)
    assert e.value.code == api.E_SHAPE
    h = ctypes.c_void_p()
    for bad in (api.make_config(w, gamma=1.0), api.make_config(w, temperature=0.0),
                api.make_config(w, layers=0), api.make_config(w, offset_min=2),
                api.make_config(w, alpha_autotune=1, alpha=0.0),
                api.make_config(w, alpha_autotune=1, target_entropy=float("nan")),
                api.make_config(w, alpha_autotune=2)):
        assert api.lib().crl_create(ctypes.byref(bad), ctypes.byref(h)) == api.E_INVALID_ARG
        assert h.value is None
    cfg = api.make_config(w)
    cfg.goal_idx[1] = w.D                      # goal dim outside the observation
    assert api.lib().crl_create(ctypes.byref(cfg), ctypes.byref(h)) == api.E_INVALID_ARG


def test_tracing_counts_relabel_bytes():
    w = small(B=64)
    ctx, _, _ = setup(w, n=40)
    ctx.trace_start("relabel", 16)
    for step in range(3):
        ctx.sample(step=step)
    n, ms, work = ctx.trace_stop()
    assert n == 3 and ms > 0
    per = (w.D + w.A + 1 + w.G) * 4 + (w.D + w.A + w.G) * 4 + 12
    assert work == pytest.approx(3 * w.B * per)


@pytest.mark.parametrize("precision,path", [("fp32", "plain"), ("bf16", "plain"), ("bf16", "fused")])
def test_graph_replay_matches_eager(precision, path):
    """crl_update_step on a side stream (captured once, then replayed as a CUDA graph)
    gives bit-identical losses and parameters to eager calls on the default stream."""
    w = small(B=64, repr=64)
    runs = []
    for side in (False, True):
        ctx, _, _ = setup(w, precision=precision, path=path, n=60)
        extra = workload.buffer_contents(w, n=5, mean_len=9.0, seed_offset=7)
        torch.cuda.synchronize()                 # the set-up ran on the default stream
        stream = torch.cuda.Stream() if side else torch.cuda.current_stream()
        loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
        hist = []
        with torch.cuda.stream(stream):
            for i in range(5):
                ins = [torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra]
                ctx.update_step(*ins, loss_out=loss)
                hist.append(loss.cpu().numpy().copy())
        torch.cuda.synchronize()
        runs.append((np.array(hist), {n: ctx.store[n]["params"].cpu().numpy() for n in ("phi", "psi", "pi")}))
        assert ctx.sync_status() == (0, 0)
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for n in ("phi", "psi", "pi"):
        np.testing.assert_array_equal(runs[0][1][n], runs[1][1][n])


@pytest.mark.parametrize("precision,path", [("fp32", "plain"), ("bf16", "plain"), ("bf16", "fused")])
def test_update_step_matches_separate_calls(precision, path):
    """crl_update_step (the relabel kernel packing the network inputs, the
    policy's forward inside the critic's launches, the actor head inside the
    critic's Adam launch, the step counter advanced on the device) equals insert
    + sample + crl_critic_step + crl_actor_step called one by one, bit for bit."""
    w = small(B=64, repr=64)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=7)
    runs = []
    for fused in (True, False):
        ctx, _, _ = setup(w, precision=precision, path=path, n=60)
        hist = []
        for i in range(3):
            ins = [torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra]
            if fused:
                loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
                ctx.update_step(*ins, loss_out=loss)
                hist.append(loss.cpu().numpy().copy())
            else:
                ctx.insert(*ins)
                s, a, g, _ = ctx.sample(step=i, B=w.B)
                lc = ctx.critic_step(s, a, g, apply_update=True)
                la = ctx.actor_step(s, g, apply_update=True)
                hist.append(np.concatenate([lc.cpu().numpy(), la.cpu().numpy()]))
        torch.cuda.synchronize()
        assert ctx.sync_status() == (0, 0)
        runs.append((np.array(hist), {n: ctx.store[n]["params"].cpu().numpy() for n in ("phi", "psi", "pi")}))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for n in ("phi", "psi", "pi"):
        np.testing.assert_array_equal(runs[0][1][n], runs[1][1][n], err_msg=n)


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_persistent_gemm_matches_one_tile_gemm(path):
    """The persistent tensor-core GEMM (double-buffered TMEM, several tiles per CTA:
    batch 2048 gives more tiles than SMs), the CTA-pair kernel (256-row tiles on
    two SMs, tcgen05.mma.cta_group::2) and the one-tile kernel give bit-identical
    update steps: each output element is the same sum of K = 16 slices whatever
    the tile shape (fixed tile rule; batch 2048 takes no split-K)."""
    w = small(B=2048, hidden=512, repr=64, E=8, T=400)
    prev_tune = api.set_autotune(False)
    runs = []
    try:
        for mode in ("one_tile", "persistent", "cta_pair"):
            prev = api.set_gemm_kernel(mode)
            try:
                ctx, _, _ = setup(w, precision="bf16", path=path, n=300, mean_len=40.0)
                extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=7)
                loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
                hist = []
                for i in range(3):
                    ctx.update_step(*(torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra), loss_out=loss)
                    hist.append(loss.cpu().numpy().copy())
                torch.cuda.synchronize()
                assert ctx.sync_status() == (0, 0)
                runs.append((np.array(hist), {n: ctx.store[n]["params"].cpu().numpy() for n in ("phi", "psi", "pi")}))
            finally:
                api.set_gemm_kernel(prev)
    finally:
        api.set_autotune(prev_tune)
    for r in runs[1:]:
        np.testing.assert_array_equal(runs[0][0], r[0])
        for n in ("phi", "psi", "pi"):
            np.testing.assert_array_equal(runs[0][1][n], r[1][n], err_msg=n)


@pytest.mark.parametrize("B,layernorm", [(520, False), (136, True)])
def test_cta_pair_gemm_ragged_batches(B, layernorm):
    """CTA-pair tiles over batches that end inside a 256-row tile (520 = 2 x 256 + 8:
    the last pair's odd CTA holds no rows at all; 136: one pair, rows 128..135 in the
    odd CTA) give the one-tile kernel's update steps bit for bit."""
    w = small(B=B, hidden=256, repr=64, E=8, T=300, layernorm=layernorm)
    prev_tune = api.set_autotune(False)
    runs = []
    try:
        for mode in ("one_tile", "cta_pair"):
            prev = api.set_gemm_kernel(mode)
            try:
                ctx, _, _ = setup(w, precision="bf16", path="fused", n=200, mean_len=30.0)
                extra = workload.buffer_contents(w, n=2, mean_len=9.0, seed_offset=5)
                loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
                hist = []
                for i in range(2):
                    ctx.update_step(*(torch.from_numpy(x[i:i + 1]).to(ctx.device) for x in extra), loss_out=loss)
                    hist.append(loss.cpu().numpy().copy())
                torch.cuda.synchronize()
                assert ctx.sync_status() == (0, 0)
                runs.append((np.array(hist), {n: ctx.store[n]["params"].cpu().numpy() for n in ("phi", "psi", "pi")}))
            finally:
                api.set_gemm_kernel(prev)
    finally:
        api.set_autotune(prev_tune)
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for n in ("phi", "psi", "pi"):
        np.testing.assert_array_equal(runs[0][1][n], runs[1][1][n], err_msg=n)


def test_gemm_kernel_mode_is_validated():
    assert api.lib().crl_set_gemm_kernel(4) == api.E_INVALID_ARG
    assert api.set_gemm_kernel("any") == "any"


def test_l1_energy_runs_on_every_path():
    """-L1 (App. A.2) trains on the plain paths and on the fused path (SIMT tiles)."""
    w = small(B=64, energy="l1")
    h = ctypes.c_void_p()
    for precision, path, R in (("bf16", "fused", 64), ("fp32", "plain", w.repr), ("bf16", "plain", w.repr)):
        cfg = api.make_config(w.with_(repr=R), precision=precision, path=path)
        assert api.lib().crl_create(ctypes.byref(cfg), ctypes.byref(h)) == api.OK, (precision, path)
        api.lib().crl_destroy(h)


@pytest.mark.parametrize("precision,path", [("fp32", "plain"), ("bf16", "fused")])
def test_pinned_host_inputs_equal_device_inputs(precision, path):
    """Pinned host inputs (read in place by the insert kernel through their
    device alias), pageable host inputs (staged) and device inputs give the same
    losses and parameters."""
    w = small(B=64, repr=64)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=7)
    runs = []
    for kind in ("device", "pinned", "pageable"):
        ctx, _, _ = setup(w, precision=precision, path=path, n=60)
        loss = torch.zeros(6, dtype=torch.float32, device=ctx.device)
        hist = []
        for i in range(3):
            xs = [torch.from_numpy(np.ascontiguousarray(x[i:i + 1])) for x in extra]
            if kind == "device":
                xs = [x.to(ctx.device) for x in xs]
            elif kind == "pinned":
                xs = [x.pin_memory() for x in xs]
            ctx.update_step(*xs, loss_out=loss)
            torch.cuda.synchronize()
            hist.append(loss.cpu().numpy().copy())
        assert ctx.sync_status() == (0, 0)
        runs.append((np.array(hist), {n: ctx.store[n]["params"].cpu().numpy() for n in ("phi", "psi", "pi")}))
    for other in runs[1:]:
        np.testing.assert_array_equal(runs[0][0], other[0])
        for n in ("phi", "psi", "pi"):
            np.testing.assert_array_equal(runs[0][1][n], other[1][n])


def test_split_k_weight_gradients_are_deterministic_and_match_the_oracle():
    """Batch 4096 splits the weight-gradient products (K = the batch) in two: the
    last CTA of each output tile adds the partial tiles in split order, so two
    identical critic steps give identical bits, and the gradients stay at the
    BF16 bars against the oracle."""
    w = small(B=4096, hidden=256, repr=64, E=16, T=400)
    ctx, nets, buf = setup(w, precision="bf16", path="fused", n=400, mean_len=None)
    s, a, g, _ = ctx.sample(step=2)
    runs = []
    for _ in range(2):
        loss = ctx.critic_step(s, a, g, apply_update=False).cpu().numpy()
        runs.append((loss, {n: ctx.store[n]["grads"].cpu().numpy().copy() for n in ("phi", "psi")}))
    assert ctx.sync_status() == (0, 0)
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for n in ("phi", "psi"):
        np.testing.assert_array_equal(runs[0][1][n], runs[1][1][n])
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, 2, w.B, w.goals(), w.gamma)
    h = hp(w)
    _, gphi, gpsi, _, _ = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o, w.energy, h["tau"],
                                                           w.loss, w.sym_reduction, h["beta"], w.penalty_axis)
    for net, ref in (("phi", gphi), ("psi", gpsi)):
        for got_l, ref_l in zip(ctx.network(net, "grads"), ref):
            for k in ref_l:
                x, y = got_l[k].ravel(), ref_l[k].ravel()
                assert x @ y / (np.linalg.norm(x) * np.linalg.norm(y)) >= 0.999, (net, k)
