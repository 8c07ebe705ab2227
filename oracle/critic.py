"""Energy functions, InfoNCE objectives and the logsumexp penalty, with their gradient.

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes
--------------------
* §3.1: the critic is an energy f(s, a, g) of phi(s, a) and psi(g); the loss
  is a function of the B x B matrix {f(s_i, a_i, g_j)}; the base loss is
  symmetric InfoNCE with an L2 energy.
* App. A.2 lists the energies: cosine, dot, -L1, -L2, -L2^2; and the InfoNCE
  objectives: forward (softmax over goals j for each (s_i, a_i)), backward
  (softmax over state-actions j for each goal g_i) and symmetric (their sum).
* Algorithm 1 adds beta * L_logsumexp to the critic loss; §5.3 and App. B.3
  set beta = 0.1.

Readings where the paper is silent or inconsistent
---------------------------------------------------
C1  L2 energy carries the minus sign of App. A.2, f = -||phi - psi||_2 (the
    formula under §3.1 drops it, which would make the positive pair the least
    likely one; treated as a typo).
C2  F_ij = f(phi_i, psi_j) / tau with a temperature tau (tau = 1 unless set).
C3  The negatives are all B in-batch goals / state-actions, the positive
    included (K = |B|, as in the FlatNCE rows of App. A.2).
C4  The objectives are averaged over the batch (mean instead of the sum
    inside the batch expectation), so that equal representations give log B.
C5  Symmetric InfoNCE: the paper writes the sum of the two directions
    ("sum"); the default reduction here is their mean ("mean"), and both are
    available: L_sym,sum = 2 * L_sym,mean = L_fwd + L_bwd.
C6  The logsumexp penalty is not defined in the paper.  Reading: the mean
    over the batch of the squared row logsumexp, r_i = LSE_j F_ij, times beta
    ("row"); "col" uses c_j = LSE_i F_ij; "both" averages the two.
C7  The L2 gradient is undefined where phi_i = psi_j; the subgradient 0 is
    taken there (distances below 1e-12).

The other objectives of App. A.2 and §5.2 (``critic_loss``, ``critic_grad_F``)
------------------------------------------------------------------------------
C8  FlatNCE (App. A.2): S_i = sum_j exp(F_ij - F_ii) over the whole batch
    (j = i included, as printed); the forward direction anchors on (s_i, a_i)
    and sums over goals j, the backward direction anchors on g_i and sums over
    state-actions j.  The printed loss -sum_i log(S_i / detach S_i) has the
    value 0 (it is reported as 0), and the printed leading minus would make
    its gradient the negated InfoNCE gradient, i.e. training would ascend
    InfoNCE, at odds with §5.2's report that FlatNCE trains about as well as
    the InfoNCE objectives.  Reading: the gradient is that of +mean_i log S_i
    (the minus is a sign slip); because the j = i term of S_i is the constant
    1, this gradient equals InfoNCE's of the same direction.
C9  Forward-backward (App. A.2, Monte Carlo form): the second sum of the
    printed formula runs inside the sum over i, so
    L_FB = mean_i [ -exp(F_ii) + 1/(2(B - 1)) sum_{j != i} exp(F_ij)^2 ],
    defined for B >= 2.
C10 DPO, IPO, SPPO (App. A.2): the double sums over (i, j) run over all B^2
    pairs, j = i included as printed, and are averaged over the pairs (the
    mean of reading C4 applied to both sums).  For SPPO the (F_ii - 1)^2 term
    sits inside the sum over j, so it enters with weight 1 / B per anchor.
C11 NCE-binary (§5.2 names it as the objective originally proposed for CRL;
    App. A.2 does not define it).  Reading: binary cross-entropy of sigma(F_ij)
    against the label [i = j] (the positive on the diagonal, every other pair
    a negative), averaged over the B^2 pairs.
C12 The logsumexp penalty (reading C6) is added to every objective (§5.2
    applies the 0.1 regulariser to each objective).  The reported parts keep
    InfoNCE's forward and backward values as diagnostics for every objective;
    "contrastive" is the chosen objective's value and total = contrastive +
    penalty.
"""

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ENERGIES = ("l2", "dot", "cos", "l1", "l2sq")
LOSSES = ("fwd", "bwd", "sym")
OBJECTIVES = LOSSES + ("flatnce_fwd", "flatnce_bwd", "fb", "dpo", "ipo", "sppo", "nce_binary")


# The distance energies are computed one row i at a time from the differences
# phi_i - psi_j (no expanded form).  Rows are grouped into fixed blocks of
# ROW_BLOCK rows that run on a thread pool (numpy's element-wise kernels release
# the interpreter lock); the block partition does not depend on the thread
# count, so every result is the same on any machine.
ROW_BLOCK = 256


def _threads():
    """Worker threads: OMP_NUM_THREADS when set, else every host core."""
    try:
        n = int(os.environ.get("OMP_NUM_THREADS", "") or (os.cpu_count() or 1))
    except ValueError:
        n = os.cpu_count() or 1
    return max(1, n)


def _over_row_blocks(n_rows, fn):
    """[fn(i0, i1) for each block [i0, i1) of ROW_BLOCK rows], in block order."""
    blocks = [(i0, min(i0 + ROW_BLOCK, n_rows)) for i0 in range(0, n_rows, ROW_BLOCK)]
    n = min(_threads(), len(blocks))
    if n <= 1:
        return [fn(i0, i1) for i0, i1 in blocks]
    with ThreadPoolExecutor(max_workers=n) as ex:
        return list(ex.map(lambda b: fn(*b), blocks))


def energy_matrix(phi, psi, energy="l2", tau=1.0):
    """F [B][B] with F_ij = f(phi_i, psi_j) / tau (App. A.2; readings C1, C2)."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    if energy in ("l2", "l2sq", "l1"):
        # one row i at a time: f(phi_i, psi_j) from the difference phi_i - psi_j
        f = np.empty((phi.shape[0], psi.shape[0]))

        def rows(i0, i1):
            for i in range(i0, i1):
                d = phi[i][None, :] - psi
                if energy == "l2":
                    f[i] = -np.sqrt((d ** 2).sum(axis=1))
                elif energy == "l2sq":
                    f[i] = -(d ** 2).sum(axis=1)
                else:
                    f[i] = -np.abs(d).sum(axis=1)

        _over_row_blocks(phi.shape[0], rows)
    elif energy == "dot":
        f = phi @ psi.T
    elif energy == "cos":
        f = (phi @ psi.T) / np.outer(np.linalg.norm(phi, axis=1), np.linalg.norm(psi, axis=1))
    else:
        raise ValueError(energy)
    return f / tau


def logit_stats(F):
    """Diagnostic of an energy matrix (no counterpart in the paper): the mean
    positive-pair logit (1/B) sum_i F_ii and the mean negative logit
    (1/(B^2 - B)) sum_{i != j} F_ij (NaN when B = 1: there are no negatives)."""
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    diag = float(np.trace(F)) / B
    off = float((F.sum() - np.trace(F)) / (B * (B - 1))) if B > 1 else float("nan")
    return diag, off


def energy_diagonal(phi, psi, energy="l2", tau=1.0):
    """f(phi_i, psi_i) / tau for each i (the positive pairs)."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    d = phi - psi
    if energy == "l2":
        f = -np.sqrt((d ** 2).sum(axis=1))
    elif energy == "l2sq":
        f = -(d ** 2).sum(axis=1)
    elif energy == "l1":
        f = -np.abs(d).sum(axis=1)
    elif energy == "dot":
        f = (phi * psi).sum(axis=1)
    elif energy == "cos":
        f = (phi * psi).sum(axis=1) / (np.linalg.norm(phi, axis=1) * np.linalg.norm(psi, axis=1))
    else:
        raise ValueError(energy)
    return f / tau


def logsumexp(x, axis):
    """Stable log(sum(exp(x))) along ``axis``."""
    m = x.max(axis=axis, keepdims=True)
    return (m + np.log(np.exp(x - m).sum(axis=axis, keepdims=True))).squeeze(axis)


def direction_weights(loss, sym_reduction):
    """(w_fwd, w_bwd) of the two InfoNCE directions (App. A.2; reading C5)."""
    if loss == "fwd":
        return 1.0, 0.0
    if loss == "bwd":
        return 0.0, 1.0
    if loss == "sym":
        return (0.5, 0.5) if sym_reduction == "mean" else (1.0, 1.0)
    raise ValueError(loss)


def penalty_weights(penalty_axis):
    """(w_row, w_col) of the squared-logsumexp penalty (reading C6)."""
    return {"row": (1.0, 0.0), "col": (0.0, 1.0), "both": (0.5, 0.5)}[penalty_axis]


def infonce_loss(F, loss="sym", sym_reduction="mean", beta=0.1, penalty_axis="row"):
    """Loss parts from the energy matrix (App. A.2, Algorithm 1; readings C3-C6).

    Returns dict with total, fwd, bwd, contrastive, penalty, and r, c (the row
    and column logsumexp vectors).
    """
    F = np.asarray(F, dtype=np.float64)
    r = logsumexp(F, axis=1)
    c = logsumexp(F, axis=0)
    diag = np.diagonal(F)
    l_fwd = np.mean(r - diag)
    l_bwd = np.mean(c - diag)
    wf, wb = direction_weights(loss, sym_reduction)
    contrastive = wf * l_fwd + wb * l_bwd
    pr, pc = penalty_weights(penalty_axis)
    penalty = beta * (pr * np.mean(r ** 2) + pc * np.mean(c ** 2))
    return {"total": contrastive + penalty, "fwd": l_fwd, "bwd": l_bwd,
            "contrastive": contrastive, "penalty": penalty, "r": r, "c": c}


def infonce_grad_F(F, loss="sym", sym_reduction="mean", beta=0.1, penalty_axis="row"):
    """dL/dF [B][B] of ``infonce_loss``'s total.

    With P_ij = exp(F_ij - r_i) (row softmax) and Q_ij = exp(F_ij - c_j)
    (column softmax):
      dL_fwd/dF = (P - I) / B,   dL_bwd/dF = (Q - I) / B,
      d(beta mean r^2)/dF = 2 beta r_i P_ij / B,  d(beta mean c^2)/dF = 2 beta c_j Q_ij / B.
    """
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    r = logsumexp(F, axis=1)
    c = logsumexp(F, axis=0)
    P = np.exp(F - r[:, None])
    Q = np.exp(F - c[None, :])
    eye = np.eye(B)
    wf, wb = direction_weights(loss, sym_reduction)
    pr, pc = penalty_weights(penalty_axis)
    G = wf * (P - eye) + wb * (Q - eye)
    G = G + 2.0 * beta * (pr * r[:, None] * P + pc * c[None, :] * Q)
    return G / B


def sigmoid(x):
    """sigma(x) = 1 / (1 + exp(-x)), as exp(-log(1 + exp(-x))) without overflow."""
    return np.exp(-np.logaddexp(0.0, -np.asarray(x, dtype=np.float64)))


def neg_log_sigmoid(x):
    """-log sigma(x) = log(1 + exp(-x)), without overflow."""
    return np.logaddexp(0.0, -np.asarray(x, dtype=np.float64))


def objective_value(F, loss):
    """The value of an objective outside the InfoNCE family (App. A.2; C8-C11)."""
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    d = np.diagonal(F)
    if loss in ("flatnce_fwd", "flatnce_bwd"):
        # S_i over goals j (fwd) or over state-actions j (bwd); log(S_i / detach S_i)
        E = F - d[:, None] if loss == "flatnce_fwd" else F.T - d[:, None]
        S = np.exp(E).sum(axis=1)
        S_detached = S.copy()
        return float(-np.mean(np.log(S / S_detached)))
    if loss == "fb":
        if B < 2:
            raise ValueError("the forward-backward objective needs B >= 2")
        off = ~np.eye(B, dtype=bool)
        neg = np.where(off, np.exp(F) ** 2, 0.0).sum(axis=1) / (2.0 * (B - 1))
        return float(np.mean(-np.exp(d) + neg))
    if loss == "dpo":
        delta = d[:, None] - F                               # F(s_i, a_i, g_i) - F(s_i, a_i, g_j)
        return float(np.mean(neg_log_sigmoid(delta)))
    if loss == "ipo":
        delta = d[:, None] - F
        return float(np.mean((delta - 1.0) ** 2))
    if loss == "sppo":
        pos = np.broadcast_to(d[:, None], F.shape)
        return float(np.mean((pos - 1.0) ** 2 + (F + 1.0) ** 2))
    if loss == "nce_binary":
        y = np.eye(B)
        # -log sigma(F) for the positives, -log(1 - sigma(F)) = -log sigma(-F) for the negatives
        return float(np.mean(y * neg_log_sigmoid(F) + (1.0 - y) * neg_log_sigmoid(-F)))
    raise ValueError(loss)


def objective_grad_F(F, loss):
    """dL/dF [B][B] of ``objective_value`` (the gradient of reading C8 for FlatNCE)."""
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    d = np.diagonal(F)
    eye = np.eye(B)
    if loss in ("flatnce_fwd", "flatnce_bwd"):
        # mean_i log S_i with S_i = sum_j exp(E_ij), E_ij = F_ij - F_ii (fwd): dS_i/dF_ij = exp(E_ij)
        # for j != i, dS_i/dF_ii = -sum_{j != i} exp(E_ij) (the j = i term is constant).
        E = F - d[:, None] if loss == "flatnce_fwd" else F.T - d[:, None]
        W = np.exp(E) / np.exp(E).sum(axis=1, keepdims=True)
        Woff = W * (1.0 - eye)
        G = (Woff - np.diag(Woff.sum(axis=1))) / B
        return G if loss == "flatnce_fwd" else G.T
    if loss == "fb":
        G = np.exp(2.0 * F) * (1.0 - eye) / (B * (B - 1.0))
        return G - np.diag(np.exp(d)) / B
    if loss in ("dpo", "ipo"):
        delta = d[:, None] - F
        # dL/d(delta_ij) / B^2; delta_ij rises with F_ii and falls with F_ij
        h = -sigmoid(-delta) if loss == "dpo" else 2.0 * (delta - 1.0)
        h = h / B ** 2
        return -h + np.diag(h.sum(axis=1))
    if loss == "sppo":
        return 2.0 * (F + 1.0) / B ** 2 + np.diag(2.0 * (d - 1.0)) / B
    if loss == "nce_binary":
        return (sigmoid(F) - eye) / B ** 2
    raise ValueError(loss)


def critic_loss(F, loss="sym", sym_reduction="mean", beta=0.1, penalty_axis="row"):
    """Loss parts of any objective of App. A.2 / §5.2 plus the penalty (C4-C12).

    Same keys as ``infonce_loss``; for the objectives outside the InfoNCE family
    "fwd" / "bwd" stay InfoNCE's values (diagnostics) and "contrastive" is the
    objective's value.
    """
    if loss in LOSSES:
        return infonce_loss(F, loss, sym_reduction, beta, penalty_axis)
    parts = infonce_loss(F, "fwd", sym_reduction, beta, penalty_axis)
    value = objective_value(F, loss)
    parts["contrastive"] = value
    parts["total"] = value + parts["penalty"]
    return parts


def penalty_grad_F(F, beta, penalty_axis):
    """dL/dF of beta * (pr mean r^2 + pc mean c^2) (reading C6)."""
    F = np.asarray(F, dtype=np.float64)
    B = F.shape[0]
    r = logsumexp(F, axis=1)
    c = logsumexp(F, axis=0)
    pr, pc = penalty_weights(penalty_axis)
    P = np.exp(F - r[:, None])
    Q = np.exp(F - c[None, :])
    return 2.0 * beta * (pr * r[:, None] * P + pc * c[None, :] * Q) / B


def critic_grad_F(F, loss="sym", sym_reduction="mean", beta=0.1, penalty_axis="row"):
    """dL/dF of ``critic_loss``'s total."""
    if loss in LOSSES:
        return infonce_grad_F(F, loss, sym_reduction, beta, penalty_axis)
    return objective_grad_F(F, loss) + penalty_grad_F(F, beta, penalty_axis)


def energy_backward(phi, psi, G, energy="l2", tau=1.0):
    """Given G = dL/dF, return (dphi [B][R], dpsi [B][R]) for F = f(phi_i, psi_j) / tau."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    if energy == "dot":
        return G @ psi / tau, G.T @ phi / tau
    if energy == "cos":
        nphi = np.linalg.norm(phi, axis=1, keepdims=True)
        npsi = np.linalg.norm(psi, axis=1, keepdims=True)
        x, y = phi / nphi, psi / npsi
        dx = G @ y / tau
        dy = G.T @ x / tau
        dphi = (dx - x * (x * dx).sum(axis=1, keepdims=True)) / nphi
        dpsi = (dy - y * (y * dy).sum(axis=1, keepdims=True)) / npsi
        return dphi, dpsi
    if energy not in ("l2", "l2sq", "l1"):
        raise ValueError(energy)
    # One row i at a time over the differences phi_i - psi_j:
    #   L2:   dF_ij/dphi_i = -(phi_i - psi_j) / (tau d_ij)   (0 where d_ij = 0, reading C7)
    #   L2^2: dF_ij/dphi_i = -2 (phi_i - psi_j) / tau
    #   L1:   dF_ij/dphi_i = -sign(phi_i - psi_j) / tau
    # and dF_ij/dpsi_j is the negative of each.  dpsi sums the terms of every
    # row: within a block of rows in row order, then the blocks in block order.
    dphi = np.zeros_like(phi)

    def rows(i0, i1):
        part = np.zeros_like(psi)
        for i in range(i0, i1):
            diff = phi[i][None, :] - psi                   # [j][r]
            if energy == "l2":
                d = np.sqrt((diff ** 2).sum(axis=1))
                safe = d >= 1e-12
                h = np.where(safe, G[i] / (tau * np.where(safe, d, 1.0)), 0.0)
                term = h[:, None] * diff
            elif energy == "l2sq":
                term = (2.0 * G[i] / tau)[:, None] * diff
            else:
                term = (G[i] / tau)[:, None] * np.sign(diff)
            dphi[i] = -term.sum(axis=0)
            part += term
        return part

    dpsi = np.zeros_like(psi)
    for part in _over_row_blocks(phi.shape[0], rows):
        dpsi += part
    return dphi, dpsi


def energy_diagonal_backward(phi, psi, gdiag, energy="l2", tau=1.0):
    """Given gdiag_i = dL/dF_ii, return (dphi, dpsi) for the positive pairs only."""
    phi = np.asarray(phi, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    g = np.asarray(gdiag, dtype=np.float64)[:, None]
    if energy == "dot":
        return g * psi / tau, g * phi / tau
    if energy == "cos":
        nphi = np.linalg.norm(phi, axis=1, keepdims=True)
        npsi = np.linalg.norm(psi, axis=1, keepdims=True)
        x, y = phi / nphi, psi / npsi
        dx, dy = g * y / tau, g * x / tau
        return ((dx - x * (x * dx).sum(axis=1, keepdims=True)) / nphi,
                (dy - y * (y * dy).sum(axis=1, keepdims=True)) / npsi)
    diff = phi - psi
    if energy == "l2":
        d = np.sqrt((diff ** 2).sum(axis=1, keepdims=True))
        safe = d >= 1e-12
        h = np.where(safe, g / (tau * np.where(safe, d, 1.0)), 0.0)
        return -h * diff, h * diff
    if energy == "l2sq":
        return -2.0 * g * diff / tau, 2.0 * g * diff / tau
    if energy == "l1":
        return -g * np.sign(diff) / tau, g * np.sign(diff) / tau
    raise ValueError(energy)
