"""Encoder and actor MLPs with optional LayerNorm, forward and hand-derived backward.

Test infrastructure only (see ``oracle/__init__``).

What the paper fixes
--------------------
* §3.1: the critic uses a state-action representation phi(s, a) and a goal
  representation psi(g); §4.3 / §5.4 scale these networks in width and depth,
  and §5.4 adds Layer Normalization before every activation for the large
  (4 x 1024) networks.
* App. B.3 (Table "Hyperparameters"): hidden layers [256, 256] for both
  encoders and the actor, representation dimension 64.

Readings where the paper is silent
----------------------------------
M1  Activation: ReLU; no activation after the output layer.
M2  LayerNorm (when enabled) sits between each hidden Linear and its ReLU, with
    a learned affine (gamma, beta), eps = 1e-6 and the biased variance.
M3  A layer is y = x W^T + b with W stored [out][in] (the layout of
    ``torch.nn.Linear``); the input of phi is concat(s, a), of psi is g and of
    the actor is concat(s, g).

A network is a list of layer dicts {"W", "b"[, "ln_g", "ln_b"]}; hidden layers
first, output layer last (no LayerNorm keys).
"""

import numpy as np

LN_EPS = 1e-6


def relu(x):
    return np.maximum(x, 0.0)


def layer_norm(z, gain, bias, eps=LN_EPS):
    """Reading M2: normalise each row over features with the biased variance."""
    mu = z.mean(axis=1, keepdims=True)
    var = ((z - mu) ** 2).mean(axis=1, keepdims=True)
    zhat = (z - mu) / np.sqrt(var + eps)
    return zhat * gain + bias, zhat, 1.0 / np.sqrt(var + eps)


def forward(net, x):
    """Run the MLP on x [M][in]; returns (out [M][out], cache for ``backward``)."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for layer in net[:-1]:
        z = h @ layer["W"].T + layer["b"]
        if "ln_g" in layer:
            u, zhat, rstd = layer_norm(z, layer["ln_g"], layer["ln_b"])
        else:
            u, zhat, rstd = z, None, None
        cache.append({"h_in": h, "u": u, "zhat": zhat, "rstd": rstd})
        h = relu(u)
    out = h @ net[-1]["W"].T + net[-1]["b"]
    cache.append({"h_in": h})
    return out, cache


def layer_norm_backward(du, zhat, rstd, gain):
    """Gradient of y = zhat * gain + bias through the row normalisation."""
    dzhat = du * gain
    n = du.shape[1]
    dz = rstd * (dzhat - dzhat.sum(axis=1, keepdims=True) / n
                 - zhat * (dzhat * zhat).sum(axis=1, keepdims=True) / n)
    return dz, (du * zhat).sum(axis=0), du.sum(axis=0)


def backward(net, cache, dout):
    """Chain rule through ``forward``: returns (grads list like ``net``, dx [M][in])."""
    grads = [None] * len(net)
    last = net[-1]
    dy = np.asarray(dout, dtype=np.float64)
    grads[-1] = {"W": dy.T @ cache[-1]["h_in"], "b": dy.sum(axis=0)}
    dh = dy @ last["W"]
    for li in range(len(net) - 2, -1, -1):
        layer, c = net[li], cache[li]
        du = dh * (c["u"] > 0)
        g = {}
        if "ln_g" in layer:
            dz, g["ln_g"], g["ln_b"] = layer_norm_backward(du, c["zhat"], c["rstd"], layer["ln_g"])
        else:
            dz = du
        g["W"] = dz.T @ c["h_in"]
        g["b"] = dz.sum(axis=0)
        grads[li] = g
        dh = dz @ layer["W"]
    return grads, dh
