"""FP64 reference of the surrogate MLP -- TEST INFRASTRUCTURE ONLY.

Network: 24 -> 128 -> 128 -> 128 -> 2 with exact GELU, x -> 0.5 x (1 + erf(x/sqrt 2)),
between the linear layers; outputs (mu, s) where s is the log-variance of a
Gaussian over the target y = log1p(sum of w_i w_j of a node pair).
Loss (mean over the batch) = 0.5 (s + (y - mu)^2 exp(-s)).

Parameters are a dict of float64 arrays: W1 (128, 24), b1 (128), W2 (128, 128),
b2, W3 (128, 128), b3, W4 (2, 128), b4 (2); a layer computes z = W h + b.
The backward pass is the chain rule written out; tests check it against
central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

SHAPES = {"W1": (128, 24), "b1": (128,), "W2": (128, 128), "b2": (128,),
          "W3": (128, 128), "b3": (128,), "W4": (2, 128), "b4": (2,)}
S_CLAMP = 12.0  # |s| is clamped to this in the loss (both implementations)

_erf = np.vectorize(math.erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def init_params(seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES.items():
        if name.startswith("W"):
            fan_in = shp[1]
            p[name] = rng.standard_normal(shp) * math.sqrt(2.0 / fan_in)
        else:
            p[name] = np.zeros(shp)
    return p


def forward(p: dict, x: np.ndarray):
    """x (B, 24) -> (out (B, 2), cache)."""
    z1 = x @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = gelu(z3)
    out = h3 @ p["W4"].T + p["b4"]
    return out, (x, z1, h1, z2, h2, z3, h3)


def loss(out: np.ndarray, y: np.ndarray):
    mu, s = out[:, 0], np.clip(out[:, 1], -S_CLAMP, S_CLAMP)
    r = y - mu
    return float(np.mean(0.5 * (s + r * r * np.exp(-s))))


def loss_grad(out: np.ndarray, y: np.ndarray):
    """d loss / d out (B, 2) for the mean loss."""
    B = len(y)
    mu, s_raw = out[:, 0], out[:, 1]
    s = np.clip(s_raw, -S_CLAMP, S_CLAMP)
    r = y - mu
    e = np.exp(-s)
    g = np.zeros_like(out)
    g[:, 0] = -r * e / B
    inside = (s_raw > -S_CLAMP) & (s_raw < S_CLAMP)
    g[:, 1] = np.where(inside, 0.5 * (1.0 - r * r * e), 0.0) / B
    return g


def backward(p: dict, cache, dout: np.ndarray) -> dict:
    x, z1, h1, z2, h2, z3, h3 = cache
    g = {}
    g["W4"] = dout.T @ h3
    g["b4"] = dout.sum(0)
    dz3 = (dout @ p["W4"]) * gelu_grad(z3)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return g


def loss_and_grads(p: dict, x: np.ndarray, y: np.ndarray):
    out, cache = forward(p, x)
    return loss(out, y), backward(p, cache, loss_grad(out, y))


# ---- the surrogate's mean-consistent objective --------------------------------
# For a pair with label Y >= 0 (its exact yield) and baseline B >= 0 (the
# calibrated ST-form estimate) the network's first output mu sets the predicted
# mean lam = (B + 1) exp(mu); the second output s is the log variance of the
# log-space residual r = log1p(Y) - log1p(lam).  Per pair
#     P = (lam - Y log lam) / (B + 1)          (weighted Poisson deviance:
#                                              its minimiser is lam = E[Y | x])
#     V = 0.5 (s + r^2 exp(-s)) with lam held fixed in r (semi-gradient: the
#                                              variance head does not move mu)
# and the objective is the batch mean of P + V.
MU_CLAMP = 30.0


def mean_outputs(out, B):
    mu = np.minimum(out[:, 0], MU_CLAMP)
    return (B + 1.0) * np.exp(mu)


def loss_mean(out, Y, B, lam_fixed=None):
    lam = mean_outputs(out, B)
    lam_r = lam if lam_fixed is None else lam_fixed
    s = np.clip(out[:, 1], -S_CLAMP, S_CLAMP)
    r = np.log1p(Y) - np.log1p(lam_r)
    P = (lam - Y * np.log(lam)) / (B + 1.0)
    V = 0.5 * (s + r * r * np.exp(-s))
    return float(np.mean(P + V))


def loss_mean_grad(out, Y, B):
    n = len(Y)
    lam = mean_outputs(out, B)
    s_raw = out[:, 1]
    s = np.clip(s_raw, -S_CLAMP, S_CLAMP)
    r = np.log1p(Y) - np.log1p(lam)
    g = np.zeros_like(out)
    g[:, 0] = np.where(out[:, 0] < MU_CLAMP, (lam - Y) / (B + 1.0), 0.0) / n
    inside = (s_raw > -S_CLAMP) & (s_raw < S_CLAMP)
    g[:, 1] = np.where(inside, 0.5 * (1.0 - r * r * np.exp(-s)), 0.0) / n
    return g
