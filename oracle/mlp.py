"""FP64 numpy oracle of the learned chemistry model (TEST INFRASTRUCTURE ONLY).

Sec. 3.2 of the paper: the network input is x = {T, p, F(Y)} with the Box-Cox
map F(Y) = (Y^lambda - 1)/lambda, lambda = 0.1 (the source prints the formula
garbled; its stated range [-1/lambda, 0] on [0, 1] fixes this reading), the
target is u* = Y(t + dt) - Y(t), both Z-score normalised with training-set
statistics; hidden layers 1600/800/400 with GELU; Adam; and the L1 loss of
Eq. 5, L = (1/B) sum_i |u*_i - u_i|_1 (the 1-norm over the outputs of each
sample, averaged over the samples).

Layers are y = W x + b with W stored [out, in]. Matrix products use numpy's
matmul as the library primitive; nothing is blocked, fused or reordered.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

LAMBDA_BC = 0.1
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8

_erf = np.vectorize(math.erf, otypes=[np.float64])


def boxcox(Y, lam: float = LAMBDA_BC):
    """F(Y) = (max(Y, 0)^lam - 1) / lam  (Sec. 3.2)."""
    return (np.power(np.maximum(Y, 0.0), lam) - 1.0) / lam


def features(T, p, Y):
    """Rows x = (T, p, F(Y_1), ..., F(Y_N)) for SoA inputs T[B], p[B], Y[N, B]."""
    return np.concatenate([np.asarray(T, np.float64)[:, None], np.asarray(p, np.float64)[:, None],
                           boxcox(np.asarray(Y, np.float64)).T], axis=1)


def zscore_stats(x, floor: float = 1e-12):
    """Per-column mean and standard deviation; a column with sigma < floor (a
    constant input such as p = 1 atm) gets sigma = 1."""
    mu = x.mean(axis=0)
    sd = x.std(axis=0)
    sd = np.where(sd < floor, 1.0, sd)
    return mu, sd


def gelu(z):
    """Exact GELU: z Phi(z), Phi the standard normal CDF."""
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    Phi = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return Phi + z * phi


def init_params(widths: List[int], seed: int) -> List[Dict[str, np.ndarray]]:
    """W, b ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), seeded (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    layers = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        a = 1.0 / math.sqrt(fi)
        layers.append({"W": rng.uniform(-a, a, (fo, fi)), "b": rng.uniform(-a, a, fo)})
    return layers


def forward(layers, z, act_last: bool = False):
    """Returns (output, cache); cache holds each layer's input and pre-activation."""
    h = np.asarray(z, np.float64)
    cache = []
    for i, L in enumerate(layers):
        pre = h @ L["W"].T + L["b"]
        cache.append((h, pre))
        last = i == len(layers) - 1
        h = gelu(pre) if (not last or act_last) else pre
    return h, cache


def l1_loss(out, target):
    """Eq. 5: L = (1/B) sum_i sum_k |u*_ik - u_ik| and dL/du = sign(u - u*) / B (sign(0) = 0)."""
    B = out.shape[0]
    d = out - target
    return float(np.abs(d).sum() / B), np.sign(d) / B


def backward(layers, cache, dout, act_last: bool = False):
    """Gradients of a scalar loss with dL/d(output) = dout; returns [{'W','b'}]."""
    grads = [None] * len(layers)
    g = np.asarray(dout, np.float64)
    for i in range(len(layers) - 1, -1, -1):
        h_in, pre = cache[i]
        last = i == len(layers) - 1
        if not last or act_last:
            g = g * gelu_grad(pre)
        grads[i] = {"W": g.T @ h_in, "b": g.sum(axis=0)}
        g = g @ layers[i]["W"]
    return grads


def ensemble_grads(nets, z, target, sign_from=None):
    """Sec. 3.2 trains each species' network on its own output: network g's loss is Eq. 5 on
    column g alone, and since no parameter is shared its gradient is that loss's gradient.
    nets[g] = [{'W', 'b'}] layers of network g. Returns (sum over g of the losses, per-network
    gradients). sign_from (optional, [B, G]): outputs on which the L1 subgradient sign is taken."""
    total, grads = 0.0, []
    for g, layers in enumerate(nets):
        out, cache = forward(layers, z)
        loss, dout = l1_loss(out, target[:, g:g + 1])
        if sign_from is not None:
            _, dout = l1_loss(sign_from[:, g:g + 1], target[:, g:g + 1])
        total += loss
        grads.append(backward(layers, cache, dout))
    return total, grads


def adam_init(layers):
    return {"t": 0, "m": [{k: np.zeros_like(v) for k, v in L.items()} for L in layers],
            "v": [{k: np.zeros_like(v) for k, v in L.items()} for L in layers]}


def adam_step(layers, grads, state, lr: float):
    """Adam (Kingma and Ba, 2015) with bias correction, in place."""
    state["t"] += 1
    t = state["t"]
    for L, G, M, V in zip(layers, grads, state["m"], state["v"]):
        for k in L:
            M[k] = ADAM_B1 * M[k] + (1 - ADAM_B1) * G[k]
            V[k] = ADAM_B2 * V[k] + (1 - ADAM_B2) * G[k] * G[k]
            mh = M[k] / (1 - ADAM_B1 ** t)
            vh = V[k] / (1 - ADAM_B2 ** t)
            L[k] = L[k] - lr * mh / (np.sqrt(vh) + ADAM_EPS)
