"""The gradient error model of tests/grad_bounds.py on the CPU: the arithmetic of
the device's training step, emulated in numpy (BF16 rounding at the device's
storage points, FP32 products and sums), stays within the model's 8-sigma
bound of the FP64 backward, while a gradient with one row's sign flipped or two
rows swapped does not (the bound is tight enough to catch such bugs)."""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.grad_bounds import check, gradients_with_sigma, separated_targets


def _f32(x):
    return np.asarray(x, np.float32)


def _emulated_device_grads(layers, z, target):
    """The device's forward and backward with BF16 storage and FP32 arithmetic."""
    bf = A.to_bf16
    zf = np.asarray(z, np.float32).astype(np.float64)
    B = zf.shape[0]
    h = A.split_bf16(zf)
    hs, pres = [bf(zf)], []
    for i, (W, b) in enumerate(layers):
        pre = (_f32(h) @ _f32(bf(W)).T).astype(np.float64) + b
        pre = _f32(pre).astype(np.float64)
        pres.append(pre)
        if i < len(layers) - 1:
            h = bf(M.gelu(pre))
            hs.append(h)
    g = np.sign(pres[-1] - target) / B
    out = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        out[i] = ((_f32(g).T @ _f32(hs[i])).astype(np.float64), _f32(g).sum(axis=0).astype(np.float64))
        if i > 0:
            dX = (_f32(g) @ _f32(bf(layers[i][0]))).astype(np.float64)
            g = bf(dX * M.gelu_grad(pres[i - 1]))
    return out


@pytest.fixture(scope="module")
def case():
    B = 256
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, B, 2031, synth.padded_ld(B))
    widths = [mech.N + 2, 256, 128, 64, mech.N - 1]
    layers = synth.mlp_layers(widths, 5031)
    x = M.features(T[:B], p[:B], Y[:, :B])
    mu, sd = M.zscore_stats(x)
    z = (x - mu) / sd
    uq = A.network(layers, np.asarray(z, np.float32).astype(np.float64), round_bf16=True)
    target = separated_targets(uq, np.random.default_rng(3))
    _, go, sig, _ = gradients_with_sigma(layers, z, target, uq)
    return go, sig, _emulated_device_grads(layers, z, target)


def test_emulated_device_within_bound(case):
    go, sig, dev = case
    for l in range(4):
        for j in range(2):
            assert check(dev[l][j], go[l][j], sig[l][j], "layer %d %d" % (l, j)) < 1.0


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_planted_mistakes_fail(case, l):
    go, sig, dev = case
    W = dev[l][0].copy()
    W[3] = -W[3]
    with pytest.raises(AssertionError):
        check(W, go[l][0], sig[l][0], "sign")
    W = dev[l][0].copy()
    W[[3, 4]] = W[[4, 3]]
    with pytest.raises(AssertionError):
        check(W, go[l][0], sig[l][0], "swap")
    b = dev[l][1].copy()
    b[[1, 2]] = b[[2, 1]]
    with pytest.raises(AssertionError):
        check(b, go[l][1], sig[l][1], "bias swap")
