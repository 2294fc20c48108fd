"""Pins of the MLP oracle (Sec. 3.2; Eq. 5).

Box-Cox end points from the paper's stated range, GELU's value and slope at 0
and its odd-part identity, an identity network, the backward pass against
central finite differences, the L1 subgradient, and Adam's first step in
closed form.
"""
import math

import numpy as np

from oracle import mlp as M


def test_boxcox_range_endpoints():
    # Sec. 3.2: [0, 1] maps onto [-1/lambda, 0] with lambda = 0.1
    assert M.boxcox(np.array([1.0]))[0] == 0.0
    assert abs(M.boxcox(np.array([0.0]))[0] + 10.0) < 1e-15
    y = np.linspace(0, 1, 101)
    f = M.boxcox(y)
    assert np.all(np.diff(f) > 0) and f.min() >= -10.0 and f.max() <= 0.0
    assert M.boxcox(np.array([-1e-3]))[0] == -10.0   # negative Y clamps to 0
    # lambda -> 0 limit is the log transform
    assert abs(M.boxcox(np.array([0.3]), lam=1e-8)[0] - math.log(0.3)) < 1e-7


def test_gelu_values():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    x = np.linspace(-4, 4, 17)
    assert np.allclose(M.gelu(x) - M.gelu(-x), x, atol=1e-15)
    assert abs(M.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    h = 1e-6
    assert np.allclose((M.gelu(x + h) - M.gelu(x - h)) / (2 * h), M.gelu_grad(x), atol=1e-9)


def test_identity_network():
    L = [{"W": np.eye(5), "b": np.zeros(5)}]
    z = np.random.default_rng(0).normal(size=(7, 5))
    out, _ = M.forward(L, z)
    assert np.array_equal(out, z)


def test_backward_matches_fd():
    layers = M.init_params([6, 9, 7, 4], seed=3)
    rng = np.random.default_rng(4)
    z = rng.normal(size=(5, 6))
    c = rng.normal(size=(5, 4))
    f = lambda Ls: float((M.forward(Ls, z)[0] * c).sum())
    out, cache = M.forward(layers, z)
    grads = M.backward(layers, cache, c)
    h = 1e-6
    for li in range(3):
        for key in ("W", "b"):
            P = layers[li][key]
            it = np.nditer(P, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = P[idx]
                P[idx] = old + h
                fp = f(layers)
                P[idx] = old - h
                fm = f(layers)
                P[idx] = old
                fd = (fp - fm) / (2 * h)
                assert abs(fd - grads[li][key][idx]) <= 1e-7 * max(1.0, abs(fd))


def test_l1_subgradient():
    out = np.array([[1.0, -2.0, 3.0], [0.5, 0.5, 0.0]])
    tgt = np.array([[0.0, -2.0, 4.0], [1.0, 0.0, 0.0]])
    loss, g = M.l1_loss(out, tgt)
    assert loss == (1.0 + 0.0 + 1.0 + 0.5 + 0.5 + 0.0) / 2
    assert np.array_equal(g, np.array([[0.5, 0.0, -0.5], [-0.5, 0.5, 0.0]]))


def test_adam_first_step_closed_form():
    layers = [{"W": np.array([[1.0, -2.0]]), "b": np.array([0.5])}]
    grads = [{"W": np.array([[0.3, -4.0]]), "b": np.array([0.0])}]
    st = M.adam_init(layers)
    W0 = layers[0]["W"].copy()
    M.adam_step(layers, grads, st, lr=1e-3)
    g = grads[0]["W"]
    assert np.allclose(layers[0]["W"], W0 - 1e-3 * g / (np.abs(g) + M.ADAM_EPS), rtol=0, atol=1e-15)
    assert layers[0]["b"][0] == 0.5


def test_adam_constant_gradient_moves_lr_per_step():
    # with a constant g the bias corrections give m_hat = g and v_hat = g^2 at every t, so each
    # step moves by lr g / (|g| + eps); a wrong correction exponent drifts away from this
    layers = [{"W": np.array([[0.0, 0.0]]), "b": np.array([0.0])}]
    grads = [{"W": np.array([[2.5, -0.01]]), "b": np.array([1.0])}]
    st = M.adam_init(layers)
    for _ in range(25):
        M.adam_step(layers, grads, st, lr=1e-3)
    g = grads[0]["W"]
    assert np.allclose(layers[0]["W"], -25e-3 * g / (np.abs(g) + M.ADAM_EPS), rtol=1e-12, atol=0)
    assert np.isclose(layers[0]["b"][0], -25e-3 / (1.0 + M.ADAM_EPS), rtol=1e-12, atol=0)


def test_adam_two_steps_worked_by_hand():
    # g = +1 then -1, beta1 = 0.9, beta2 = 0.999:
    # t = 1: m = 0.1, v = 0.001 -> m_hat = 1, v_hat = 1: step -lr / (1 + eps)
    # t = 2: m = 0.09 - 0.1 = -0.01, v = 0.000999 + 0.001 = 0.001999
    #        m_hat = -0.01 / (1 - 0.81) = -1/19, v_hat = 0.001999 / (1 - 0.998001) = 1: step +lr / (19 (1 + eps))
    layers = [{"W": np.array([[0.0]]), "b": np.array([0.0])}]
    st = M.adam_init(layers)
    lr = 1e-3
    M.adam_step(layers, [{"W": np.array([[1.0]]), "b": np.array([0.0])}], st, lr)
    M.adam_step(layers, [{"W": np.array([[-1.0]]), "b": np.array([0.0])}], st, lr)
    assert np.isclose(layers[0]["W"][0, 0], -lr * (18.0 / 19.0) / (1.0 + M.ADAM_EPS), rtol=1e-12, atol=0)


def test_zscore_statistics_by_hand():
    # per column: the mean and the population standard deviation (divisor n); a constant column
    # (the 1 atm pressure) gets sigma = 1
    x = np.array([[5.0, 1.0, -2.0], [5.0, 2.0, 2.0], [5.0, 3.0, -2.0], [5.0, 4.0, 2.0]])
    mu, sd = M.zscore_stats(x)
    assert np.array_equal(mu, [5.0, 2.5, 0.0])
    assert np.allclose(sd, [1.0, np.sqrt(1.25), 2.0], rtol=1e-15, atol=0)


def test_two_term_bf16_input():
    # the network input is carried as hi + lo BF16 terms: 16 significant bits
    from oracle import ann as A
    rng = np.random.default_rng(9)
    z = (rng.normal(size=20000) * 10.0 ** rng.uniform(-4, 2, 20000)).astype(np.float32).astype(np.float64)
    s = A.split_bf16(z)
    assert np.all(np.abs(s - z) <= 2.0 ** -16 * np.abs(z))
    assert np.mean(np.abs(A.to_bf16(z) - z) > 2.0 ** -16 * np.abs(z)) > 0.9   # one BF16 term is not enough
    b = A.to_bf16(z)
    assert np.array_equal(A.split_bf16(b), b)                                 # BF16 values: lo = 0
