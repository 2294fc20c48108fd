"""Pins of the oracle's per-species ensemble (Sec. 3.2: one network per species mass fraction,
hidden layers 1600, 800 and 400, each trained on its own output).

* The ensemble is one multi-output network whose first layer stacks the G first layers and whose
  later layers are block-diagonal: the already-pinned multi-output oracle on that network gives
  the same outputs (FP64 and with the device's BF16 rounding points) and, on the diagonal
  blocks, the same gradients. Pairing network g's hidden layers with another network's output
  row, or a transposed block, fails it.
* Networks that share their hidden layers reduce to the multi-output network of those layers.
* Permuting the networks permutes the output columns.
* The gradients agree with central finite differences of the summed per-network L1 losses.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth


def _blockdiag(nets):
    from scipy.linalg import block_diag
    first = (np.vstack([n[0][0] for n in nets]), np.concatenate([n[0][1] for n in nets]))
    rest = [(block_diag(*[n[l][0] for n in nets]), np.concatenate([n[l][1] for n in nets]))
            for l in range(1, len(nets[0]))]
    return [first] + rest


def _case(G=5, seed=7):
    nets = synth.mlp_ensemble([10, 48, 32, 16, G], seed)
    z = np.random.default_rng(seed).normal(size=(300, 10))
    return nets, z


@pytest.mark.parametrize("round_bf16", [False, True])
def test_ensemble_is_a_block_diagonal_network(round_bf16):
    nets, z = _case()
    u = A.network_ensemble(nets, z, round_bf16)
    assert u.shape == (300, 5)
    ub = A.network(_blockdiag(nets), z, round_bf16)
    assert np.allclose(u, ub, rtol=1e-12, atol=1e-14)
    # network g's hidden layers with network g + 1's output layer: caught
    bad = [n[:3] + [nets[(g + 1) % 5][3]] for g, n in enumerate(nets)]
    assert not np.allclose(A.network_ensemble(bad, z), A.network(_blockdiag(nets), z), rtol=1e-3, atol=1e-6)
    # a transposed hidden block (square, so the shapes still fit): caught
    sq = synth.mlp_ensemble([10, 32, 32, 16, 3], 9)
    tr = [[n[0], (n[1][0].T.copy(), n[1][1]), n[2], n[3]] for n in sq]
    assert not np.allclose(A.network_ensemble(tr, z), A.network(_blockdiag(sq), z), rtol=1e-3, atol=1e-6)


def test_shared_hidden_layers_reduce_to_the_multi_output_network():
    layers = synth.mlp_layers([10, 48, 32, 16, 5], 8)
    z = np.random.default_rng(8).normal(size=(200, 10))
    nets = [layers[:3] + [(layers[3][0][g:g + 1], layers[3][1][g:g + 1])] for g in range(5)]
    assert np.allclose(A.network_ensemble(nets, z), A.network(layers, z), rtol=1e-12, atol=1e-14)


def test_permuting_networks_permutes_outputs():
    nets, z = _case()
    perm = [3, 0, 4, 1, 2]
    u = A.network_ensemble(nets, z)
    assert np.array_equal(A.network_ensemble([nets[g] for g in perm], z), u[:, perm])


def test_stack_and_unstack_are_inverse():
    nets, _ = _case()
    back = synth.unstack_ensemble(synth.stack_ensemble(nets), 5)
    for a, b in zip(nets, back):
        for (Wa, ba), (Wb, bb) in zip(a, b):
            assert np.array_equal(Wa, Wb) and np.array_equal(ba, bb)


def _as_dicts(net):
    return [{"W": W.copy(), "b": b.copy()} for W, b in net]


def test_ensemble_gradients_are_the_block_diagonal_ones():
    nets, z = _case(G=4, seed=11)
    target = np.random.default_rng(12).normal(size=(300, 4))
    loss, grads = M.ensemble_grads([_as_dicts(n) for n in nets], z, target)
    bd = _as_dicts(_blockdiag(nets))
    out, cache = M.forward(bd, z)
    lb, dout = M.l1_loss(out, target)
    gb = M.backward(bd, cache, dout)
    assert np.isclose(loss, lb, rtol=1e-12)
    widths = [10, 48, 32, 16, 1]
    for g in range(4):
        for l in range(4):
            r0, r1 = g * widths[l + 1], (g + 1) * widths[l + 1]
            c0, c1 = (0, 10) if l == 0 else (g * widths[l], (g + 1) * widths[l])
            assert np.allclose(grads[g][l]["W"], gb[l]["W"][r0:r1, c0:c1], rtol=1e-10, atol=1e-14)
            assert np.allclose(grads[g][l]["b"], gb[l]["b"][r0:r1], rtol=1e-10, atol=1e-14)


def test_ensemble_gradients_match_finite_differences():
    nets = synth.mlp_ensemble([4, 6, 5, 3, 2], 21)
    z = np.random.default_rng(22).normal(size=(7, 4))
    target = np.random.default_rng(23).normal(size=(7, 2))
    D = [_as_dicts(n) for n in nets]
    _, grads = M.ensemble_grads(D, z, target)

    def total():
        return M.ensemble_grads(D, z, target)[0]

    rng = np.random.default_rng(24)
    for g in range(2):
        for l in range(4):
            for key in ("W", "b"):
                a = D[g][l][key]
                for _ in range(3):
                    idx = tuple(rng.integers(0, s) for s in a.shape)
                    h = 1e-6
                    a[idx] += h
                    fp = total()
                    a[idx] -= 2 * h
                    fm = total()
                    a[idx] += h
                    fd = (fp - fm) / (2 * h)
                    assert abs(fd - grads[g][l][key][idx]) <= 1e-6 * max(1.0, abs(fd)), (g, l, key, idx)
