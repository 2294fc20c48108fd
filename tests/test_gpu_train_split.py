"""mlp_train_step in two halves on the GPU (mlp_train_grads, the gradient buffers, mlp_adam_step), as
data-parallel training uses them.

* mlp_train_grads then mlp_adam_step is bitwise mlp_train_step (parameters and gradients).
* The buffers of chem_mlp_grad_buffers alias the gradients that chem_mlp_get_grads returns.
* Two handles with the same parameters, each taking half of a batch, with their gradient buffers
  averaged in place on the device, then one Adam step each: both end bitwise equal, and their
  averaged gradients match the whole batch's gradients of a third handle to FP32 summation order.
Weights, statistics and states come from the seeded generator.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.gpu_util import to_dev
from tests.test_gpu_mlp import _mlp, _problem

pytestmark = pytest.mark.gpu
B = 256


def _data():
    n = B
    mech, T, p, Y, widths, layers, stats = _problem(n, seed=2081)
    dY = np.random.default_rng(2082).normal(size=Y.shape) * 1e-4
    return mech, T, p, Y, Y + dY, widths, layers, stats


def test_grads_then_adam_is_bitwise_train_step():
    import torch
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, Y1, widths, layers, stats = _data()
    ld = T.shape[0]
    Td, pd, Yd, Y1d = to_dev(T), to_dev(p), to_dev(Y), to_dev(Y1)
    a = _mlp("c2", widths, layers, stats)
    b = _mlp("c2", widths, layers, stats)
    for _ in range(3):
        binding.mlp_train_step(a, B, None, ld, Td, pd, Yd, Y1d, 1e-3)
        binding.mlp_train_grads(b, B, None, ld, Td, pd, Yd, Y1d)
        binding.mlp_adam_step(b, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    assert np.array_equal(a.get_grads(), b.get_grads())
    # the buffers alias the handle's gradients: W then b of each layer, the W rows padded to 8
    bufs = [t.cpu().numpy() for t in binding.grad_buffers(b)]
    g = b.get_grads()
    off = 0
    for layer in range(4):
        fi, fo = widths[layer], widths[layer + 1]
        kin = -(-fi // 8) * 8
        W = bufs[2 * layer].reshape(-1, kin)[:fo, :fi]
        assert np.array_equal(W.ravel(), g[off:off + fi * fo])
        off += fi * fo
        assert np.array_equal(bufs[2 * layer + 1][:fo], g[off:off + fo])
        off += fo
    a.free()
    b.free()


def test_two_shards_averaged_on_device_match_the_whole_batch():
    import torch
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, Y1, widths, layers, stats = _data()
    ld = T.shape[0]
    Td, pd, Yd, Y1d = to_dev(T), to_dev(p), to_dev(Y), to_dev(Y1)
    rows = torch.arange(B, dtype=torch.int32, device="cuda")
    whole = _mlp("c2", widths, layers, stats)
    binding.mlp_train_grads(whole, B, rows, ld, Td, pd, Yd, Y1d)
    ranks = [_mlp("c2", widths, layers, stats) for _ in range(2)]
    for r, net in enumerate(ranks):
        binding.mlp_train_grads(net, B // 2, rows[r * B // 2:(r + 1) * B // 2], ld, Td, pd, Yd, Y1d)
    b0, b1 = binding.grad_buffers(ranks[0]), binding.grad_buffers(ranks[1])
    for x, y in zip(b0, b1):        # the all-reduce of two ranks, on one device
        s = (x + y) * 0.5
        x.copy_(s)
        y.copy_(s)
    torch.cuda.synchronize()
    gw = whole.get_grads().astype(np.float64)
    g0 = ranks[0].get_grads().astype(np.float64)
    assert np.array_equal(ranks[0].get_grads(), ranks[1].get_grads())
    # the same sums in another order: FP32 rounding of sums over 128 and 256 rows of BF16 products
    scale = np.abs(gw).max()
    assert np.all(np.abs(g0 - gw) <= 1e-3 * np.abs(gw) + 1e-5 * scale), np.abs(g0 - gw).max() / scale
    for net in ranks:
        binding.mlp_adam_step(net, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(ranks[0].get_params(), ranks[1].get_params())
    for net in (whole, *ranks):
        net.free()
