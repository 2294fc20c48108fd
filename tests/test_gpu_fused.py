"""The fused output layers (gemm_fused34.cuh: layers 3 and 4 with h3 made on chip
and multiplied by the output weights) against the separate launches and the
oracle.

* Bitwise: every output of chem_mlp_forward with the fusion equals the output
  without it (the same BF16 roundings and k order per element), at the
  paper's widths, over one and several chunks with a ragged row count, and a
  last hidden layer the fusion does not take (64 units: off).
* chem_mlp_forward with fusion on matches the oracle as in test_gpu_mlp.py (the
  default path of the learned step).
Weights, statistics and states come from the seeded generator, never from the GPU.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, hidden, seed):
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, n, seed, synth.padded_ld(n))
    widths = [mech.N + 2, *hidden, mech.N - 1]
    layers = synth.mlp_layers(widths, 3000 + seed)
    mu_x, sd_x = M.zscore_stats(M.features(T[:n], p[:n], Y[:, :n]))
    rng = np.random.default_rng(seed + 7)
    stats = (mu_x, sd_x, rng.uniform(-1e-5, 1e-5, mech.N - 1), 10.0 ** rng.uniform(-6, -3, mech.N - 1))
    return mech, T, p, Y, widths, layers, stats


def _net(widths, layers, stats, **kw):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], **kw)
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    return net


def _u(net, T, p, Y, n):
    import torch
    from paper_2312_05800_gb300 import binding
    u = torch.full((n, 32), float("nan"), dtype=torch.float32, device="cuda")
    binding.chem_mlp_forward(net, n, T.shape[0], to_dev(T), to_dev(p), to_dev(Y), u, 32)
    torch.cuda.synchronize()
    assert net.error() == 0
    return u.cpu().numpy()


@pytest.mark.parametrize("n,hidden,chunk", [(3001, (1600, 800, 400), 2048), (20000, (1600, 800, 400), 8192),
                                            (1000, (640, 256, 64), 4096), (2600, (1600, 560, 400), 1024)])
def test_fused_layers_are_bitwise_the_two_launches(n, hidden, chunk):
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats = _problem(n, hidden, 2071)
    net = _net(widths, layers, stats, chunk=chunk)
    expect = binding.CHEM_FUSE_34 if hidden[2] == 400 else 0
    assert net.fusion == expect
    uf = _u(net, T, p, Y, n)
    k = widths[4]
    net.set_fusion(0)
    assert net.fusion == 0
    u2 = _u(net, T, p, Y, n)
    assert np.array_equal(uf[:, :k], u2[:, :k]), np.argwhere(uf[:, :k] != u2[:, :k])[:5]
    net.set_fusion(binding.CHEM_FUSE_34)
    assert net.fusion == expect
    # and against the oracle with the device's BF16 rounding points
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], round_bf16=True)
    rms = np.sqrt(np.mean(uq ** 2))
    err = np.abs(uf[:, :widths[4]].astype(np.float64) - uq)
    # (the same bounds as test_gpu_mlp.py's forward parity, with the fraction inside the tight band
    # at 99.95 %: a BF16 rounding flip of one hidden unit moves an output by one BF16 step of it)
    assert np.mean(err <= 1e-2 * (np.abs(uq) + rms)) >= 0.9995
    assert np.all(err <= 3e-2 * (np.abs(uq) + rms))
    net.free()


def test_fusion_is_off_where_it_does_not_apply():
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats = _problem(256, (600, 200, 96), 2072)    # h3 not 400 units
    net = _net(widths, layers, stats)
    assert not net.fused
    with pytest.raises(binding.ChemError):
        net.set_fusion(1)                        # only CHEM_FUSE_34 (or 0) is a fusion mask
    net.free()
