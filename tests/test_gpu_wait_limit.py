"""The tensor-core pipeline's bounded waits run out on purpose (failure detection
without a GPU fault): with a limit of one try per wait, the network's GEMMs give
up, record a timeout code in the handle's error word and unwind (they wait with
the full limit for the copies and tensor-core operations they issued, free
their tensor memory and return). The call returns, the device stays usable,
and a fresh handle then computes the forward that matches the oracle."""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _net(widths, layers, stats, **kw):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], **kw)
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    return net


def test_wait_limit_runs_out_and_a_fresh_handle_is_correct():
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.get_mech("c2")
    n = 65536
    T, p, Y = synth.states_profiles(mech, n, 2061, synth.padded_ld(n))
    widths = [mech.N + 2, 1600, 800, 400, mech.N - 1]
    layers = synth.mlp_layers(widths, 5061)
    mu_x, sd_x = M.zscore_stats(M.features(T[:n], p[:n], Y[:, :n]))
    stats = (mu_x, sd_x, np.zeros(mech.N - 1), np.full(mech.N - 1, 1e-4))
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    u = torch.zeros((n, 32), dtype=torch.float32, device="cuda")
    bad = _net(widths, layers, stats, chunk=n)
    assert bad.error() == 0
    bad.set_wait_limit(1)
    binding.chem_mlp_forward(bad, n, T.shape[0], Td, pd, Yd, u, 32)     # returns; the failure is recorded
    code = bad.error()
    assert code in (1, 2, 3, 4), code
    bad.free()
    # the device still works: a fresh handle with the default limit gives the oracle's forward
    good = _net(widths, layers, stats, chunk=n)
    m = 4096
    binding.chem_mlp_forward(good, m, T.shape[0], Td, pd, Yd, u, 32)
    torch.cuda.synchronize()
    assert good.error() == 0
    ug = u.double().cpu().numpy()[:m, :widths[4]]
    uq = A.forward_u(mech, layers, stats, T[:m], p[:m], Y[:, :m], round_bf16=True)
    rms = np.sqrt(np.mean(uq ** 2))
    assert np.all(np.abs(ug - uq) <= 3e-2 * (np.abs(uq) + rms))
    # a limit of 0 restores the default
    good.set_wait_limit(0)
    binding.chem_mlp_forward(good, m, T.shape[0], Td, pd, Yd, u, 32)
    assert good.error() == 0
    good.free()
