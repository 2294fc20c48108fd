"""Zero cells is a no-op for every per-cell entry point of the learned path, PaSR and
the random-data generation (props_eval and chem_step_stiff have theirs in their own
files): each call returns without an error and writes nothing, on a 30-species
mechanism and a small network whose parameters come from the seeded generator."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech

pytestmark = pytest.mark.gpu

LD = 8


def _net():
    from paper_2312_05800_gb300 import binding
    mech = synth.get_mech("c2")
    widths = [mech.N + 2, 256, 128, 64, mech.N - 1]
    T, p, Y = synth.states_profiles(mech, 64, 2091)
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], dt=1e-6)
    net.set_params(synth.flatten_layers(synth.mlp_layers(widths, 2092)))
    mu_x, sd_x = M.zscore_stats(M.features(T[:64], p[:64], Y[:, :64]))
    net.set_norm(mu_x, sd_x, np.zeros(mech.N - 1), np.full(mech.N - 1, 1e-4))
    return mech, net


def _sentinel(shape, dtype, value):
    import torch
    return torch.full(shape, value, dtype=dtype, device="cuda")


def test_zero_cells_learned_path():
    import torch
    from paper_2312_05800_gb300 import binding
    mech, net = _net()
    N = mech.N
    T = _sentinel((LD,), torch.float64, 1234.5)
    p = _sentinel((LD,), torch.float64, 101325.0)
    Y = _sentinel((N, LD), torch.float64, 0.25)
    st = _sentinel((LD,), torch.int32, 77)
    u = _sentinel((LD, 32), torch.float32, float("nan"))
    binding.chem_mlp_forward(net, 0, LD, T, p, Y, u, 32)
    binding.chem_step_ann(dev_mech("c2"), net, 0, LD, 1e-6, binding.CHEM_PREC_BF16, None, T, p, Y, st)
    outs = [_sentinel((LD,), torch.float32, -1.0) for _ in range(4)]
    Dk = _sentinel((N, LD), torch.float32, -1.0)
    binding.chem_step_ann_props(dev_mech("c2"), net, 0, LD, 1e-6, binding.CHEM_PREC_BF16, None, T, p, Y, st,
                                *outs, Dk)
    torch.cuda.synchronize()
    assert net.error() == 0
    assert torch.all(T == 1234.5) and torch.all(Y == 0.25) and torch.all(st == 77)
    assert torch.all(torch.isnan(u))
    assert all(torch.all(o == -1.0) for o in outs) and torch.all(Dk == -1.0)
    net.free()


def test_zero_cells_pasr_and_random_data():
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.get_mech("c2")
    N = mech.N
    x = _sentinel((LD,), torch.float64, 3.0)
    Y0 = _sentinel((N, LD), torch.float64, 0.5)
    T1 = _sentinel((LD,), torch.float64, -7.0)
    Y1 = _sentinel((N, LD), torch.float64, -7.0)
    tc, kap = _sentinel((LD,), torch.float64, -7.0), _sentinel((LD,), torch.float64, -7.0)
    binding.chem_pasr(dev_mech("c2"), 0, LD, 1e-6, x, x, Y0, x, x, T1, Y1, tc, kap)
    c = _sentinel((3 + N, LD), torch.float64, 0.0)
    keep = _sentinel((LD,), torch.uint8, 9)
    binding.chem_hfrd_perturb(dev_mech("c2"), binding.hfrd_params(T_min=300.0, T_max=2000.0, p_min=1e5,
                                                                   p_max=1e5, Yb_min=0.7, Yb_max=0.75),
                              synth.element_table(mech), 0, LD, x, x, Y0, c, T1, x, Y1, keep)
    torch.cuda.synchronize()
    for t in (T1, Y1, tc, kap):
        assert torch.all(t == -7.0)
    assert torch.all(keep == 9) and torch.all(x == 3.0)
