"""Faults injected from the host: nothing here faults, traps or hangs a GPU.

A network with one non-finite weight predicts NaN for every cell. Without the
out-of-distribution guard every cell keeps its state, bit for bit, with status
CHEM_CELL_NONFINITE; with the guard every cell goes to the stiff fallback, whose
result equals chem_step_stiff's with the same options (status CHEM_CELL_FALLBACK).
Non-finite states and a step budget of one step are covered by the stiff tests
(status codes 4 and 2). The file runs after every parity test (only the
allocation-free entry point's test comes later)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _net(mech, T, p, Y, n, nan_weight):
    from paper_2312_05800_gb300 import binding
    widths = [mech.N + 2, 64, 32, 16, mech.N - 1]
    layers = synth.mlp_layers(widths, 77)
    if nan_weight:
        W0 = layers[0][0].copy()
        W0[3, 2] = np.nan
        layers = [(W0, layers[0][1])] + layers[1:]
    mu_x, sd_x = M.zscore_stats(M.features(T[:n], p[:n], Y[:, :n]))
    net = binding.Mlp(dev_mech("c1"), hidden=widths[1:4], dt=1e-6)
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(mu_x, sd_x, np.zeros(mech.N - 1), np.full(mech.N - 1, 1e-4))
    return net


def test_non_finite_predictions_never_reach_the_state():
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.mech_c1()
    n = 256
    T, p, Y = synth.states_dirichlet(mech, n, 2081)
    ld = T.shape[0]
    opts = binding.make_opts(rtol=1e-6, atol_Y=1e-13, atol_T=1e-6, h0=1e-9, max_steps=20000)
    # finite weights, no guard: every cell predicted
    good = _net(mech, T, p, Y, n, False)
    st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    binding.chem_step_ann(dev_mech("c1"), good, n, ld, 1e-6, 0, opts, to_dev(T), to_dev(p), to_dev(Y), st)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy()[:n] == binding.CELL_OK)
    good.free()
    # a NaN weight, no guard: the state is kept and flagged
    bad = _net(mech, T, p, Y, n, True)
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    binding.chem_step_ann(dev_mech("c1"), bad, n, ld, 1e-6, 0, opts, Td, pd, Yd, st)
    torch.cuda.synchronize()
    assert bad.error() == 0
    assert np.all(st.cpu().numpy()[:n] == 4)                      # CHEM_CELL_NONFINITE
    assert np.array_equal(Td.cpu().numpy(), T) and np.array_equal(Yd.cpu().numpy(), Y)
    # the same network behind the guard (fitted on these cells, so none is off-grid): every cell
    # falls back to the stiff integrator
    binding.chem_mlp_fit_ood(bad, dev_mech("c1"), n, ld, to_dev(T), to_dev(p), to_dev(Y), mech.roles["water"], 64, 1)
    Ta, Ya = to_dev(T), to_dev(Y)
    binding.chem_step_ann(dev_mech("c1"), bad, n, ld, 1e-6, 0, opts, Ta, pd, Ya, st)
    Ts, Ys = to_dev(T), to_dev(Y)
    ss = torch.zeros(ld, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(dev_mech("c1"), n, ld, 1e-6, opts, Ts, pd, Ys, ss)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy()[:n] == binding.CELL_FALLBACK)
    assert np.all(ss.cpu().numpy()[:n] == binding.CELL_OK)
    assert np.array_equal(Ta.cpu().numpy(), Ts.cpu().numpy()) and np.array_equal(Ya.cpu().numpy(), Ys.cpu().numpy())
    bad.free()
