"""props_eval on the GPU against the FP64 oracle (Sec. 2: thermal and
transport properties per cell; Sec. 3.1: mixture-averaged transport).

FP64: 1e-12 relative. FP32: 1e-5 relative for cp, mu, lambda and D_k; for h
the scale is sum_k Y_k |h_k| because h crosses zero. Sizes span several
blocks and a ragged tail; the full 2M-cell workload is checked on sampled cells.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, h_scale, to_dev

pytestmark = pytest.mark.gpu


def _run(name, T, p, Y, n, ld, dtype):
    import torch
    from paper_2312_05800_gb300 import binding
    m = dev_mech(name)
    td = torch.float32 if dtype == binding.CHEM_F32 else torch.float64          # state
    to = torch.float64 if dtype == binding.CHEM_F64 else torch.float32          # properties
    Td, pd, Yd = to_dev(T, td), to_dev(p, td), to_dev(Y, td)
    outs = [torch.full((ld,), float("nan"), dtype=to, device="cuda") for _ in range(4)]
    Dk = torch.full((m.N, ld), float("nan"), dtype=to, device="cuda")
    binding.props_eval(m, n, ld, dtype, Td, pd, Yd, *outs, Dk)
    torch.cuda.synchronize()
    return [o.double().cpu().numpy() for o in outs] + [Dk.double().cpu().numpy()]


def _compare(oracle, name, T, p, Y, n, got, rtol):
    mech = synth.get_mech(name)
    cp, h, mu, lam, Dk = oracle.props(mech, T, p, Y, ncells=n)
    hs = h_scale(oracle, mech, T, Y, n)
    assert np.all(np.abs(got[0][:n] - cp[:n]) <= rtol * np.abs(cp[:n]))
    assert np.all(np.abs(got[1][:n] - h[:n]) <= rtol * hs)
    assert np.all(np.abs(got[2][:n] - mu[:n]) <= rtol * np.abs(mu[:n]))
    assert np.all(np.abs(got[3][:n] - lam[:n]) <= rtol * np.abs(lam[:n]))
    assert np.all(np.abs(got[4][:, :n] - Dk[:, :n]) <= rtol * np.abs(Dk[:, :n]))


def test_fp64_c1_full(oracle):
    from paper_2312_05800_gb300 import binding
    m = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m, 4096, 2001)
    got = _run("c1", T, p, Y, 4096, 4096, binding.CHEM_F64)
    _compare(oracle, "c1", T, p, Y, 4096, got, 1e-12)


@pytest.mark.parametrize("name,n", [("c1", 4093), ("c2", 65531), ("c5", 8189)])
def test_fp32_ragged(oracle, name, n):
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech(name)
    ld = synth.padded_ld(n) + 8
    T, p, Y = (synth.states_dirichlet(m, n, 7, ld) if name == "c1" else synth.states_profiles(m, n, 7, ld))
    got = _run(name, T, p, Y, n, ld, binding.CHEM_F32)
    _compare(oracle, name, T, p, Y, n, got, 1e-5)
    # cells past ncells are untouched
    assert np.all(np.isnan(got[0][n:])) and np.all(np.isnan(got[4][:, n:]))


def test_fp64_c2_and_pure_species(oracle):
    from paper_2312_05800_gb300 import binding
    m = synth.mech_c2()
    n = 1024
    T, p, Y = synth.states_profiles(m, n, 11)
    Y[:, :m.N] = 0.0
    for k in range(m.N):
        Y[k, k] = 1.0          # the first N cells are pure species
    got = _run("c2", T, p, Y, n, synth.padded_ld(n), binding.CHEM_F64)
    _compare(oracle, "c2", T, p, Y, n, got, 1e-12)


def test_zero_cells_and_partial_outputs():
    import torch
    from paper_2312_05800_gb300 import binding
    m = dev_mech("c2")
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    binding.props_eval(m, 0, 8, binding.CHEM_F32, x, x, torch.zeros(30, 8, device="cuda"), x)
    T, p, Y = synth.states_profiles(synth.mech_c2(), 8, 1)
    cp = torch.zeros(8, device="cuda")
    binding.props_eval(m, 8, 8, binding.CHEM_F32, to_dev(T, torch.float32), to_dev(p, torch.float32),
                       to_dev(Y, torch.float32), cp, None, None, None, None)
    torch.cuda.synchronize()
    assert torch.all(cp > 0)
    with pytest.raises(binding.ChemError):
        binding.props_eval(m, 9, 8, binding.CHEM_F32, x, x, x, cp)


def test_full_size_sampled(oracle):
    # the 2,097,152-cell workload in the bench's launch configuration; sampled cells vs the oracle
    import torch
    from paper_2312_05800_gb300 import binding
    m = synth.mech_c2()
    n = 2097152
    T, p, Y = synth.states_profiles(m, n, 2002)
    got = _run("c2", T, p, Y, n, n, binding.CHEM_F32)
    idx = np.random.default_rng(0).choice(n, 2048, replace=False)
    idx = np.concatenate([idx, [0, n - 1]])
    Ts, ps, Ys = T[idx].copy(), p[idx].copy(), Y[:, idx].copy()
    sub = [g[idx] for g in got[:4]] + [got[4][:, idx]]
    _compare(oracle, "c2", Ts, ps, Ys, idx.size, sub, 1e-5)


@pytest.mark.parametrize("name,n", [("c2", 65531), ("c5", 8189), ("c2", 1000003), ("c1", 300001)])
def test_thermo_only_pass(oracle, name, n):
    # without transport outputs props_eval runs the staged thermo-only kernel: the same FP32
    # arithmetic per species and the same species order as the full pass, so cp and h are bitwise
    # the full pass's; from FP32 and from FP64 state; a ragged last tile (n not a multiple of the
    # 512-cell tile, nor of 4); several tiles per CTA at the larger sizes (the stage ring wraps);
    # cells past n untouched
    import torch
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech(name)
    ld = synth.padded_ld(n) + 8
    T, p, Y = synth.states_profiles(m, n, 13, ld)
    for dtype, td in ((binding.CHEM_F32, torch.float32), (binding.CHEM_F64_IN_F32, torch.float64)):
        full = _run(name, T, p, Y, n, ld, dtype)
        Td, pd, Yd = to_dev(T, td), to_dev(p, td), to_dev(Y, td)
        cp = torch.full((ld,), float("nan"), dtype=torch.float32, device="cuda")
        h = torch.full((ld,), float("nan"), dtype=torch.float32, device="cuda")
        binding.props_eval(dev_mech(name), n, ld, dtype, Td, pd, Yd, cp, h, None, None, None)
        torch.cuda.synchronize()
        cp, h = cp.double().cpu().numpy(), h.double().cpu().numpy()
        assert np.array_equal(cp[:n], full[0][:n]), np.abs(cp[:n] / full[0][:n] - 1).max()
        assert np.array_equal(h[:n], full[1][:n]), np.abs(h[:n] - full[1][:n]).max()
        assert np.all(np.isnan(cp[n:])) and np.all(np.isnan(h[n:]))
