"""The stiff integrator's mixed mode (CHEM_ODE_MIXED: FP32 rate exponentials and
fall-off blending, FP32 LU with one FP64 iterative-refinement step per stage
solve) against the FP64 oracle.

* At rtol 1e-5, the tightest tolerance it takes, the mixed mode stays within
  20 rtol of the oracle's tight integration (the FP32 parts perturb the rates by
  about 1e-6 relative and the refined solves are FP64-grade); below it the call
  integrates in FP64 (bitwise the FP64 mode).
* At the throughput setting (rtol 1e-2) on on-manifold and off-manifold cells,
  its error against the oracle's tight integration (relative L2 of dY over the
  major species, max |dT|) is within 1.5x (+1e-4, +0.01 K) of the FP64 mode's
  at the same tolerance.
* A team of four warps per cell gives bitwise the one-warp result, as in FP64.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu
DT = 1.0e-6
TIGHT = dict(rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=20000)
LOOSE = dict(rtol=1e-2, atol_Y=1e-8, atol_T=1e-2, h0=1e-9, max_steps=10000)


def _gpu(name, T, p, Y, n, ld, mode, **opts):
    import torch
    from paper_2312_05800_gb300 import binding
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -7, dtype=torch.int32, device="cuda")
    ns = torch.zeros(ld, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(dev_mech(name), n, ld, DT, binding.make_opts(mode=mode, **opts), Td, pd, Yd, st, ns)
    torch.cuda.synchronize()
    return Td.cpu().numpy(), Yd.cpu().numpy(), st.cpu().numpy(), ns.cpu().numpy()


def _err(mech, T0, Y0, Ta, Ya, Tr, Yr, n):
    major = [k for k in range(mech.N) if k != mech.bath and Y0[k, :n].mean() >= 1e-2]
    rel = max(np.linalg.norm((Ya[k, :n] - Y0[k, :n]) - (Yr[k, :n] - Y0[k, :n]))
              / np.linalg.norm(Yr[k, :n] - Y0[k, :n]) for k in major)
    return rel, float(np.abs(Ta[:n] - Tr[:n]).max())


@pytest.mark.parametrize("name,n", [("c2", 203), ("c5", 37)])
def test_mixed_moderate_tolerance_close_to_oracle(oracle, name, n):
    # rtol 1e-5, the tightest the mixed mode takes: within 20 rtol of the oracle's tight integration
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech(name)
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_profiles(m, n, 2101, ld)
    opts = dict(rtol=1e-5, atol_Y=1e-11, atol_T=1e-5, h0=1e-9, max_steps=20000)
    Tg, Yg, sg, _ = _gpu(name, T, p, Y, n, ld, binding.CHEM_ODE_MIXED, **opts)
    To, Yo, so, _ = oracle.step_stiff(m, T, p, Y, DT, ncells=n, **TIGHT)
    assert np.all(sg[:n] == 0) and np.all(so[:n] == 0)
    assert np.all(np.abs(Tg[:n] - To[:n]) <= 2e-4 * To[:n]), np.abs(Tg[:n] / To[:n] - 1).max()
    err = np.abs(Yg[:, :n] - Yo[:, :n]) - (2e-4 * np.abs(Yo[:, :n]) + 2e-10)
    assert np.all(err <= 0), err.max()


def test_mixed_below_its_tolerance_integrates_in_fp64(oracle):
    # a tighter rtol than 1e-5 takes the FP64 arithmetic: bitwise the FP64 mode's result
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech("c2")
    n = 203
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_profiles(m, n, 2104, ld)
    a = _gpu("c2", T, p, Y, n, ld, binding.CHEM_ODE_MIXED, **TIGHT)
    b = _gpu("c2", T, p, Y, n, ld, binding.CHEM_ODE_FP64, **TIGHT)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("off_manifold", [False, True])
def test_mixed_throughput_setting_error(oracle, off_manifold):
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech("c2")
    n = 600
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_profiles(m, n, 2102, ld)
    if off_manifold:
        T, Y, _ = synth.perturb_off_manifold(T, Y, n, 1.0, 2103)
    To, Yo, so, _ = oracle.step_stiff(m, T, p, Y, DT, ncells=n, **TIGHT)
    assert np.all(so[:n] == 0)
    Tx, Yx, sx, _ = _gpu("c2", T, p, Y, n, ld, binding.CHEM_ODE_MIXED, **LOOSE)
    Td, Yd, sd, _ = _gpu("c2", T, p, Y, n, ld, binding.CHEM_ODE_FP64, **LOOSE)
    assert np.all(sx[:n] == 0) and np.all(sd[:n] == 0)
    rx, tx = _err(m, T, Y, Tx, Yx, To, Yo, n)
    rd, td = _err(m, T, Y, Td, Yd, To, Yo, n)
    assert rx <= 1.5 * rd + 1e-4, (rx, rd)
    assert tx <= 1.5 * td + 0.01, (tx, td)


def test_mixed_team_mode_is_bitwise_warp_mode():
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech("c2")
    n_big = 2000
    T, p, Y = synth.states_profiles(m, n_big, 31, synth.padded_ld(n_big))
    Tw, Yw, sw, nw = _gpu("c2", T, p, Y, n_big, T.shape[0], binding.CHEM_ODE_MIXED, **LOOSE)
    n = 100
    Tt, Yt, st, nt = _gpu("c2", T, p, Y, n, T.shape[0], binding.CHEM_ODE_MIXED, **LOOSE)
    assert np.array_equal(st[:n], sw[:n]) and np.array_equal(nt[:n], nw[:n])
    assert np.array_equal(Tt[:n], Tw[:n]) and np.array_equal(Yt[:, :n], Yw[:, :n])


def test_mode_is_validated():
    import torch
    from paper_2312_05800_gb300 import binding
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.ChemError):
        binding.chem_step_stiff(dev_mech("c1"), 4, 8, DT, binding.make_opts(mode=5), x, x,
                                torch.zeros(9, 8, dtype=torch.float64, device="cuda"), s)
