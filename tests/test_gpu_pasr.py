"""chem_pasr (Sec. 4.1: PaSR scaling kappa = tau_c / (tau_c + tau_mix)) against the oracle.

* c2 stratified-profile cells (ragged count, several blocks per SM), seeded Taylor and
  Kolmogorov time scales spread over four decades: tau_c within 1e-9 relative (the FP64
  right-hand sides agree to about 1e-12; the maximum over species is continuous), kappa
  within 1e-9, and the scaled step T0 + kappa (T1 - T0), Y0 + kappa (Y1 - Y0) within FP64
  rounding of the oracle's, where (T1, Y1) is the GPU stiff integrator's step.
* The qualifying decision Y_k >= y_min is taken on the same FP64 inputs on both sides:
  cells whose species sit exactly at y_min, and a y_min that leaves no species (tau_c = inf,
  kappa = 1, the step unchanged).
* Without T and Y only tau_c and kappa are written; cells past ncells are untouched.
"""
import numpy as np
import pytest

from oracle import pasr as P
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _times(n, seed):
    rng = np.random.default_rng(seed)
    ld = synth.padded_ld(n)
    tt = np.full(ld, 1.0)
    tk = np.full(ld, 1.0)
    tt[:n] = 10.0 ** rng.uniform(-6, -2, n)
    tk[:n] = 10.0 ** rng.uniform(-7, -3, n)
    return tt, tk


def test_pasr_parity_c2(oracle):
    import torch
    from paper_2312_05800_gb300 import binding
    n = 3001
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, n, 2061, synth.padded_ld(n))
    ld = T.shape[0]
    tt, tk = _times(n, 2062)
    dm = dev_mech("c2")
    T0d, pd, Y0d = to_dev(T), to_dev(p), to_dev(Y)
    T1d, Y1d = T0d.clone(), Y0d.clone()
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(dm, n, ld, 1e-6, binding.make_opts(rtol=1e-6, atol_Y=1e-13, atol_T=1e-6, h0=1e-9,
                                                               max_steps=20000), T1d, pd, Y1d, st)
    torch.cuda.synchronize()
    T1, Y1 = T1d.cpu().numpy(), Y1d.cpu().numpy()
    tc = torch.full((ld,), -7.0, dtype=torch.float64, device="cuda")
    kp = torch.full((ld,), -7.0, dtype=torch.float64, device="cuda")
    y_min = 1e-6
    binding.chem_pasr(dm, n, ld, y_min, T0d, pd, Y0d, to_dev(tt), to_dev(tk), T1d, Y1d, tc, kp)
    torch.cuda.synchronize()
    otc = P.chemical_time(mech, T[:n], p[:n], Y[:, :n], y_min)
    okp = P.kappa(otc, tt[:n], tk[:n])
    gtc, gkp = tc.cpu().numpy(), kp.cpu().numpy()
    assert np.all(np.isfinite(otc))
    assert np.allclose(gtc[:n], otc, rtol=1e-9, atol=0), np.abs(gtc[:n] / otc - 1).max()
    assert np.allclose(gkp[:n], okp, rtol=1e-9, atol=0)
    assert np.all(gtc[n:] == -7.0) and np.all(gkp[n:] == -7.0)
    assert okp.min() < 0.1 and okp.max() > 0.9             # mixing-limited and chemistry-limited cells both occur
    To, Yo = P.apply(T[:n], Y[:, :n], T1[:n], Y1[:, :n], okp)
    Tg, Yg = T1d.cpu().numpy(), Y1d.cpu().numpy()
    assert np.allclose(Tg[:n], To, rtol=1e-12, atol=0)
    assert np.all(np.abs(Yg[:, :n] - Yo) <= 1e-9 * np.abs(Y1[:, :n] - Y[:, :n]) + 4e-16 * np.abs(Yo) + 1e-300)
    assert np.array_equal(Tg[n:], T1[n:]) and np.array_equal(Yg[:, n:], Y1[:, n:])


def test_pasr_y_min_edges(oracle):
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.get_mech("c1")
    n = 64
    T, p, Y = synth.states_dirichlet(mech, n, 2063)
    y_min = float(np.sort(Y[:, 0])[mech.N // 2])       # one cell's species sits exactly at y_min
    Y[:, 1] = Y[:, 0]
    T[1] = T[0]
    tt, tk = _times(n, 2064)
    dm = dev_mech("c1")
    tc = torch.zeros(n, dtype=torch.float64, device="cuda")
    kp = torch.zeros(n, dtype=torch.float64, device="cuda")
    binding.chem_pasr(dm, n, n, y_min, to_dev(T), to_dev(p), to_dev(Y), to_dev(tt), to_dev(tk), None, None, tc, kp)
    torch.cuda.synchronize()
    otc = P.chemical_time(mech, T, p, Y, y_min)
    ok = np.isfinite(otc)
    g = tc.cpu().numpy()
    assert np.array_equal(np.isfinite(g), ok)
    assert np.allclose(g[ok], otc[ok], rtol=1e-9, atol=0)
    assert np.allclose(kp.cpu().numpy(), P.kappa(otc, tt[:n], tk[:n]), rtol=1e-9, atol=0)
    # no species reaches y_min = 2: tau_c = inf, kappa = 1, the step comes back unchanged
    T1d, Y1d = to_dev(T + 10.0), to_dev(Y * 0.5)
    binding.chem_pasr(dm, n, n, 2.0, to_dev(T), to_dev(p), to_dev(Y), to_dev(tt), to_dev(tk), T1d, Y1d, tc, kp)
    torch.cuda.synchronize()
    assert np.all(np.isinf(tc.cpu().numpy())) and np.all(kp.cpu().numpy() == 1.0)
    assert np.allclose(T1d.cpu().numpy(), T + 10.0, rtol=1e-15) and np.allclose(Y1d.cpu().numpy(), Y * 0.5,
                                                                                    rtol=0, atol=1e-16)
    with pytest.raises(binding.ChemError):
        binding.chem_pasr(dm, n, n, 1e-6, to_dev(T), to_dev(p), to_dev(Y), to_dev(tt), to_dev(tk), T1d, None)
    with pytest.raises(binding.ChemError):
        binding.chem_pasr(dm, n, n, 0.0, to_dev(T), to_dev(p), to_dev(Y), to_dev(tt), to_dev(tk))
