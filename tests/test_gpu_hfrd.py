"""The random training-data generation of Sec. 3.1 (Eq. 1-4, Table 1, the lean
equilibrium-air blend) on the GPU against oracle/hfrd.py, on the same random draws.

* chem_hfrd_perturb: T' and p' bitwise (the same rounded FP64 operations);
  Y' within 1e-14 relative (the power function's last bits may differ); the
  keep mask bit for bit, except states whose H/C, O/N or phi lies within 1e-12
  relative of a Table 1 bound in the oracle (where the two sums' rounding
  orders may decide differently; the test reports how many there are and
  requires it to be a negligible fraction). Ragged n over several blocks.
* chem_hfrd_blend: bitwise the oracle's blend.
* train.lean_equilibrium (props_eval Newton + chem_step_stiff over 1 s)
  against the oracle's adiabatic equilibrium: T within 1e-6 K, Y within 1e-10.
* train.hfrd_states keeps only states that pass Table 1.
"""
import numpy as np
import pytest

from oracle import hfrd as H
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def test_perturb_matches_oracle_on_the_same_draws():
    import torch
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech("c2")
    n = 20001
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_profiles(m, n, 2081, ld)
    ranges = H.dataset_ranges(m, T[:n], p[:n], Y[:, :n])
    rng = np.random.default_rng(2082)
    c = np.zeros((3 + m.N, ld))
    c[:, :n] = rng.uniform(-1.0, 1.0, (3 + m.N, n))
    To, po, Yo, ok = H.perturb(m, T[:n], p[:n], Y[:, :n], c[:, :n], ranges)
    keep_o = H.accept(m, Yo, ok)
    prm = binding.hfrd_params(T_min=ranges[0], T_max=ranges[1], p_min=ranges[2], p_max=ranges[3], Yb_min=ranges[4],
                              Yb_max=ranges[5])
    T2 = torch.zeros(ld, dtype=torch.float64, device="cuda")
    p2 = torch.zeros_like(T2)
    Y2 = torch.zeros((m.N, ld), dtype=torch.float64, device="cuda")
    keep = torch.full((ld,), 7, dtype=torch.uint8, device="cuda")
    binding.chem_hfrd_perturb(dev_mech("c2"), prm, synth.element_table(m), n, ld, to_dev(T), to_dev(p), to_dev(Y),
                              to_dev(c), T2, p2, Y2, keep)
    torch.cuda.synchronize()
    Tg, pg, Yg, kg = T2.cpu().numpy(), p2.cpu().numpy(), Y2.cpu().numpy(), keep.cpu().numpy()
    assert np.array_equal(Tg[:n], To) and np.array_equal(pg[:n], po)
    assert np.all(kg[n:] == 7)                                  # nothing past n is written
    assert np.all(np.abs(Yg[:, :n][:, ok] - Yo[:, ok]) <= 1e-14 * np.abs(Yo[:, ok]) + 1e-300)
    # the mask: bit for bit away from the Table 1 bounds
    hc, on, phi = H.ratios(m, Yo)
    near = np.zeros(n, bool)
    for v, (lo, hi) in ((hc, H.HC_RANGE), (on, H.ON_RANGE), (phi, H.PHI_RANGE)):
        with np.errstate(invalid="ignore"):
            near |= ok & ((np.abs(v - lo) <= 1e-12 * abs(lo)) | (np.abs(v - hi) <= 1e-12 * abs(hi)))
    assert near.sum() <= 2, near.sum()
    assert np.array_equal(kg[:n][~near].astype(bool), keep_o[~near])
    # the draws reject some states and keep others
    assert 0.05 < keep_o.mean() < 0.95, keep_o.mean()


def test_blend_matches_oracle():
    import torch
    from paper_2312_05800_gb300 import binding
    m = synth.get_mech("c2")
    n = 1001
    ld = synth.padded_ld(n)
    rng = np.random.default_rng(2083)
    s = np.zeros(ld)
    s[:n] = rng.uniform(0.0, 1.0, n)
    Ya = rng.dirichlet(np.ones(m.N))
    Yb = rng.dirichlet(np.ones(m.N))
    T = torch.zeros(ld, dtype=torch.float64, device="cuda")
    Y = torch.zeros((m.N, ld), dtype=torch.float64, device="cuda")
    binding.chem_hfrd_blend(m.N, n, ld, to_dev(s), 1750.0, Ya, 300.0, Yb, T, Y)
    torch.cuda.synchronize()
    To, Yo = H.blend(s[:n], 1750.0, Ya, 300.0, Yb)
    assert np.array_equal(T.cpu().numpy()[:n], To)
    assert np.array_equal(Y.cpu().numpy()[:, :n], Yo)


def test_lean_equilibrium_matches_oracle():
    from paper_2312_05800_gb300 import train
    m = synth.get_mech("c2")
    Tg, Yg = train.lean_equilibrium(dev_mech("c2"), m, 0.45)
    To, Yo = H.adiabatic_equilibrium(m, 0.45)
    assert abs(Tg - To) <= 1e-6, (Tg, To)
    assert np.all(np.abs(Yg - Yo) <= 1e-10), np.abs(Yg - Yo).max()


def test_hfrd_states_pass_table_1():
    from paper_2312_05800_gb300 import train
    m = synth.get_mech("c2")
    n, ld, T, p, Y = train.hfrd_states(dev_mech("c2"), m, 4000, 2084, lean_frac=0.0)
    assert 100 < n < 4000
    Yh = Y.cpu().numpy()[:, :n]
    assert H.accept(m, Yh).mean() >= 0.999
    assert np.all(T.cpu().numpy()[:n] > 0) and np.allclose(Yh.sum(axis=0), 1.0, rtol=0, atol=1e-12)
