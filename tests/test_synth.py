"""Seeded input generator: determinism, element balance, coverage and state sanity."""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth


@pytest.mark.parametrize("name,N,R,ntroe,n3b", [("c1", 9, 20, 0, 4), ("c2", 30, 180, 18, 27), ("c5", 53, 325, 33, 49)])
def test_mechanism_shape_and_balance(name, N, R, ntroe, n3b):
    m = synth.get_mech(name)
    assert (m.N, m.R) == (N, R)
    assert int((m.rtype == 2).sum()) == ntroe and int((m.rtype == 1).sum()) == n3b
    nr, npd = m.nu()
    assert np.all((npd - nr) @ m.elem == 0)
    used = (nr + npd).sum(axis=0) > 0
    assert used.sum() == N - 1 and not used[m.bath]
    fresh = synth.make_mech(name, N, R, ntroe, n3b, m.elements, {"c1": 1001, "c2": 1002, "c5": 1005}[name])
    assert synth.mech_to_bytes(fresh) == synth.mech_to_bytes(m)


def test_states_sum_to_one_and_are_seeded():
    m = synth.mech_c2()
    a = synth.states_profiles(m, 1000, 9)
    b = synth.states_profiles(m, 1000, 9)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    T, p, Y = a
    assert np.abs(Y[:, :1000].sum(axis=0) - 1).max() < 1e-14
    assert T[:1000].min() >= 300.0 and T[:1000].max() < 2800.0
    assert np.all(Y[:, :1000] > 0)
    # the bath species has the largest mean mass fraction
    assert int(np.argmax(Y[:, :1000].mean(axis=1))) == m.bath
    m1 = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m1, 4096, 2001)
    assert T.shape[0] % 4 == 0 and np.all(p[:4096] == synth.P_ATM)


def test_perturbation_fraction():
    m = synth.mech_c2()
    T, p, Y = synth.states_profiles(m, 5000, 3)
    T2, Y2, mask = synth.perturb_off_manifold(T, Y, 5000, 0.02, 4)
    assert mask.sum() == 100
    assert np.allclose(np.abs(T2[mask] - T[mask])[T[mask] > 600], 300.0)
    assert np.abs(Y2[:, :5000].sum(axis=0) - 1).max() < 1e-14


def test_state_seeds_sample_one_distribution():
    # different state seeds draw from the same distribution (per-species statistics agree)
    m = synth.mech_c2()
    a = synth.states_profiles(m, 20000, 11)[2][:, :20000]
    b = synth.states_profiles(m, 20000, 12)[2][:, :20000]
    la, lb = np.log10(a).mean(axis=1), np.log10(b).mean(axis=1)
    assert np.abs(la - lb).max() < 0.05


@pytest.mark.parametrize("name", ["c1", "c2", "c5"])
def test_seeded_parameter_ranges(name):
    # the stated draws: log10 A ~ U[8, 14] in cm-mol-s (converted to SI by 1e-6 per order above one),
    # beta ~ U[-1.5, 1.5], Ea ~ U[0, 40] kcal/mol; Troe a, T***, T*, T** and log10 A0 - log10 A_inf
    # ~ U[2, 5]; third-body efficiencies U[0.5, 2.5] on three species, 1 elsewhere; LJ sigma and eps/k
    m = synth.get_mech(name)
    order = (m.reac >= 0).sum(axis=1) + (m.rtype == 1)          # a plain third body adds one order
    la = np.log10(m.A) + 6.0 * (order - 1)
    assert la.min() >= 8.0 - 1e-9 and la.max() <= 14.0 + 1e-9
    assert m.beta.min() >= -1.5 and m.beta.max() <= 1.5
    kcal = m.Ea / 4184.0
    assert kcal.min() >= 0.0 and kcal.max() <= 40.0
    troe = m.rtype == 2
    if troe.any():
        d = np.log10(m.A0[troe]) - np.log10(m.A[troe]) + 6.0       # k0 carries one more order
        assert d.min() >= 2.0 - 1e-9 and d.max() <= 5.0 + 1e-9
        a, t3, t1, t2 = m.troe[troe].T
        assert a.min() >= 0.3 and a.max() <= 0.8 and t3.min() >= 50 and t3.max() <= 300
        assert t1.min() >= 500 and t1.max() <= 3000 and t2.min() >= 2000 and t2.max() <= 8000
    tb = m.rtype != 0
    if tb.any():
        e = m.eff[tb]
        assert np.all((e != 1.0).sum(axis=1) <= 3)
        off = e[e != 1.0]
        assert off.min() >= 0.5 and off.max() <= 2.5
    assert np.all(m.eff[~tb] == 1.0)
    assert m.sigma.min() >= 2.5 and m.sigma.max() <= 5.0
    assert m.eps_k.min() >= 50.0 and m.eps_k.max() <= 600.0
    # every reaction runs exothermic in its forward direction
    nr, npd = m.nu()
    assert np.all((npd - nr) @ m.hf298 <= 0.0)
