"""Pins of the oracle's NASA-7 thermodynamics (Sec. 2: thermal properties per cell).

Each check is fixed by mathematics or by the generator's own data, not by
re-typing the oracle's formulas: continuity at the 1000 K break, the exact
integral relations dH/dT = cp and dS/dT = cp/T, the seeded H(298.15) and
S(298.15), closeness to the seeded cp(T) curve the fit was made from, and the
mass-weighted linearity of the mixture sums.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth

MECHS = ["c1", "c2", "c5"]


@pytest.mark.parametrize("name", MECHS)
def test_nasa_continuity_at_1000K(oracle, name):
    m = synth.get_mech(name)
    for k in range(m.N):
        lo = oracle.species_thermo(m, k, 1000.0 * (1 - 1e-15))
        hi = oracle.species_thermo(m, k, 1000.0)
        for a, b in zip(lo[:3], hi[:3]):
            assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1.0)


@pytest.mark.parametrize("name", MECHS)
def test_dH_dT_equals_cp_and_dS_dT_equals_cp_over_T(oracle, name):
    m = synth.get_mech(name)
    d = 1e-3
    for k in range(m.N):
        for T in (350.0, 700.0, 1500.0, 2800.0):
            cpR = oracle.species_thermo(m, k, T)[0]
            Hp = oracle.species_thermo(m, k, T + d)[1] * (T + d)
            Hm = oracle.species_thermo(m, k, T - d)[1] * (T - d)
            Sp = oracle.species_thermo(m, k, T + d)[2]
            Sm = oracle.species_thermo(m, k, T - d)[2]
            assert abs((Hp - Hm) / (2 * d) - cpR) <= 1e-6 * abs(cpR)
            assert abs((Sp - Sm) / (2 * d) - cpR / T) <= 1e-6 * abs(cpR / T)
            # d(cp/R)/dT by central difference
            cp_p = oracle.species_thermo(m, k, T + d)[0]
            cp_m = oracle.species_thermo(m, k, T - d)[0]
            dcp = oracle.species_thermo(m, k, T)[3]
            assert abs((cp_p - cp_m) / (2 * d) - dcp) <= 1e-6 * max(abs(dcp), 1e-6)


@pytest.mark.parametrize("name", MECHS)
def test_reference_state_values(oracle, name):
    m = synth.get_mech(name)
    for k in range(m.N):
        _, H_RT, S_R, _ = oracle.species_thermo(m, k, 298.15)
        assert abs(H_RT * synth.R_GAS * 298.15 - m.hf298[k]) <= 1e-9 * max(abs(m.hf298[k]), 1e3)
        assert abs(S_R - m.s298[k]) <= 1e-10 * abs(m.s298[k])


def test_cp_close_to_seeded_curve(oracle):
    # the fit reproduces the rigid-rotor + Einstein curve it was made from
    m = synth.mech_c2()
    Ts = np.array([320.0, 600.0, 900.0, 1200.0, 2000.0, 3300.0])
    for k in range(m.N):
        cps = np.array([oracle.species_thermo(m, k, T)[0] for T in Ts])
        na = int(m.elem[k].sum())
        base = 2.5 if na == 1 else (3.5 if na == 2 else 4.0)
        # physically: cp/R between the rigid-rotor value and the full classical limit
        nmodes = 0 if na == 1 else (1 if na == 2 else 3 * na - 6)
        assert np.all(cps > base - 0.3) and np.all(cps < base + nmodes + 0.3)
        assert np.all(np.diff(cps) > -0.1)   # cp grows with T


def test_mixture_sums_single_species_and_linearity(oracle):
    m = synth.mech_c2()
    N = m.N
    T = np.full(4, 1234.5)
    p = np.full(4, synth.P_ATM)
    for k in (0, 3, 17):
        Y = np.zeros((N, 4))
        Y[k] = 1.0
        cp, h, *_ = oracle.props(m, T, p, Y)
        cpR, H_RT, _, _ = oracle.species_thermo(m, k, 1234.5)
        assert abs(cp[0] - cpR * synth.R_GAS / m.W[k]) <= 1e-13 * cp[0]
        assert abs(h[0] - H_RT * synth.R_GAS * 1234.5 / m.W[k]) <= 1e-9 * abs(h[0]) + 1e-6
    rng = np.random.default_rng(5)
    Ya = rng.dirichlet(np.ones(N), 1).T
    Yb = rng.dirichlet(np.ones(N), 1).T
    Y = np.concatenate([Ya, Yb, 0.3 * Ya + 0.7 * Yb, Ya], axis=1)
    cp, h, *_ = oracle.props(m, T, p, Y)
    assert abs(cp[2] - (0.3 * cp[0] + 0.7 * cp[1])) <= 1e-13 * cp[2]
    assert abs(h[2] - (0.3 * h[0] + 0.7 * h[1])) <= 1e-12 * (abs(h[0]) + abs(h[1]))
