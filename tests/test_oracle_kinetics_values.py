"""Value pins of the oracle's rate constants (Sec. 3.1: the reaction ODEs of
the mechanism integrated over dt).

The closed-form tests of test_oracle_kinetics.py use temperature-independent
rate constants and no third body. These pin the remaining factors of the rate
of progress by value, each with a mechanism whose composition follows a closed
form, so that a units slip or a wrong sign in a factor changes the answer:

* Arrhenius: k = A T^beta exp(-Ea / (R T)) with beta != 0 and Ea != 0, at three
  temperatures (a flipped beta, or Ea read in cal/mol, fails);
* third body: A + A (+M) -> C + D with [M] = sum_k eff_k C_k from unequal
  efficiencies (an unweighted or missing [M] fails);
* Troe fall-off: k = k_inf Pr / (1 + Pr) F with Pr = k0 [M] / k_inf. F = 1
  (F_cent = 1) gives the Lindemann form, whose limits are k0 [M] (Pr -> 0) and
  k_inf (Pr -> inf); F itself is checked against values worked by hand from the
  Gilbert-Luther-Troe expressions
      c = -0.4 - 0.67 log10 F_cent,  n = 0.75 - 1.27 log10 F_cent,  d = 0.14,
      log10 F = log10 F_cent / (1 + ((log10 Pr + c) / (n - d (log10 Pr + c)))^2),
      F_cent = (1 - a) exp(-T / T***) + a exp(-T / T*) + exp(-T** / T).

Every species has the same molar mass and the same constant c_p and formation
enthalpy, so T and rho stay constant; products carry a large entropy so that
K_c = e^500 and the reverse rate vanishes.
"""
import numpy as np
import pytest

from tests.mechs import tiny_mech

R = 8.314462618          # J/mol/K
P = 101325.0             # Pa
W = 0.028                # kg/mol, every species
TIGHT = dict(rtol=1e-11, atol_Y=1e-16, atol_T=1e-10)


def _conc_total(T, p=P):
    """C_total = rho / W = p / (R T) (mol/m^3) for equal molar masses."""
    return p / (R * T)


# ---------------------------------------------------------------------------
# Arrhenius
# ---------------------------------------------------------------------------

A_ARR, BETA, EA = 3.65e6, 0.7, 8.0e4     # s^-1 K^-beta, -, J/mol


def _arrhenius_mech():
    # A -> B, bath
    return tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 520.0), (3.5, 0.0, 20.0)],
                     [dict(reac=[0], prod=[1], A=A_ARR, beta=BETA, Ea=EA)])


@pytest.mark.parametrize("T", [800.0, 1500.0, 2200.0])
def test_arrhenius_first_order_decay(oracle, T):
    m = _arrhenius_mech()
    k = A_ARR * T ** BETA * np.exp(-EA / (R * T))
    Y0 = np.array([0.3, 0.1, 0.6])
    # the rate of progress at the start: q = k C_A
    w, q = oracle.rates(m, T, P, Y0)
    CA = _conc_total(T) * Y0[0]
    assert abs(q[0] - k * CA) <= 1e-12 * k * CA
    # the integrated decay over dt = 1/k: Y_A = Y_A0 exp(-k t) exactly
    dt = 1.0 / k
    y, st, _ = oracle.integrate_cell(m, P, dt, np.concatenate([[T], Y0]), **TIGHT)
    assert st == 0
    ref = 0.3 * np.exp(-1.0)
    assert abs(y[1] - ref) <= 1e-9 * ref
    assert abs(y[0] - T) <= 1e-9 * T


# ---------------------------------------------------------------------------
# Third body
# ---------------------------------------------------------------------------

A_3B, BETA_3B, EA_3B = 2.0e4, -0.8, 1.2e4    # m^6 mol^-2 s^-1 K^-beta, -, J/mol
# efficiencies of A, C, D, bath: replacing 2 A by C + D leaves [M] unchanged (-2 * 1.5 + 2.0 + 1.0 = 0)
EFF_3B = [1.5, 2.0, 1.0, 0.7]


def test_three_body_second_order_decay(oracle):
    m = tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 270.0), (3.5, 0.0, 270.0), (3.5, 0.0, 20.0)],
                  [dict(reac=[0, 0], prod=[1, 2], A=A_3B, beta=BETA_3B, Ea=EA_3B, type=1, eff=EFF_3B)])
    T = 1200.0
    Y0 = np.array([0.3, 0.05, 0.05, 0.6])
    Ct = _conc_total(T)
    M = Ct * (1.5 * 0.3 + 2.0 * 0.05 + 1.0 * 0.05 + 0.7 * 0.6)     # [M] = sum eff_k C_k
    k = A_3B * T ** BETA_3B * np.exp(-EA_3B / (R * T))
    CA0 = Ct * 0.3
    # q = k [M] C_A^2, and A is consumed twice per reaction
    w, q = oracle.rates(m, T, P, Y0)
    assert abs(q[0] - k * M * CA0 ** 2) <= 1e-12 * k * M * CA0 ** 2
    assert abs(w[0] + 2.0 * q[0]) <= 1e-12 * q[0]
    # dC_A/dt = -2 k [M] C_A^2  =>  1/C_A(t) = 1/C_A0 + 2 k [M] t
    dt = 1.0 / (2.0 * k * M * CA0)          # C_A halves
    y, st, _ = oracle.integrate_cell(m, P, dt, np.concatenate([[T], Y0]), **TIGHT)
    assert st == 0
    CA = 1.0 / (1.0 / CA0 + 2.0 * k * M * dt)
    assert abs(CA - 0.5 * CA0) <= 1e-12 * CA0
    assert abs(y[1] - 0.15) <= 1e-9 * 0.15
    # an unweighted [M] (all efficiencies 1) would give a different rate: the pin is sensitive to eff
    assert abs(M - Ct) > 1e-2 * Ct


# ---------------------------------------------------------------------------
# Troe fall-off
# ---------------------------------------------------------------------------

EFF_TROE = [1.3, 1.3, 0.8]      # A, B, bath: A -> B leaves [M] unchanged
# a, T***, T*, T** giving F_cent = 1: (1 - a) exp(-T/T***) with a = 0, T*** = 1e30 -> 1;
#                                      a exp(-T/T*) = 0;  exp(-T**/T) with T** = 1e30 -> 0
TROE_LINDEMANN = [0.0, 1e30, 1.0, 1e30]
# F_cent = 0.5 at every T: (1 - 0.5) exp(-T/1e-30) = 0, 0.5 exp(-T/1e30) = 0.5, exp(-1e30/T) = 0
TROE_HALF = [0.5, 1e-30, 1e30, 1e30]


def _troe_mech(A_inf, beta, Ea, A0, beta0, Ea0, troe):
    return tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 520.0), (3.5, 0.0, 20.0)],
                     [dict(reac=[0], prod=[1], A=A_inf, beta=beta, Ea=Ea, type=2, A0=A0, beta0=beta0, Ea0=Ea0,
                           troe=troe, eff=EFF_TROE)])


def _k_eff(oracle, m, T, p, Y0):
    """The oracle's first-order rate constant of A: q / C_A."""
    w, q = oracle.rates(m, T, p, Y0)
    return q[0] / (_conc_total(T, p) * Y0[0])


Y_TROE = np.array([0.2, 0.1, 0.7])


def _M(T, p):
    return _conc_total(T, p) * (1.3 * 0.2 + 1.3 * 0.1 + 0.8 * 0.7)


@pytest.mark.parametrize("p_atm", [1e-3, 0.1, 1.0, 10.0, 1e3])
def test_troe_lindemann_form(oracle, p_atm):
    # F_cent = 1 makes F = 1: k = k_inf Pr / (1 + Pr), Pr = k0 [M] / k_inf (T and p dependent)
    T, p = 1400.0, p_atm * P
    m = _troe_mech(4.0e9, 0.4, 3.0e4, 6.0e8, -1.2, 1.5e4, TROE_LINDEMANN)
    kinf = 4.0e9 * T ** 0.4 * np.exp(-3.0e4 / (R * T))
    k0 = 6.0e8 * T ** -1.2 * np.exp(-1.5e4 / (R * T))
    Pr = k0 * _M(T, p) / kinf
    ref = kinf * Pr / (1.0 + Pr)
    assert abs(_k_eff(oracle, m, T, p, Y_TROE) - ref) <= 1e-12 * ref


def test_troe_lindemann_limits(oracle):
    # Pr -> 0: k -> k0 [M];  Pr -> inf: k -> k_inf  (F = 1)
    T = 1400.0
    kinf = 4.0e9 * T ** 0.4 * np.exp(-3.0e4 / (R * T))
    low = _troe_mech(4.0e9, 0.4, 3.0e4, 6.0e-2, -1.2, 1.5e4, TROE_LINDEMANN)   # Pr ~ 4e-15
    k0M = 6.0e-2 * T ** -1.2 * np.exp(-1.5e4 / (R * T)) * _M(T, P)
    assert k0M / kinf < 1e-9
    assert abs(_k_eff(oracle, low, T, P, Y_TROE) - k0M) <= 1e-8 * k0M
    high = _troe_mech(4.0e9, 0.4, 3.0e4, 6.0e22, -1.2, 1.5e4, TROE_LINDEMANN)  # Pr ~ 4e9
    assert abs(_k_eff(oracle, high, T, P, Y_TROE) - kinf) <= 1e-8 * kinf


@pytest.mark.parametrize("Pr,k_over_kinf", [
    # F_cent = 0.5, Pr = 10 (worked by hand):
    #   log10 F_cent = -0.3010300;  c = -0.4 + 0.67 * 0.3010300 = -0.1983099
    #   n = 0.75 + 1.27 * 0.3010300 = 1.1323081;  L = log10 Pr + c = 0.8016901
    #   L / (n - 0.14 L) = 0.8016901 / 1.0200715 = 0.7859156;  squared 0.6176633
    #   log10 F = -0.3010300 / 1.6176633 = -0.1860894;  F = 0.6514943
    #   k / k_inf = (10 / 11) * 0.6514943 = 0.5922675
    (10.0, 0.5922675),
    # F_cent = 0.5, Pr = 0.1: L = -1 - 0.1983099 = -1.1983099; n - 0.14 L = 1.3000715;
    #   ratio -0.9217262, squared 0.8495791; log10 F = -0.3010300 / 1.8495791 = -0.1627559;
    #   F = 0.6874547;  k / k_inf = (0.1 / 1.1) * 0.6874547 = 0.0624959
    (0.1, 0.0624959),
])
def test_troe_blending_value(oracle, Pr, k_over_kinf):
    T = 1000.0
    Ainf = 2.0e5
    M = _M(T, P)
    A0 = Pr * Ainf / M            # beta = Ea = 0 on both limits: Pr = A0 [M] / A_inf exactly
    m = _troe_mech(Ainf, 0.0, 0.0, A0, 0.0, 0.0, TROE_HALF)
    k = _k_eff(oracle, m, T, P, Y_TROE)
    assert abs(k / Ainf - k_over_kinf) <= 2e-7
    # the integrated decay of A follows exp(-k t) with that k
    dt = 1.0 / (k_over_kinf * Ainf)
    y, st, _ = oracle.integrate_cell(m, P, dt, np.concatenate([[T], Y_TROE]), **TIGHT)
    assert st == 0
    assert abs(y[1] - 0.2 * np.exp(-1.0)) <= 1e-6 * 0.2 * np.exp(-1.0)


def test_troe_fcent_temperature_dependence(oracle):
    # a = 0.6, T*** = 150 K, T* = 1200 K, T** = 4000 K at T = 1000 K (worked by hand):
    #   F_cent = 0.4 exp(-6.666667) + 0.6 exp(-0.833333) + exp(-4)
    #          = 0.4 * 0.00127263 + 0.6 * 0.43459821 + 0.01831564 = 0.2795836
    #   at Pr = 1: log10 F_cent = -0.5534883; c = -0.4 + 0.67 * 0.5534883 = -0.0291629 = L
    #   n = 0.75 + 1.27 * 0.5534883 = 1.4529301;  L / (n - 0.14 L) = -0.0291629 / 1.4570129 = -0.0200155
    #   log10 F = -0.5534883 / 1.0004006 = -0.5532666;  F = 0.2797263;  k / k_inf = 0.5 F = 0.1398632
    T = 1000.0
    Ainf = 2.0e5
    A0 = 1.0 * Ainf / _M(T, P)
    m = _troe_mech(Ainf, 0.0, 0.0, A0, 0.0, 0.0, [0.6, 150.0, 1200.0, 4000.0])
    assert abs(_k_eff(oracle, m, T, P, Y_TROE) / Ainf - 0.1398632) <= 2e-7
