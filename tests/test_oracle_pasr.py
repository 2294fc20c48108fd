"""Pins of the oracle's PaSR scaling (Sec. 4.1: kappa = tau_c / (tau_c + tau_mix), tau_c
from the slowest species formation rate, tau_mix the geometric mean of the Taylor and
Kolmogorov time scales).

* A -> B, first order with rate constant k, equal molar masses, no heat release: the
  species times are 1/k for A and Y_B / (k Y_A) for B in closed form, and the inert bath
  species has no time; tau_c is the larger of the two. y_min removes species below it, and
  a cell with no qualifying species has tau_c = inf and kappa = 1.
* On the 30-species mechanism the rates behind tau_c agree with the rate of change of the
  integrated reactor itself (Richardson-extrapolated forward differences of the oracle's
  stiff integrator over 1e-13 s), an independent route to dY_k/dt, to 1e-5 plus the
  differences' rounding (which grows with the species time).
* kappa = 1 (tau_mix = 0) gives back the chemistry step; tau_mix = tau_c halves it.
"""
import numpy as np

from oracle import pasr as P
from paper_2312_05800_gb300 import synth
from tests.mechs import tiny_mech


def _a_to_b(k):
    # irreversible through a large entropy gain of B (K_c = e^500), constant cp, no heat of reaction
    return tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 520.0), (3.5, 0.0, 20.0)], [dict(reac=[0], prod=[1], A=k)])


def test_species_times_closed_form(oracle):
    k = 3.0e5
    m = _a_to_b(k)
    T = np.array([900.0, 1200.0, 1500.0])
    p = np.full(3, synth.P_ATM)
    Y = np.array([[0.3, 0.02, 0.5], [0.1, 0.4, 1e-9], [0.6, 0.58, 0.5 - 1e-9]])
    tc = P.chemical_time(m, T, p, Y, y_min=1e-12)
    ref = np.maximum(1.0 / k, Y[1] / (k * Y[0]))
    assert np.allclose(tc, ref, rtol=1e-12, atol=0)
    # y_min above Y_B: only A counts
    tc2 = P.chemical_time(m, T, p, Y, y_min=0.5)
    assert np.isinf(tc2[0]) and np.isinf(tc2[1])          # Y_A < 0.5 and Y_B < 0.5: none qualifies
    assert np.isclose(tc2[2], 1.0 / k, rtol=1e-12)        # Y_A = 0.5 >= y_min qualifies
    assert np.all(P.kappa(tc2[:2], [1e-3, 1e-3], [1e-5, 1e-5]) == 1.0)


def test_rates_agree_with_the_integrated_reactor(oracle):
    import oracle as O
    m = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(m, 24, 2051)
    eps = 1e-13
    opts = dict(rtol=1e-12, atol_Y=1e-20, atol_T=1e-12, h0=eps, max_steps=100)
    T1, Y1, st1, _ = O.step_stiff(m, T.copy(), p, Y.copy(), eps, **opts)
    T2, Y2, st2, _ = O.step_stiff(m, T.copy(), p, Y.copy(), eps / 2, **dict(opts, h0=eps / 2))
    assert np.all(st1 == 0) and np.all(st2 == 0)
    rate = 2.0 * (Y2 - Y) / (eps / 2) - (Y1 - Y) / eps        # Richardson: O(eps^2)
    y_min = 1e-6
    fd = np.empty(24)
    for i in range(24):
        r = np.abs(rate[:, i])
        ok = (Y[:, i] >= y_min) & (r > 0)
        fd[i] = (Y[ok, i] / r[ok]).max()
    tc = P.chemical_time(m, T, p, Y, y_min)
    # the differences of rounded Y carry 2 ulp(Y) each, three of them in the Richardson
    # combination: a relative error of about 3 x 4.4e-16 tau / eps in a species time
    tol = 1e-5 + 3 * 4.4e-16 * tc / eps
    assert np.all(np.abs(tc / fd - 1) <= tol), (np.abs(tc / fd - 1) / tol).max()
    assert np.mean(tol < 1e-4) > 0.5            # most cells are tested tightly


def test_kappa_limits():
    rng = np.random.default_rng(4)
    T0, T1 = rng.uniform(500, 2000, 50), rng.uniform(500, 2000, 50)
    Y0, Y1 = rng.uniform(0, 1, (7, 50)), rng.uniform(0, 1, (7, 50))
    tc = 10.0 ** rng.uniform(-8, -3, 50)
    k1 = P.kappa(tc, np.zeros(50), np.ones(50))
    assert np.all(k1 == 1.0)
    Ta, Ya = P.apply(T0, Y0, T1, Y1, k1)
    assert np.allclose(Ta, T1, rtol=1e-15) and np.allclose(Ya, Y1, rtol=0, atol=1e-15)
    kh = P.kappa(tc, tc, tc)                                  # sqrt(tc tc) = tc
    assert np.allclose(kh, 0.5, rtol=1e-15)
    Th, Yh = P.apply(T0, Y0, T1, Y1, kh)
    assert np.allclose(Th, 0.5 * (T0 + T1), rtol=1e-14) and np.allclose(Yh, 0.5 * (Y0 + Y1), atol=1e-15)
