"""Pins of the oracle's mixture-averaged transport (Sec. 2: transport
properties per cell; Sec. 3.1 names the Hirschfelder-Curtiss model).

Wilke's mixing rule reduces to the pure-species value; two species with equal
W and viscosity mix to that viscosity; the off-diagonal Wilke weights, recovered
from binary-mixture viscosities, obey Wilke's reciprocity and reproduce the
conductivity, which mixes with the same weights; the binary mixture-averaged diffusion
coefficient has a closed form in the binary coefficient; D scales as 1/p while
mu and lambda do not depend on p; a monatomic gas has the kinetic-theory conductivity
(15/4) mu R / W; and the fitted species values stay within the
fit residual of the raw Chapman-Enskog expressions the fits were made from.
"""
import numpy as np

from paper_2312_05800_gb300 import synth
from tests.mechs import tiny_mech

P = synth.P_ATM


def _polyval(c, x):
    return np.polynomial.polynomial.polyval(x, c)


def test_pure_species_limits(oracle):
    m = synth.mech_c2()
    N = m.N
    Ts = np.array([300.0, 800.0, 1500.0, 2600.0])
    for k in (0, 5, 13, 29):
        Y = np.zeros((N, 4))
        Y[k] = 1.0
        cp, h, mu, lam, Dk = oracle.props(m, Ts, np.full(4, P), Y)
        for i, T in enumerate(Ts):
            muk = np.exp(_polyval(m.visc_fit[k], np.log(T / 1000.0)))
            cpR = oracle.species_thermo(m, k, T)[0]
            assert abs(mu[i] - muk) <= 1e-13 * muk
            assert abs(lam[i] - muk * (cpR + 1.25) * synth.R_GAS / m.W[k]) <= 1e-12 * lam[i]


def test_monatomic_conductivity_is_the_kinetic_theory_value(oracle):
    # For a monatomic gas (cp = 5R/2 per mole) the first Chapman-Enskog approximation gives
    # lambda = (15/4) mu R / W, a textbook result independent of the Eucken form the oracle
    # uses for every species; the two coincide here.
    vis = np.array([-10.7, 0.7, -0.03, 0.002, 0.0])
    m = tiny_mech([(2.5, 0.0, 18.0), (2.5, 0.0, 18.0)], [dict(reac=[0], prod=[1], A=1.0)], W=[0.040, 0.040])
    m.visc_fit = np.stack([vis, vis])
    Ts = np.array([300.0, 1200.0, 2500.0])
    Y = np.array([[1.0, 0.4, 0.0], [0.0, 0.6, 1.0]])
    cp, h, mu, lam, Dk = oracle.props(m, Ts, np.full(3, P), Y)
    assert np.allclose(lam, 3.75 * mu * synth.R_GAS / 0.040, rtol=1e-13, atol=0)


def test_equal_species_mix_to_same_viscosity(oracle):
    vis = np.array([-10.9, 0.65, -0.02, 0.003, 0.0])
    m = tiny_mech([(3.5, 0.0, 20.0), (4.5, 0.0, 22.0), (3.5, 0.0, 20.0)], [dict(reac=[0], prod=[1], A=1.0)])
    m.visc_fit = np.stack([vis, vis, vis + 0.3])
    Y = np.array([[0.3, 0.7], [0.7, 0.3], [0.0, 0.0]])
    cp, h, mu, lam, Dk = oracle.props(m, np.array([900.0, 1700.0]), np.full(2, P), Y)
    for i, T in enumerate((900.0, 1700.0)):
        ref = np.exp(_polyval(vis, np.log(T / 1000.0)))
        assert abs(mu[i] - ref) <= 1e-13 * ref


def test_binary_diffusion_closed_form(oracle):
    m = tiny_mech([(3.5, 0.0, 20.0), (4.0, 0.0, 22.0)], [dict(reac=[0], prod=[1], A=1.0)], W=[0.004, 0.032])
    g = np.zeros((2, 2, 5))
    g[0, 1] = g[1, 0] = [3.1e4, 2.0e3, 150.0, -20.0, 3.0]
    m.diff_fit = g
    Y1 = np.array([0.1, 0.5, 0.9])
    Y = np.stack([Y1, 1 - Y1])
    T = np.array([500.0, 1200.0, 2400.0])
    p = np.array([P, 2 * P, 0.5 * P])
    cp, h, mu, lam, Dk = oracle.props(m, T, p, Y)
    X1 = (Y1 / 0.004) / (Y1 / 0.004 + (1 - Y1) / 0.032)
    D12 = T ** 1.5 / (p * _polyval(g[0, 1], np.log(T / 1000.0)))
    assert np.allclose(Dk[0], D12 * (1 - Y1) / (1 - X1), rtol=1e-13, atol=0)
    assert np.allclose(Dk[1], D12 * Y1 / X1, rtol=1e-13, atol=0)


def test_pressure_scaling(oracle):
    m = synth.mech_c2()
    T, p, Y = synth.states_profiles(m, 16, 7)
    a = oracle.props(m, T, p, Y)
    b = oracle.props(m, T, 2 * p, Y)
    assert np.allclose(b[4][:, :16], 0.5 * a[4][:, :16], rtol=1e-14, atol=0)
    for i in range(4):
        assert np.allclose(b[i][:16], a[i][:16], rtol=1e-14, atol=0)


def test_fits_follow_chapman_enskog(oracle):
    # fitted species viscosity and binary diffusivity vs the raw kinetic-theory formulas
    m = synth.mech_c2()
    Ts = np.array([300.0, 1000.0, 3000.0])
    mk = m.W / synth.N_AVO
    for k in (1, 7, 20):
        sig = m.sigma[k] * 1e-10
        raw = (5 / 16) * np.sqrt(np.pi * mk[k] * synth.K_BOLTZ * Ts) / (
            np.pi * sig ** 2 * synth._omega22(Ts / m.eps_k[k]))
        Y = np.zeros((m.N, 3))
        Y[k] = 1.0
        mu = oracle.props(m, Ts, np.full(3, P), Y)[2]
        assert np.all(np.abs(mu - raw) <= 0.02 * raw)
    j, k = 3, 11
    sjk = 0.5 * (m.sigma[j] + m.sigma[k]) * 1e-10
    ejk = np.sqrt(m.eps_k[j] * m.eps_k[k])
    mjk = mk[j] * mk[k] / (mk[j] + mk[k])
    Draw = (3 / 16) * np.sqrt(2 * np.pi * (synth.K_BOLTZ * Ts) ** 3 / mjk) / (
        P * np.pi * sjk ** 2 * synth._omega11(Ts / ejk))
    Dfit = Ts ** 1.5 / (P * _polyval(m.diff_fit[j, k], np.log(Ts / 1000.0)))
    assert np.all(np.abs(Dfit - Draw) <= 0.02 * Draw)


def test_wilke_off_diagonal_weights(oracle):
    # For a binary mixture, mu = X1 mu1 / (X1 + X2 P12) + X2 mu2 / (X1 P21 + X2) with the two
    # off-diagonal Wilke weights P12, P21. Recovered from the oracle's mixture viscosity at two
    # compositions (and checked at a third), they must satisfy Wilke's reciprocity
    # P21 / P12 = (mu2 / mu1) (W1 / W2), a property of the weights, not their formula; the
    # conductivity, which mixes with the same weights, must give the same pair.
    from scipy.optimize import fsolve
    m = tiny_mech([(3.5, 0.0, 20.0), (4.0, 0.0, 22.0)], [dict(reac=[0], prod=[1], A=1.0)], W=[0.004, 0.032])
    m.visc_fit = np.array([[-11.3, 0.7, 0.0, 0.0, 0.0], [-10.4, 0.62, 0.01, 0.0, 0.0]])
    T = 1300.0
    Y1 = np.array([1.0, 0.0, 0.2, 0.55, 0.85])
    Y = np.stack([Y1, 1 - Y1])
    cp, h, mu, lam, Dk = oracle.props(m, np.full(5, T), np.full(5, P), Y)
    X1 = (Y1 / 0.004) / (Y1 / 0.004 + (1 - Y1) / 0.032)
    X2 = 1 - X1
    mix = lambda prop, phi, i: (X1[i] * prop[0] / (X1[i] + X2[i] * phi[0]) +
                                X2[i] * prop[1] / (X1[i] * phi[1] + X2[i]))   # prop[0], prop[1]: pure values
    phi = fsolve(lambda f: [mix(mu, f, 2) - mu[2], mix(mu, f, 3) - mu[3]], [1.0, 1.0], xtol=1e-14)
    assert abs(mix(mu, phi, 4) - mu[4]) <= 1e-10 * mu[4]
    assert abs(phi[1] / phi[0] - (mu[1] / mu[0]) * (0.004 / 0.032)) <= 1e-8 * phi[1] / phi[0]
    for i in (2, 3, 4):
        assert abs(mix(lam, phi, i) - lam[i]) <= 1e-10 * lam[i]
