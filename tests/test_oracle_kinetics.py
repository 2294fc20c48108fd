"""Pins of the oracle's kinetics and reactor right-hand side (Sec. 3.1: the
reaction ODEs integrated over dt = 1 us).

Closed forms of first- and second-order reactions, equilibrium reached by long
integration (zero affinity computed from chemical potentials), conservation of
mass and elements by the source terms, and the analytic Jacobian against
central finite differences of the right-hand side.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.mechs import tiny_mech

P = synth.P_ATM
TIGHT = dict(rtol=1e-11, atol_Y=1e-16, atol_T=1e-10)


def _first_order(reversible: bool, k: float):
    # A -> B (irreversible through a huge entropy gain: Kc = e^500) or A <=> B (Kc = 1)
    sB = 20.0 if reversible else 520.0
    return tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, sB), (3.5, 0.0, 20.0)],
                     [dict(reac=[0], prod=[1], A=k)])


def test_first_order_irreversible_closed_form(oracle):
    k = 1.0e6
    m = _first_order(False, k)
    y0 = np.array([1000.0, 0.3, 0.1, 0.6])
    dt = 1.0e-6
    y, st, _ = oracle.integrate_cell(m, P, dt, y0, **TIGHT)
    assert st == 0
    assert abs(y[1] - 0.3 * np.exp(-k * dt)) <= 1e-9 * 0.3 * np.exp(-k * dt)
    assert abs(y[2] - (0.4 - y[1])) <= 1e-14
    assert abs(y[0] - 1000.0) <= 1e-9


def test_first_order_reversible_closed_form(oracle):
    k = 2.0e6
    m = _first_order(True, k)
    y0 = np.array([800.0, 0.35, 0.05, 0.6])
    dt = 1.0e-6
    y, st, _ = oracle.integrate_cell(m, P, dt, y0, **TIGHT)
    s = 0.4
    ref = s / 2 + (0.35 - s / 2) * np.exp(-2 * k * dt)
    assert st == 0
    assert abs(y[1] - ref) <= 1e-9 * ref


def test_second_order_closed_form(oracle):
    # A + B -> C + D, equal W and cp, no heat release: T and rho stay constant
    m = tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 20.0), (3.5, 0.0, 270.0), (3.5, 0.0, 270.0), (3.5, 0.0, 20.0)],
                  [dict(reac=[0, 1], prod=[2, 3], A=2.0e5)])
    T = 1000.0
    y0 = np.array([T, 0.3, 0.2, 0.0, 0.0, 0.5])
    dt = 1.0e-6
    y, st, _ = oracle.integrate_cell(m, P, dt, y0, **TIGHT)
    rho = P * 0.028 / (synth.R_GAS * T)
    CA0, CB0 = rho * 0.3 / 0.028, rho * 0.2 / 0.028
    D = CB0 - CA0
    CA = D / ((CB0 / CA0) * np.exp(D * 2.0e5 * dt) - 1.0)
    assert st == 0
    assert abs(y[1] - CA * 0.028 / rho) <= 1e-9 * y[1]


def _mu_RT(oracle, m, T, p, Y, k):
    cpR, H_RT, S_R, _ = oracle.species_thermo(m, k, T)
    X = (Y / m.W) / (Y / m.W).sum()
    return H_RT - S_R + np.log(X[k] * p / synth.P_STD)


def test_equilibrium_zero_affinity(oracle):
    # long integration reaches equilibrium: every reaction has zero affinity
    # sum_k nu_kj mu_k = 0 with mu_k = H_k - T S_k + RT ln(X_k p / P_std)
    m = synth.mech_c1()
    T0, p0, Y0 = synth.states_dirichlet(m, 4, 77)
    nr, npd = m.nu()
    nu = npd - nr
    for i in range(2):
        y0 = np.concatenate([[T0[i]], Y0[:, i]])
        y, st, _ = oracle.integrate_cell(m, P, 1.0, y0, rtol=1e-10, atol_Y=1e-20, atol_T=1e-10, max_steps=200000)
        assert st == 0
        T, Y = y[0], y[1:]
        mus = np.array([_mu_RT(oracle, m, T, P, Y, k) for k in range(m.N)])
        aff = nu @ mus
        assert np.all(np.abs(aff) < 1e-5), aff
        w, q = oracle.rates(m, T, P, Y)
        kf, kr = oracle.rate_constants(m, T, P, Y)
        # net rates vanish against the one-way rates
        C = (P / (synth.R_GAS * T)) * (Y / m.W) / (Y / m.W).sum()
        fwd = kf * np.prod(np.where(nr > 0, C[None, :] ** nr, 1.0), axis=1)
        assert np.all(np.abs(q) <= 1e-5 * fwd + 1e-300)


@pytest.mark.parametrize("name", ["c1", "c2", "c5"])
def test_source_terms_conserve_mass_and_elements(oracle, name):
    m = synth.get_mech(name)
    T, p, Y = synth.states_dirichlet(m, 8, 11)
    for i in range(8):
        w, q = oracle.rates(m, T[i], p[i], Y[:, i])
        scale_m = np.sum(np.abs(m.W * w))
        assert abs(np.sum(m.W * w)) <= 1e-13 * scale_m
        for e in range(m.elem.shape[1]):
            scale = np.sum(np.abs(m.elem[:, e] * w)) + 1e-300
            assert abs(np.sum(m.elem[:, e] * w)) <= 1e-12 * scale


def _fd_jac(oracle, m, p, y):
    n = y.size
    J = np.zeros((n, n))
    for b in range(n):
        h = 1e-6 * (abs(y[b]) if b == 0 else max(abs(y[b]), 1e-4))
        yp = y.copy(); ym = y.copy()
        yp[b] += h; ym[b] -= h
        J[:, b] = (oracle.rhs(m, p, yp) - oracle.rhs(m, p, ym)) / (2 * h)
    return J


def _troe_mech():
    # A + B (+M) <=> C (+M) with Troe fall-off, plus a three-body and an elementary reaction
    return tiny_mech([(3.5, 100e3, 20.0), (4.0, 50e3, 22.0), (5.0, -200e3, 25.0), (3.0, 0.0, 18.0), (3.5, 0.0, 20.0)],
                     [dict(reac=[0, 1], prod=[2], A=3.0e7, beta=0.4, Ea=2.0e4, type=2, A0=5.0e9, beta0=-0.9,
                           Ea0=1.0e4, troe=[0.6, 150.0, 1200.0, 4000.0], eff=[1.0, 2.0, 0.7, 1.5, 1.0]),
                      dict(reac=[0, 0], prod=[3], A=1.0e6, beta=-0.5, type=1, eff=[1.2, 1.0, 2.5, 0.5, 1.0]),
                      dict(reac=[1, 3], prod=[0, 2], A=4.0e6, beta=1.1, Ea=3.0e4)],
                     W=[0.020, 0.030, 0.050, 0.040, 0.028])


@pytest.mark.parametrize("which", ["c1", "c2", "troe"])
def test_analytic_jacobian_matches_fd(oracle, which):
    m = _troe_mech() if which == "troe" else synth.get_mech(which)
    if which == "troe":
        states = [np.array([T, 0.2, 0.15, 0.1, 0.05, 0.5]) for T in (600.0, 1300.0, 2100.0)]
    else:
        T, p, Y = synth.states_dirichlet(m, 3, 21)
        states = [np.concatenate([[T[i]], Y[:, i]]) for i in range(3)]
    for y in states:
        J = oracle.jac(m, P, y)
        Jfd = _fd_jac(oracle, m, P, y)
        rowscale = np.abs(J).max(axis=1, keepdims=True)
        err = np.abs(J - Jfd) / (rowscale + 1e-300)
        assert err.max() < 1e-6, err.max()
