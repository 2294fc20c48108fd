"""Pins of the oracle's stiff integrator (Sec. 3.1: direct integration of the
reaction ODEs over dt = 1 us; the paper's CPU-DI baseline of Sec. 4.2).

The Rosenbrock solution is checked against: the order of the method observed
on a nonlinear problem with a closed form, L-stability on a very stiff linear
problem, exact conservation of the linear invariants (sum Y, elements), the
adiabatic-isobaric enthalpy invariant, an independent library integrator
(scipy's Radau IIA) on the same right-hand side, and the status codes.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.mechs import tiny_mech

P = synth.P_ATM


def _second_order_mech(k):
    return tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 20.0), (3.5, 0.0, 270.0), (3.5, 0.0, 270.0), (3.5, 0.0, 20.0)],
                     [dict(reac=[0, 1], prod=[2, 3], A=k)])


def test_rodas3_order_three(oracle):
    k = 2.0e5
    m = _second_order_mech(k)
    T = 1000.0
    y0 = np.array([T, 0.3, 0.2, 0.0, 0.0, 0.5])
    dt = 2.0e-6
    rho = P * 0.028 / (synth.R_GAS * T)
    CA0, CB0 = rho * 0.3 / 0.028, rho * 0.2 / 0.028
    D = CB0 - CA0
    exact = D / ((CB0 / CA0) * np.exp(D * k * dt) - 1.0) * 0.028 / rho
    errs = []
    for nsub in (8, 16, 32, 64):
        y = oracle.rodas3_fixed(m, P, dt, nsub, y0)
        errs.append(abs(y[1] - exact))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 3.0) < 0.25), orders


def test_l_stability_very_stiff(oracle):
    # A <=> B with k dt = 1e6: one large step lands on the equilibrium
    m = tiny_mech([(3.5, 0.0, 20.0), (3.5, 0.0, 20.0), (3.5, 0.0, 20.0)], [dict(reac=[0], prod=[1], A=1.0e12)])
    y0 = np.array([900.0, 0.4, 0.0, 0.6])
    y = oracle.rodas3_fixed(m, P, 1.0e-6, 1, y0)
    assert abs(y[1] - 0.2) < 1e-6 and abs(y[2] - 0.2) < 1e-6


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_linear_invariants_and_enthalpy(oracle, name):
    m = synth.get_mech(name)
    n = 6
    if name == "c1":
        T, p, Y = synth.states_dirichlet(m, n, 31)
    else:
        T, p, Y = synth.states_profiles(m, n, 32)
    rtol = 1e-8
    T1, Y1, st, ns = oracle.step_stiff(m, T, p, Y, 1e-6, ncells=n, rtol=rtol, atol_Y=1e-14, atol_T=1e-8)
    assert np.all(st[:n] == 0)
    assert np.abs(Y1[:, :n].sum(axis=0) - Y[:, :n].sum(axis=0)).max() < 1e-13
    el0 = m.elem.T @ (Y[:, :n] / m.W[:, None])
    el1 = m.elem.T @ (Y1[:, :n] / m.W[:, None])
    assert np.abs(el1 - el0).max() <= 1e-13 * np.abs(el0).max()
    cp0, h0, *_ = oracle.props(m, T, p, Y, ncells=n)
    cp1, h1, *_ = oracle.props(m, T1, p, Y1, ncells=n)
    # enthalpy scale: sum_k Y_k |h_k| + cp T (h crosses zero)
    hk = np.array([[oracle.species_thermo(m, k, T[i])[1] * synth.R_GAS * T[i] / m.W[k] for i in range(n)]
                   for k in range(m.N)])
    scale = (Y[:, :n] * np.abs(hk)).sum(axis=0) + cp0[:n] * T[:n]
    assert np.all(np.abs(h1[:n] - h0[:n]) <= 100 * rtol * scale)


def test_agrees_with_scipy_radau(oracle):
    scipy_integrate = pytest.importorskip("scipy.integrate")
    m = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m, 3, 41)
    dt = 1.0e-6
    for i in range(3):
        y0 = np.concatenate([[T[i]], Y[:, i]])
        y, st, _ = oracle.integrate_cell(m, P, dt, y0, rtol=1e-10, atol_Y=1e-16, atol_T=1e-9)
        sol = scipy_integrate.solve_ivp(lambda t, v: oracle.rhs(m, P, v), (0.0, dt), y0, method="Radau",
                                        jac=lambda t, v: oracle.jac(m, P, v), rtol=1e-11, atol=1e-16)
        assert sol.success and st == 0
        yr = sol.y[:, -1]
        assert abs(y[0] - yr[0]) <= 1e-6 * yr[0]
        assert np.all(np.abs(y[1:] - yr[1:]) <= 1e-6 * np.abs(yr[1:]) + 1e-12)


def test_status_codes(oracle):
    m = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m, 2, 51)
    y0 = np.concatenate([[T[0]], Y[:, 0]])
    _, st, ns = oracle.integrate_cell(m, P, 1e-6, y0, max_steps=1)
    assert st == 2 and ns == 1
    bad = y0.copy()
    bad[0] = np.nan
    _, st, _ = oracle.integrate_cell(m, P, 1e-6, bad)
    assert st == 4
