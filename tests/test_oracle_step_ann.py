"""Pins of the oracle's learned step (oracle/ann.py::step_ann, Sec. 3.2): what the
network's output u becomes in the state, with the network itself taken out.

A network whose weights are all zero outputs its last bias b for every cell (GELU(0) = 0
in the hidden layers), so u is known exactly. With constant-cp species (the NASA-7 rows
hold a1 and a6 only, a1 = c for every species) the mixture enthalpy is linear in T,
    h / R = sum_k Y_k (c T + a6_k) / W_k,
and the T that keeps h at its value before the step has a closed form:
    T' = [sum_k Y_k (c T + a6_k) / W_k - sum_k Y'_k a6_k / W_k] / (c sum_k Y'_k / W_k).
Unequal molar masses make the mixture cp depend on the new composition. The closed form
catches an enthalpy target taken at the new composition (T would not move) and a reversed
update (no convergence); the slope of the iteration only sets its speed. Checked:
* zero output: the state is unchanged;
* de-normalisation dY = u sd_u + mu_u, bath closure (the bath takes -sum dY), sum Y' = 1;
* a clamped species: max(., 0) then renormalisation, values worked by hand;
* T' against the closed form above.
"""
import numpy as np

from tests.mechs import tiny_mech

C_R = 3.5                                  # cp / R of every species (molar)
HF = [-1.1e5, 2.0e5, -3.9e5, 0.0]          # J/mol at 298.15 K; the last species is the bath
W = [0.016, 0.032, 0.044, 0.028]           # kg/mol


def _mech():
    return tiny_mech([(C_R, h, 20.0) for h in HF], [], W=W, name="step_ann_pins")


def _zero_net(mech, b_out, hidden=(8, 8, 8)):
    widths = [mech.N + 2, *hidden, mech.N - 1]
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(widths[:-1], widths[1:])]
    layers[-1] = (layers[-1][0], np.asarray(b_out, np.float64))
    return layers


def _stats(mech, sd_u, mu_u):
    return (np.zeros(mech.N + 2), np.ones(mech.N + 2), np.asarray(mu_u, np.float64), np.asarray(sd_u, np.float64))


def _state(n=3):
    Y = np.array([[0.10, 0.05, 0.20],
                  [0.20, 0.15, 0.05],
                  [0.05, 0.30, 0.10],
                  [0.65, 0.50, 0.65]])[:, :n]
    T = np.array([900.0, 1500.0, 2100.0])[:n]
    p = np.full(n, 101325.0)
    return T, p, Y


def _T_closed_form(mech, T, Y, Y1):
    a6 = mech.nasa_lo[:, 5][:, None]
    Wk = np.asarray(mech.W)[:, None]
    h0 = np.sum(Y * (C_R * T + a6) / Wk, axis=0)
    return (h0 - np.sum(Y1 * a6 / Wk, axis=0)) / (C_R * np.sum(Y1 / Wk, axis=0))


def test_zero_output_keeps_the_state(oracle):
    from oracle import ann as A
    mech = _mech()
    T, p, Y = _state()
    T1, Y1 = A.step_ann(mech, _zero_net(mech, np.zeros(3)), _stats(mech, np.ones(3), np.zeros(3)), T, p, Y)
    assert np.allclose(Y1, Y, rtol=0, atol=1e-15)
    assert np.allclose(T1, T, rtol=1e-12, atol=0)


def test_denormalised_output_closure_and_energy(oracle):
    from oracle import ann as A
    mech = _mech()
    T, p, Y = _state()
    b = np.array([1.0, -0.5, 2.0])                  # u for every cell
    sd_u = np.array([2e-3, 4e-3, 1e-3])
    mu_u = np.array([1e-3, 0.0, -5e-4])
    dY = b * sd_u + mu_u                             # (3e-3, -2e-3, 1.5e-3): no species leaves [0, 1]
    T1, Y1 = A.step_ann(mech, _zero_net(mech, b), _stats(mech, sd_u, mu_u), T, p, Y)
    expect = Y.copy()
    expect[:3] += dY[:, None]
    expect[3] -= dY.sum()
    assert np.allclose(Y1, expect, rtol=0, atol=1e-15)
    assert np.allclose(Y1.sum(axis=0), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(T1, _T_closed_form(mech, T, Y, Y1), rtol=1e-11, atol=0)
    # the step moved enthalpy between species, so T did move
    assert np.all(np.abs(T1 - T) > 1.0)


def test_clamped_species_and_renormalisation(oracle):
    from oracle import ann as A
    mech = _mech()
    T, p, Y = _state(1)                              # Y = (0.10, 0.20, 0.05, 0.65)
    b = np.array([-0.15, 0.05, 0.0])
    T1, Y1 = A.step_ann(mech, _zero_net(mech, b), _stats(mech, np.ones(3), np.zeros(3)), T, p, Y)
    # by hand: species 0 -> 0.10 - 0.15 < 0 -> 0; species 1 -> 0.25; species 2 -> 0.05;
    # bath 0.65 + 0.10 = 0.75; the sum 1.05 rescales all four
    expect = np.array([0.0, 0.25, 0.05, 0.75]) / 1.05
    assert np.allclose(Y1[:, 0], expect, rtol=0, atol=1e-15)
    assert np.allclose(T1, _T_closed_form(mech, T, Y, Y1), rtol=1e-11, atol=0)
