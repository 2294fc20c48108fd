"""Pins of the oracle's random training-data generation (Sec. 3.1, Eq. 1-4 and Table 1).

* With every c = 0, Eq. 1-4 and the renormalisation return the base state (mass fractions
  that sum to 1 are a fixed point); for any c the result sums to 1 and Y'_N2 is the Eq. 3
  value; c = +-1 reaches the stated extremes of T' (alpha of the dataset's T range).
* Element ratios from their definition: the pure fuel has H/C = 4, air has O/N = 2/(2 x 3.76),
  a stoichiometric fuel-air mixture has phi = 1 and air phi = 0, complete combustion keeps phi
  (elements are conserved), and so does any blend of a mixture with its products.
* Table 1 keeps fuel-air states built at phi inside [0.20, 1.15] and removes those outside; extra
  H2 raises H/C and extra CO lowers it.
* The lean-mixing endpoint: the adiabatic equilibrium of the phi = 0.45 mixture conserves the
  elements and the enthalpy of the unburnt mixture, and its net rates vanish; the blend with
  air reaches both endpoints and is linear in the element moles.
"""
import numpy as np
import pytest

from oracle import hfrd as H
from paper_2312_05800_gb300 import synth


def _base(n=500, seed=2071):
    m = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(m, n, seed, ld=n)
    return m, T, p, Y


def test_zero_draws_return_the_base_state():
    m, T, p, Y = _base()
    Y = Y / Y.sum(axis=0, keepdims=True)
    r = H.dataset_ranges(m, T, p, Y)
    T2, p2, Y2, ok = H.perturb(m, T, p, Y, np.zeros((3 + m.N, len(T))), r)
    assert ok.all()
    assert np.array_equal(T2, T) and np.array_equal(p2, p)
    assert np.allclose(Y2, Y, rtol=1e-14, atol=1e-300)


def test_random_draws_sum_to_one_and_reach_the_stated_extremes():
    m, T, p, Y = _base()
    r = H.dataset_ranges(m, T, p, Y)
    rng = np.random.default_rng(5)
    c = rng.uniform(-1.0, 1.0, (3 + m.N, len(T)))
    c[0, :2] = (1.0, -1.0)
    T2, p2, Y2, ok = H.perturb(m, T, p, Y, c, r)
    assert ok.mean() > 0.99
    assert np.allclose(Y2[:, ok].sum(axis=0), 1.0, rtol=0, atol=1e-14)
    yb = Y[m.bath] + H.ALPHA * c[2] * (r[5] - r[4])
    assert np.array_equal(Y2[m.bath, ok], yb[ok])
    dT = T2 - T
    assert np.isclose(dT[0], H.ALPHA * (r[1] - r[0]), rtol=1e-15) and np.isclose(dT[1], -H.ALPHA * (r[1] - r[0]))
    assert np.all(np.abs(dT) <= H.ALPHA * (r[1] - r[0]) * (1 + 1e-15))
    assert np.array_equal(p2, p)              # the base states share one pressure: p_max - p_min = 0


def test_element_ratios_from_their_definition():
    m = synth.get_mech("c2")
    r = m.roles
    Yf = np.zeros((m.N, 1))
    Yf[r["fuel"]] = 1.0
    assert np.isclose(H.ratios(m, Yf)[0][0], 4.0, rtol=1e-14)
    Ta, Ya = H.air(m)
    hc, on, phi = H.ratios(m, Ya[:, None])
    assert np.isclose(on[0], 2.0 / (2.0 * 3.76), rtol=1e-14) and phi[0] == 0.0
    for phi0 in (0.45, 1.0, 1.15):
        Yu, Yb = H.premixed(m, phi0)
        assert np.isclose(H.ratios(m, Yu[:, None])[2][0], phi0, rtol=1e-13)
        assert np.isclose(H.ratios(m, Yb[:, None])[2][0], phi0, rtol=1e-13)
    # any blend of a mixture with its own products keeps its phi (elements are conserved)
    Yu, Yb = H.premixed(m, 0.8)
    _, Ym = H.blend(np.linspace(0.0, 1.0, 11), 300.0, Yu, 2000.0, Yb)
    assert np.allclose(H.ratios(m, Ym)[2], 0.8, rtol=1e-13)


def _premixed_states(m, phis, seed):
    """Fuel-air mixtures at the given phi, each blended with its products at a seeded progress."""
    rng = np.random.default_rng(seed)
    cols = []
    for phi in phis:
        Yu, Yb = H.premixed(m, phi)
        c = rng.uniform()
        cols.append((1.0 - c) * Yu + c * Yb)
    return np.stack(cols, axis=1)


def test_table_1_keeps_and_removes_by_phi():
    m = synth.get_mech("c2")
    rng = np.random.default_rng(2073)
    inside = _premixed_states(m, rng.uniform(0.21, 1.14, 100), 2074)
    outside = _premixed_states(m, np.concatenate([rng.uniform(0.05, 0.19, 50), rng.uniform(1.16, 2.0, 50)]), 2075)
    assert H.accept(m, inside).all()
    assert not H.accept(m, outside).any()
    # H/C outside its bounds: hydrogen-rich (H2 added) and carbon-rich (CO added) mixtures
    Yh = inside.copy()
    Yh[m.roles["h2"]] += 0.05
    Yc = inside.copy()
    Yc[m.roles["co"]] += 0.2
    hc_h, hc_c = H.ratios(m, Yh)[0], H.ratios(m, Yc)[0]
    assert np.array_equal(H.accept(m, Yh), (hc_h <= H.HC_RANGE[1]) & (H.ratios(m, Yh)[2] <= H.PHI_RANGE[1]))
    assert np.all(hc_h > 4.0) and np.all(hc_c < 4.0)


def test_lean_equilibrium_and_air_blend(oracle):
    import oracle as O
    m = synth.get_mech("c2")
    Te, Ye = H.adiabatic_equilibrium(m, 0.45)
    Yu, _ = H.premixed(m, 0.45)
    assert np.allclose(H.element_moles(m, Ye[:, None])[:, 0], H.element_moles(m, Yu[:, None])[:, 0], rtol=1e-10)
    pa = np.array([synth.P_ATM])
    h_eq = O.props(m, np.array([Te]), pa, Ye[:, None])[1][0]
    h_u = O.props(m, np.array([300.0]), pa, Yu[:, None])[1][0]
    assert abs(h_eq - h_u) <= 1e-8 * abs(h_u) + 1e-6
    f = O.rhs(m, synth.P_ATM, np.concatenate([[Te], Ye]))
    assert np.abs(f[1:]).max() < 1e-3 and abs(f[0]) < 1e-2       # at rest (per second)
    Ta, Ya = H.air(m)
    s = np.array([0.0, 0.25, 0.5, 1.0])
    Tb, Yb = H.blend(s, Ta, Ya, Te, Ye)
    assert Tb[0] == Ta and Tb[-1] == Te and np.array_equal(Yb[:, 0], Ya) and np.allclose(Yb[:, -1], Ye, rtol=1e-15)
    ne = H.element_moles(m, Yb)
    assert np.allclose(ne[:, 1], 0.75 * ne[:, 0] + 0.25 * ne[:, 3], rtol=1e-12)
