"""FP64 oracle of the random training-data generation of Sec. 3.1 (TEST INFRASTRUCTURE ONLY).

Each base composition (T, p, Y) of the dataset (flamelet states in the paper; seeded
profile states here) yields a random composition by Eq. 1-4, with uniform random numbers
c in [-1, 1] passed in as inputs:
  T'     = T + alpha c_T (T_max - T_min)                 (Eq. 1)
  p'     = p + beta c_p (p_max - p_min)                  (Eq. 2)
  Y'_N2  = Y_N2 + alpha c_N2 (Y_N2,max - Y_N2,min)       (Eq. 3)
  Y'_j   = Y_j ^ (1 + gamma c_j) for every other species (Eq. 4)
alpha = 0.125, beta = 10, gamma = 0.1; max and min are over the base dataset. The species
other than N2 are then scaled to sum to 1 - Y'_N2. A state is kept when its molar element
ratios and equivalence ratio lie within Table 1: H/C in [2.65, 4.67], O/N in [0.254, 0.32],
phi in [0.20, 1.15], with phi = (2 n_C + n_H / 2) / n_O from the element moles n_e.
The lean-mixing states are linear blends, for all species and T, between the adiabatic
equilibrium of the leanest mixture (phi = 0.45) and ambient air.

Readings (the paper is silent on them): an independent c for each equation and for each
species; N2 is the bath species; a state whose Y'_N2 leaves [0, 1), whose T' or p' is not
positive, or whose other species all vanish is rejected; the 500 K threshold applies to the
base states (the paper sets it while collecting flamelet data). Plain loops and numpy.
"""
from __future__ import annotations

import numpy as np

ALPHA, BETA, GAMMA = 0.125, 10.0, 0.1
HC_RANGE = (2.65, 4.67)
ON_RANGE = (0.254, 0.32)
PHI_RANGE = (0.20, 1.15)


def dataset_ranges(mech, T, p, Y, t_min: float = 0.0):
    """(T_min, T_max, p_min, p_max, N2_min, N2_max) over the base states with T >= t_min."""
    keep = np.asarray(T) >= t_min
    b = mech.bath
    return (float(T[keep].min()), float(T[keep].max()), float(p[keep].min()), float(p[keep].max()),
            float(Y[b, keep].min()), float(Y[b, keep].max()))


def perturb(mech, T, p, Y, c, ranges):
    """Eq. 1-4 and the renormalisation. c: [3 + N, n] uniform numbers, rows c_T, c_p, c_N2,
    then c_j for species j (the bath row unused). Returns (T', p', Y', ok) where ok marks
    the states whose values are admissible (before the Table 1 test)."""
    Tmin, Tmax, pmin, pmax, nmin, nmax = ranges
    b = mech.bath
    n = len(T)
    T2 = np.empty(n)
    p2 = np.empty(n)
    Y2 = np.zeros((mech.N, n))
    ok = np.ones(n, bool)
    for i in range(n):
        T2[i] = T[i] + ALPHA * c[0, i] * (Tmax - Tmin)
        p2[i] = p[i] + BETA * c[1, i] * (pmax - pmin)
        yb = Y[b, i] + ALPHA * c[2, i] * (nmax - nmin)
        s = 0.0
        for k in range(mech.N):
            if k != b:
                Y2[k, i] = max(Y[k, i], 0.0) ** (1.0 + GAMMA * c[3 + k, i])
                s += Y2[k, i]
        if not (0.0 <= yb < 1.0) or s <= 0.0 or T2[i] <= 0.0 or p2[i] <= 0.0:
            ok[i] = False
            continue
        for k in range(mech.N):
            if k != b:
                Y2[k, i] *= (1.0 - yb) / s
        Y2[b, i] = yb
    return T2, p2, Y2, ok


def element_moles(mech, Y):
    """n_e = sum_k a_ek Y_k / W_k (mol of element e per kg), [E, n]."""
    return (np.asarray(mech.elem, np.float64).T @ (np.asarray(Y, np.float64) / np.asarray(mech.W)[:, None]))


def ratios(mech, Y):
    """(H/C, O/N, phi) per state from the element moles."""
    E = mech.elements
    ne = element_moles(mech, Y)
    nC, nH, nO, nN = ne[E.index("C")], ne[E.index("H")], ne[E.index("O")], ne[E.index("N")]
    with np.errstate(divide="ignore", invalid="ignore"):
        return nH / nC, nO / nN, (2.0 * nC + 0.5 * nH) / nO


def accept(mech, Y, ok=None):
    """Table 1: H/C, O/N and phi within their bounds (inclusive)."""
    hc, on, phi = ratios(mech, Y)
    a = ((hc >= HC_RANGE[0]) & (hc <= HC_RANGE[1]) & (on >= ON_RANGE[0]) & (on <= ON_RANGE[1])
         & (phi >= PHI_RANGE[0]) & (phi <= PHI_RANGE[1]))
    return a if ok is None else (a & ok)


def premixed(mech, phi: float):
    """Mass fractions of the fuel / air mixture at equivalence ratio phi (3.76 mol N2 per mol O2)
    and of its complete-combustion products."""
    r = mech.roles
    E = mech.elements
    fuel, ox, bath, water, co2 = r["fuel"], r["oxidizer"], mech.bath, r["water"], r["co2"]
    nC, nH = mech.elem[fuel, E.index("C")], mech.elem[fuel, E.index("H")]
    o2_st = nC + nH / 4.0
    Xu = np.zeros(mech.N)
    Xu[fuel] = phi / o2_st
    Xu[ox] = 1.0
    Xu[bath] = 3.76
    burnt = min(1.0, 1.0 / phi) * Xu[fuel]
    Xb = Xu.copy()
    Xb[fuel] -= burnt
    Xb[ox] = max(Xb[ox] - burnt * o2_st, 0.0)
    Xb[water] += burnt * nH / 2.0
    Xb[co2] += burnt * nC
    to_mass = lambda X: X * mech.W / np.dot(X, mech.W)
    return to_mass(Xu), to_mass(Xb)


def adiabatic_equilibrium(mech, phi: float = 0.45, T0: float = 300.0, p: float = 101325.0, t_end: float = 1.0):
    """The adiabatic, isobaric equilibrium of the phi mixture: its complete-combustion products
    at the temperature that holds the unburnt mixture's enthalpy (Newton on NASA-7 h), integrated
    by the oracle's reactor to t_end. Returns (T_eq, Y_eq)."""
    import oracle as O
    Yu, Yb = premixed(mech, phi)
    pa = np.array([p])
    h0 = O.props(mech, np.array([T0]), pa, Yu[:, None])[1][0]
    T = 2000.0
    for _ in range(100):
        cp, h = O.props(mech, np.array([T]), pa, Yb[:, None])[:2]
        d = (h[0] - h0) / cp[0]
        T -= d
        if abs(d) < 1e-10:
            break
    y, st, _ = O.integrate_cell(mech, p, t_end, np.concatenate([[T], Yb]), rtol=1e-10, atol_Y=1e-16, atol_T=1e-10,
                                h0=1e-9, max_steps=200000)
    if st != 0:
        raise RuntimeError("equilibrium integration failed with status %d" % st)
    return y[0], y[1:]


def air(mech, T: float = 300.0):
    """(T, Y) of ambient air: 1 mol O2 with 3.76 mol N2."""
    X = np.zeros(mech.N)
    X[mech.roles["oxidizer"]] = 1.0
    X[mech.bath] = 3.76
    return T, X * mech.W / np.dot(X, mech.W)


def blend(s, T_a, Y_a, T_b, Y_b):
    """States on the line from (T_a, Y_a) at s = 0 to (T_b, Y_b) at s = 1, for all species."""
    s = np.asarray(s, np.float64)
    return (1.0 - s) * T_a + s * T_b, (1.0 - s)[None, :] * Y_a[:, None] + s[None, :] * Y_b[:, None]
