"""FP64 oracle of the PaSR scaling of the chemistry (TEST INFRASTRUCTURE ONLY), Sec. 4.1.

The partially stirred reactor closure scales a cell's reaction rate by
kappa = tau_c / (tau_c + tau_mix). The paper names the two time scales in words only;
the readings written out here:
  tau_c   the characteristic chemical time from the slowest species formation rate: the
          largest species time Y_k / |dY_k/dt| over the species with Y_k >= y_min and
          dY_k/dt != 0, at the state before the step (dY_k/dt from the reactor equations of
          Sec. 3.1); +inf when no species qualifies.
  tau_mix the geometric mean of the Taylor and Kolmogorov time scales, sqrt(tau_T tau_K).
  kappa   tau_c / (tau_c + tau_mix), and 1 where tau_c is infinite.
One chemistry step (T0, Y0) -> (T1, Y1) becomes Y' = Y0 + kappa (Y1 - Y0),
T' = T0 + kappa (T1 - T0). Plain loops over cells; the right-hand side is the C oracle's.
"""
from __future__ import annotations

import numpy as np


def chemical_time(mech, T, p, Y, y_min: float):
    """tau_c per cell for SoA T[n], p[n], Y[N, n]."""
    import oracle as O
    n = len(T)
    out = np.empty(n)
    for i in range(n):
        y = np.concatenate([[T[i]], Y[:, i]])
        f = O.rhs(mech, float(p[i]), y)
        best = -np.inf
        for k in range(mech.N):
            rate = abs(f[1 + k])
            if Y[k, i] >= y_min and rate > 0.0:
                best = max(best, Y[k, i] / rate)
        out[i] = best if best > -np.inf else np.inf
    return out


def kappa(tau_c, tau_taylor, tau_kolmogorov):
    tau_mix = np.sqrt(np.asarray(tau_taylor, np.float64) * np.asarray(tau_kolmogorov, np.float64))
    tau_c = np.asarray(tau_c, np.float64)
    with np.errstate(invalid="ignore"):
        k = tau_c / (tau_c + tau_mix)
    return np.where(np.isinf(tau_c), 1.0, k)


def apply(T0, Y0, T1, Y1, kap):
    """The scaled step: (T0 + kappa (T1 - T0), Y0 + kappa (Y1 - Y0))."""
    return T0 + kap * (T1 - T0), Y0 + kap[None, :] * (Y1 - Y0)
