"""FP64 oracle of the physics terms of the training loss (TEST INFRASTRUCTURE ONLY), Sec. 3.2.

Beside Eq. 5 the paper adds three principles to the loss: mass-fraction unity, energy
conservation and the heat release rate. It gives no formula or weight; the readings here:
  * The network's outputs are the non-bath species; the bath takes dY_bath = -sum_k dY_k, so
    sum Y = 1 holds by construction. The unity term therefore penalises the error of the
    implied bath change:  L_m = (1/B) sum_i |sum_k (dY_ik - dY*_ik)| / s_m.
  * Energy is conserved by the step's temperature update (h(T', Y') = h(T, Y)). What the
    composition change must get right is the chemical heat it releases at the cell's
    temperature, q = -sum_k h_k(T) dY_k (J/kg, bath included through the closure), so the
    energy and heat-release principles are one term:  L_q = (1/B) sum_i |q_i - q*_i| / s_q.
  * dY_k = sd_k u_k + mu_k (de-normalised outputs); s_m is the mean total absolute change of the
    output species, (1/B) sum_i sum_k |dY*_ik|, and s_q the mean absolute heat release of the
    training targets (the mean bath change itself is no scale: a bath species that takes part in
    no reaction, like N2 in these mechanisms, changes by exactly zero); the total loss is
    Eq. 5 + lam_m L_m + lam_q L_q.
Returns the loss and dL/du (sign(0) = 0). Plain numpy and the C oracle's species enthalpies.
"""
from __future__ import annotations

import numpy as np

from . import mlp as M


def species_enthalpy(mech, T):
    """h_k(T) in J/kg for every species, [N, n]."""
    import oracle as O
    from paper_2312_05800_gb300 import synth
    T = np.asarray(T, np.float64)
    h = np.empty((mech.N, len(T)))
    for i, t in enumerate(T):
        for k in range(mech.N):
            h[k, i] = O.species_thermo(mech, k, t)[1] * synth.R_GAS * t / mech.W[k]
    return h


def heat_release(mech, T, dY_out, sp):
    """q = -sum_k h_k(T) dY_k over all species, with dY_bath = -sum of the outputs' dY. dY_out: [B, G]."""
    h = species_enthalpy(mech, T)                                # [N, B]
    c = h[sp, :] - h[mech.bath, :][None, :]                      # [G, B]: the closure folded in
    return -(c.T * dY_out).sum(axis=1), c.T


def scales(mech, T, dY_target, sp):
    """(s_m, s_q): the mean over samples of sum_k |dY*_k| and of |q*|."""
    q, _ = heat_release(mech, T, dY_target, sp)
    return float(np.abs(dY_target).sum(axis=1).mean()), float(np.abs(q).mean())


def loss(mech, u, u_target, T, stats, sp, lam_m, lam_q, s_m, s_q):
    """Eq. 5 plus the two physics terms on normalised outputs u, u* [B, G]."""
    mu_u, sd_u = stats[2], stats[3]
    B = u.shape[0]
    l1, g = M.l1_loss(u, u_target)
    dY = u * sd_u + mu_u
    dYt = u_target * sd_u + mu_u
    rm = (dY - dYt).sum(axis=1)
    q, c = heat_release(mech, T, dY, sp)
    qt, _ = heat_release(mech, T, dYt, sp)
    rq = q - qt
    total = l1 + lam_m * np.abs(rm).sum() / (B * s_m) + lam_q * np.abs(rq).sum() / (B * s_q)
    g = g + (lam_m / (B * s_m)) * np.sign(rm)[:, None] * sd_u[None, :]
    g = g - (lam_q / (B * s_q)) * np.sign(rq)[:, None] * c * sd_u[None, :]
    return float(total), g
