"""Pins of the oracle's physics loss terms (Sec. 3.2: mass-fraction unity, energy and heat
release added to Eq. 5; forms and weights are readings, stated in oracle/physics_loss.py).

* The heat release from species enthalpies equals the change of the mixture enthalpy at fixed
  temperature computed by the oracle's property routine (h is linear in Y), closure included.
* With the prediction equal to the target both physics terms vanish and the loss is Eq. 5's.
* The gradient agrees with central finite differences away from the kinks.
* A prediction that conserves the bath change but misplaces heat (energy moved between two
  species of different enthalpy) is caught by the heat term alone.
"""
import numpy as np

import oracle as O
from oracle import ann as A
from oracle import mlp as M
from oracle import physics_loss as PL
from paper_2312_05800_gb300 import synth


def _case(B=6, seed=3):
    m = synth.get_mech("c1")
    T, p, Y = synth.states_dirichlet(m, B, seed)
    sp = A.out_species(m)
    G = len(sp)
    rng = np.random.default_rng(seed)
    mu_u = rng.normal(size=G) * 1e-5
    sd_u = 10.0 ** rng.uniform(-4, -2, G)
    return m, T[:B], p[:B], Y[:, :B], sp, (None, None, mu_u, sd_u), rng


def test_heat_release_is_the_mixture_enthalpy_change(oracle):
    m, T, p, Y, sp, stats, rng = _case()
    dY = rng.normal(size=(len(T), len(sp))) * 1e-3
    q, _ = PL.heat_release(m, T, dY, sp)
    Y1 = Y.copy()
    Y1[sp, :] += dY.T
    Y1[m.bath, :] -= dY.sum(axis=1)
    h0 = O.props(m, T, p, Y)[1]
    h1 = O.props(m, T, p, Y1)[1]
    assert np.allclose(q, -(h1 - h0), rtol=1e-9, atol=1e-9 * np.abs(h0).max())


def test_terms_vanish_on_the_target(oracle):
    m, T, p, Y, sp, stats, rng = _case()
    u = rng.normal(size=(len(T), len(sp)))
    L, g = PL.loss(m, u, u, T, stats, sp, 0.3, 0.3, 1.0, 1.0)
    l1, g1 = M.l1_loss(u, u)
    assert L == l1 == 0.0 and np.array_equal(g, g1)


def test_gradient_matches_finite_differences(oracle):
    m, T, p, Y, sp, stats, rng = _case()
    u = rng.normal(size=(len(T), len(sp)))
    ut = u + rng.normal(size=u.shape) * 0.5
    args = (T, stats, sp, 0.7, 0.4, 2e-3, 5e3)
    L, g = PL.loss(m, u, ut, *args)
    for _ in range(12):
        i, k = rng.integers(0, u.shape[0]), rng.integers(0, u.shape[1])
        e = 1e-7
        up, um = u.copy(), u.copy()
        up[i, k] += e
        um[i, k] -= e
        fd = (PL.loss(m, up, ut, *args)[0] - PL.loss(m, um, ut, *args)[0]) / (2 * e)
        assert abs(fd - g[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k, fd, g[i, k])


def test_heat_term_catches_misplaced_energy(oracle):
    m, T, p, Y, sp, stats, rng = _case(B=4)
    mu_u, sd_u = stats[2], stats[3]
    ut = np.zeros((len(T), len(sp)))
    # move mass between two output species: the bath change is unchanged, the heat is not
    a, b = 0, 1
    u = ut.copy()
    u[:, a] += 1e-3 / sd_u[a]
    u[:, b] -= 1e-3 / sd_u[b]
    dY, dYt = u * sd_u + mu_u, ut * sd_u + mu_u
    assert np.allclose((dY - dYt).sum(axis=1), 0.0, atol=1e-15)
    L_m_only = PL.loss(m, u, ut, T, stats, sp, 1.0, 0.0, 1.0, 1.0)[0]
    L_q_only = PL.loss(m, u, ut, T, stats, sp, 0.0, 1.0, 1.0, 1.0)[0]
    l1 = M.l1_loss(u, ut)[0]
    assert np.isclose(L_m_only, l1, rtol=1e-12)
    assert L_q_only > l1 + 1.0
