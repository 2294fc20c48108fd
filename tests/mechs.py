"""Tiny hand-built mechanisms with closed-form behaviour (test helpers)."""
import numpy as np

from paper_2312_05800_gb300 import synth


def const_cp_nasa(cp_R: float, hf: float, s_R: float):
    """NASA-7 rows for a constant-cp species with H(298.15) = hf, S(298.15)/R = s_R."""
    a = np.zeros(7)
    a[0] = cp_R
    a[5] = hf / synth.R_GAS - cp_R * 298.15
    a[6] = s_R - cp_R * np.log(298.15)
    return a, a.copy()


def tiny_mech(species, reactions, W=None, name="tiny"):
    """species: list of (cp_R, hf, s_R); reactions: list of dicts with keys
    reac, prod, A, beta, Ea, type (0/1/2), optional eff, A0, beta0, Ea0, troe."""
    N = len(species)
    R = len(reactions)
    W = np.full(N, 0.028) if W is None else np.asarray(W, float)
    lo = np.zeros((N, 7))
    hi = np.zeros((N, 7))
    for k, (c, h, s) in enumerate(species):
        lo[k], hi[k] = const_cp_nasa(c, h, s)
    rtype = np.zeros(R, np.int32)
    reac = -np.ones((R, 3), np.int32)
    prod = -np.ones((R, 3), np.int32)
    A = np.zeros(R); beta = np.zeros(R); Ea = np.zeros(R)
    A0 = np.zeros(R); beta0 = np.zeros(R); Ea0 = np.zeros(R)
    troe = np.zeros((R, 4)); eff = np.ones((R, N))
    for j, r in enumerate(reactions):
        rtype[j] = r.get("type", 0)
        reac[j, :len(r["reac"])] = r["reac"]
        prod[j, :len(r["prod"])] = r["prod"]
        A[j] = r["A"]; beta[j] = r.get("beta", 0.0); Ea[j] = r.get("Ea", 0.0)
        A0[j] = r.get("A0", 0.0); beta0[j] = r.get("beta0", 0.0); Ea0[j] = r.get("Ea0", 0.0)
        if "troe" in r:
            troe[j] = r["troe"]
        if "eff" in r:
            eff[j] = r["eff"]
    elem = np.ones((N, 1), np.int32)
    return synth.Mech(name=name, elements=["X"], elem=elem, W=W, nasa_lo=lo, nasa_hi=hi,
                      sigma=np.full(N, 3.5), eps_k=np.full(N, 100.0), visc_fit=np.zeros((N, 5)),
                      diff_fit=np.zeros((N, N, 5)), rtype=rtype, reac=reac, prod=prod, A=A, beta=beta, Ea=Ea,
                      A0=A0, beta0=beta0, Ea0=Ea0, troe=troe, eff=eff, bath=N - 1, roles={},
                      hf298=np.array([s[1] for s in species]), s298=np.array([s[2] for s in species]))
