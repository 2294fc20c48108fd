"""Seeded synthetic inputs: reaction mechanisms and cell states.

This module is the one place that both the CUDA path and the CPU oracle take
their inputs from. It builds *data* (mechanism tables and cell states); it
evaluates none of the per-cell arithmetic of the method itself (no mixture
properties, no reaction rates, no integration). The paper's own mechanism
(DRM19, Sec. 3.1) and its flamelet data are not available, so every mechanism
here is a seeded stand-in with the sizes of the workloads the paper motivates:

* ``mech_c1``: 9 species (H/O/N), 20 reversible reactions, 4 three-body.
* ``mech_c2``: 30 species (C/H/O/N), 180 reactions, 18 Troe fall-off, 27 three-body.
* ``mech_c5``: 53 species (C/H/O/N), 325 reactions, 33 Troe fall-off, 49 three-body.

Species are generic element vectors named ``S<k>``; none is copied from a real
mechanism. NASA-7 polynomials are least-squares fits to seeded smooth cp(T)
curves (rigid rotor plus seeded Einstein vibrational modes), continuous in cp,
H and S at 1000 K. Transport data are seeded Lennard-Jones parameters turned
into polynomial fits (in x = ln(T/1000)) of ln(mu_k) and of the reduced binary
resistance g_jk = p T^-3/2 / D_jk, using the Chapman-Enskog expressions with
the Neufeld-Janzen-Aziz collision-integral fits. Fits are mechanism data: both
sides evaluate the same polynomials.

Units are SI throughout (kg, m, s, mol, K, J). Arrhenius pre-factors are drawn
in cm-mol-s and converted by 10^(-6 (order - 1)).
"""
from __future__ import annotations

import dataclasses
import struct
from typing import Dict, List, Tuple

import numpy as np

R_GAS = 8.314462618          # J/mol/K
K_BOLTZ = 1.380649e-23       # J/K
N_AVO = 6.02214076e23        # 1/mol
P_STD = 101325.0             # Pa, standard-state pressure of the NASA-7 data
P_ATM = 101325.0

T_LO, T_MID, T_HI = 300.0, 1000.0, 3500.0
FIT_T_LO, FIT_T_HI = 250.0, 3500.0     # range of the transport fits

ATOMIC_W = {"C": 12.011e-3, "H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}
# enthalpy of formation of the gaseous atoms at 298.15 K (J/mol); used only to
# seed species enthalpies through an atomisation model
ATOM_HF = {"C": 716.7e3, "H": 218.0e3, "O": 249.2e3, "N": 472.7e3}

RT_ELEMENTARY, RT_THREEBODY, RT_TROE = 0, 1, 2
MAGIC = b"CHMECH01"


@dataclasses.dataclass
class Mech:
    """A reaction mechanism as plain arrays (SI units)."""
    name: str
    elements: List[str]
    elem: np.ndarray        # [N, E] int32 atom counts
    W: np.ndarray           # [N] kg/mol
    nasa_lo: np.ndarray     # [N, 7] valid on [T_LO, T_MID)
    nasa_hi: np.ndarray     # [N, 7] valid on [T_MID, T_HI]
    sigma: np.ndarray       # [N] Lennard-Jones diameter, Angstrom
    eps_k: np.ndarray       # [N] Lennard-Jones well depth / k_B, K
    visc_fit: np.ndarray    # [N, 5] ln(mu_k / Pa s) = sum_n c_n x^n, x = ln(T/1000)
    diff_fit: np.ndarray    # [N, N, 5] g_jk = sum_n c_n x^n (g_kk = 0)
    rtype: np.ndarray       # [R] int32: 0 elementary, 1 three-body, 2 Troe fall-off
    reac: np.ndarray        # [R, 3] int32 reactant species (repeated for nu = 2), -1 pad
    prod: np.ndarray        # [R, 3] int32 product species, -1 pad
    A: np.ndarray           # [R] SI pre-factor of k_f (k_inf for fall-off)
    beta: np.ndarray        # [R]
    Ea: np.ndarray          # [R] J/mol
    A0: np.ndarray          # [R] low-pressure limit (fall-off only, else 0)
    beta0: np.ndarray
    Ea0: np.ndarray
    troe: np.ndarray        # [R, 4] (a, T***, T*, T**) (fall-off only)
    eff: np.ndarray         # [R, N] third-body efficiencies (1 where unused)
    bath: int               # index of the inert bath species (largest mean Y)
    roles: Dict[str, int]   # fuel / oxidizer / product indices used by the state sampler
    hf298: np.ndarray       # [N] J/mol, seeded enthalpy of formation (data only)
    s298: np.ndarray        # [N] seeded S(298.15 K)/R (data only)

    @property
    def N(self) -> int:
        return int(self.W.shape[0])

    @property
    def R(self) -> int:
        return int(self.rtype.shape[0])

    def nu(self) -> Tuple[np.ndarray, np.ndarray]:
        """Dense stoichiometric matrices (nu', nu'') of shape [R, N]."""
        nr = np.zeros((self.R, self.N), np.int64)
        npd = np.zeros((self.R, self.N), np.int64)
        for j in range(self.R):
            for s in self.reac[j]:
                if s >= 0:
                    nr[j, s] += 1
            for s in self.prod[j]:
                if s >= 0:
                    npd[j, s] += 1
        return nr, npd


# ----------------------------------------------------------------------------
# thermodynamic data (fits of seeded cp curves)
# ----------------------------------------------------------------------------

def _einstein(theta: np.ndarray, T: np.ndarray) -> np.ndarray:
    x = theta[None, :] / T[:, None]
    ex = np.exp(-x)
    return (x * x * ex / (1.0 - ex) ** 2).sum(axis=1)


def _cp_curve(natoms: int, thetas: np.ndarray, T: np.ndarray) -> np.ndarray:
    base = 2.5 if natoms == 1 else (3.5 if natoms == 2 else 4.0)
    if thetas.size == 0:
        return np.full_like(T, base)
    return base + _einstein(thetas, T)


def _fit_nasa(natoms: int, thetas: np.ndarray, hf: float, s298: float):
    """NASA-7 low/high coefficient sets for one species.

    Low range: unconstrained least squares of cp/R in tau = T/1000.
    High range: least squares with cp/R pinned to the low fit at 1000 K.
    a6/a7 of the low range reproduce H(298.15) and S(298.15); those of the
    high range make H and S continuous at 1000 K.
    """
    Tl = np.linspace(T_LO, T_MID, 120)
    Th = np.linspace(T_MID, T_HI, 200)
    cl = _cp_curve(natoms, thetas, Tl)
    ch = _cp_curve(natoms, thetas, Th)
    tl = Tl / 1000.0
    Vl = np.stack([tl ** k for k in range(5)], axis=1)
    c_lo = np.linalg.lstsq(Vl, cl, rcond=None)[0]
    cp1 = float(c_lo.sum())                       # cp/R of the low fit at tau = 1
    th = Th / 1000.0
    Vh = np.stack([th ** k - 1.0 for k in range(1, 5)], axis=1)
    d = np.linalg.lstsq(Vh, ch - cp1, rcond=None)[0]
    c_hi = np.concatenate([[cp1 - d.sum()], d])
    scale = np.array([1.0, 1e-3, 1e-6, 1e-9, 1e-12])
    lo = np.zeros(7)
    hi = np.zeros(7)
    lo[:5] = c_lo * scale
    hi[:5] = c_hi * scale

    def h_poly(a, T):   # H/R without a6
        return T * (a[0] + a[1] * T / 2 + a[2] * T ** 2 / 3 + a[3] * T ** 3 / 4 + a[4] * T ** 4 / 5)

    def s_poly(a, T):   # S/R without a7
        return a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4

    T0 = 298.15
    lo[5] = hf / R_GAS - h_poly(lo, T0)
    lo[6] = s298 - s_poly(lo, T0)
    hi[5] = h_poly(lo, T_MID) + lo[5] - h_poly(hi, T_MID)
    hi[6] = s_poly(lo, T_MID) + lo[6] - s_poly(hi, T_MID)
    return lo, hi


# ----------------------------------------------------------------------------
# transport data
# ----------------------------------------------------------------------------

def _omega22(ts: np.ndarray) -> np.ndarray:
    # Neufeld, Janzen and Aziz (1972) fit of the reduced collision integral
    return 1.16145 * ts ** -0.14874 + 0.52487 * np.exp(-0.77320 * ts) + 2.16178 * np.exp(-2.43787 * ts)


def _omega11(ts: np.ndarray) -> np.ndarray:
    return (1.06036 * ts ** -0.15610 + 0.19300 * np.exp(-0.47635 * ts)
            + 1.03587 * np.exp(-1.52996 * ts) + 1.76474 * np.exp(-3.89411 * ts))


def _transport_fits(W: np.ndarray, sigma: np.ndarray, eps_k: np.ndarray):
    N = W.size
    T = np.geomspace(FIT_T_LO, FIT_T_HI, 160)
    x = np.log(T / 1000.0)
    V = np.stack([x ** k for k in range(5)], axis=1)
    m = W / N_AVO
    sig = sigma * 1e-10
    mu = (5.0 / 16.0) * np.sqrt(np.pi * m[None, :] * K_BOLTZ * T[:, None]) / (
        np.pi * sig[None, :] ** 2 * _omega22(T[:, None] / eps_k[None, :]))
    visc = np.linalg.lstsq(V, np.log(mu), rcond=None)[0].T.copy()          # [N, 5]
    sjk = 0.5 * (sig[:, None] + sig[None, :])
    ejk = np.sqrt(eps_k[:, None] * eps_k[None, :])
    mjk = m[:, None] * m[None, :] / (m[:, None] + m[None, :])
    # g_jk = p T^-1.5 / D_jk with D_jk = 3/16 sqrt(2 pi (kT)^3 / m_jk) / (p pi s^2 Omega11)
    pref = (16.0 / 3.0) * np.pi * sjk ** 2 * np.sqrt(mjk) / (np.sqrt(2.0 * np.pi) * K_BOLTZ ** 1.5)
    g = pref[None, :, :] * _omega11(T[:, None, None] / ejk[None, :, :])    # [nT, N, N]
    coef = np.linalg.lstsq(V, g.reshape(T.size, N * N), rcond=None)[0]     # [5, N*N]
    diff = coef.T.reshape(N, N, 5).copy()
    diff = 0.5 * (diff + diff.transpose(1, 0, 2))
    for k in range(N):
        diff[k, k, :] = 0.0
    return visc, diff


# ----------------------------------------------------------------------------
# species and reactions
# ----------------------------------------------------------------------------

def _core_species(elements: List[str]):
    """Element vectors of the role species; values of hf are textbook-like seeds."""
    def vec(**kw):
        return tuple(kw.get(e, 0) for e in elements)
    core = [
        ("bath", vec(N=2), 0.0),
        ("oxidizer", vec(O=2), 0.0),
        ("h2", vec(H=2), 0.0),
        ("water", vec(H=2, O=1), -241.8e3),
        ("h", vec(H=1), 218.0e3),
        ("o", vec(O=1), 249.2e3),
        ("oh", vec(H=1, O=1), 39.0e3),
    ]
    if "C" in elements:
        core += [
            ("fuel", vec(C=1, H=4), -74.9e3),
            ("co2", vec(C=1, O=2), -393.5e3),
            ("co", vec(C=1, O=1), -110.5e3),
        ]
    return core


def _candidate_species(elements: List[str]):
    out = []
    has_c = "C" in elements
    for c in range(0, 4 if has_c else 1):
        for h in range(0, 9):
            for o in range(0, 4):
                for n in range(0, 1):          # nitrogen only in the inert bath
                    na = c + h + o + n
                    if na < 1 or na > 8:
                        continue
                    v = {"C": c, "H": h, "O": o, "N": n}
                    out.append(tuple(v[e] for e in elements))
    return out


def _enumerate_reactions(elem: np.ndarray):
    N = elem.shape[0]
    key = {}
    for s in range(N):
        key.setdefault(tuple(elem[s]), []).append(s)
    recomb = []   # (A, B, AB)
    for a in range(N):
        for b in range(a, N):
            t = tuple(elem[a] + elem[b])
            for c in key.get(t, []):
                recomb.append((a, b, c))
    pairs: Dict[tuple, list] = {}
    for a in range(N):
        for b in range(a, N):
            pairs.setdefault(tuple(elem[a] + elem[b]), []).append((a, b))
    exch = []
    for plist in pairs.values():
        for i in range(len(plist)):
            for j in range(i + 1, len(plist)):
                exch.append((plist[i], plist[j]))
    return recomb, exch


def make_mech(name: str, n_species: int, n_reactions: int, n_troe: int, n_threebody: int,
              elements: List[str], seed: int) -> Mech:
    """Build a seeded element-balanced mechanism (deterministic for a seed)."""
    rng = np.random.default_rng(seed)
    core = _core_species(elements)
    comp = [c[1] for c in core]
    roles = {c[0]: i for i, c in enumerate(core)}
    hf = [c[2] for c in core]
    cands = [v for v in _candidate_species(elements) if v not in comp]
    E = len(elements)
    # extra species: draw until the recombination pool is large enough
    for _attempt in range(200):
        wts = np.array([1.0 / float(sum(v)) ** 3 for v in cands])
        pick = rng.choice(len(cands), size=n_species - len(core), replace=False, p=wts / wts.sum())
        extra = [cands[i] for i in pick]
        elem = np.array(comp + extra, dtype=np.int32).reshape(n_species, E)
        recomb, exch = _enumerate_reactions(elem)
        if len(recomb) >= n_troe + n_threebody + 2 and len(exch) + len(recomb) >= n_reactions:
            break
    else:
        raise RuntimeError("could not draw a species set with enough reactions")
    natoms = elem.sum(axis=1)
    W = (elem * np.array([ATOMIC_W[e] for e in elements])[None, :]).sum(axis=1)
    # seeded enthalpies of formation of the extra species: atomisation model
    for s in range(len(core), n_species):
        atom_sum = float((elem[s] * np.array([ATOM_HF[e] for e in elements])).sum())
        bonds = max(natoms[s] - 1, 0)
        hf.append(atom_sum - bonds * rng.uniform(380e3, 470e3) + (0.0 if bonds else 0.0))
    hf = np.array(hf)
    s298 = 13.0 + 3.0 * natoms + rng.uniform(-1.0, 1.0, n_species)
    nasa_lo = np.zeros((n_species, 7))
    nasa_hi = np.zeros((n_species, 7))
    for s in range(n_species):
        nmodes = 0 if natoms[s] == 1 else (1 if natoms[s] == 2 else 3 * natoms[s] - 6)
        thetas = rng.uniform(500.0, 5000.0, nmodes)
        nasa_lo[s], nasa_hi[s] = _fit_nasa(int(natoms[s]), thetas, float(hf[s]), float(s298[s]))
    sigma = rng.uniform(2.5, 5.0, n_species)
    eps_k = rng.uniform(50.0, 600.0, n_species)
    visc, diff = _transport_fits(W, sigma, eps_k)

    # ---- reactions
    bath = roles["bath"]
    recomb = [r for r in recomb if bath not in r]
    exch = [r for r in exch if bath not in r[0] and bath not in r[1]]
    rng.shuffle(recomb)
    rng.shuffle(exch)
    n_rec = n_troe + n_threebody
    chosen = []      # (type, reactants, products)
    for k in range(n_rec):
        a, b, c = recomb[k]
        chosen.append((RT_TROE if k < n_troe else RT_THREEBODY, [a, b], [c]))
    pool = [("x", list(p), list(q)) for p, q in exch] + [("r", [a, b], [c]) for a, b, c in recomb[n_rec:]]
    order = rng.permutation(len(pool))
    used = set()
    for i in order:
        if len(chosen) >= n_reactions:
            break
        kind, rr, pp = pool[i]
        chosen.append((RT_ELEMENTARY, rr, pp))
        used.add(i)
    # coverage: every non-bath species appears in at least one reaction
    def covered():
        cov = set()
        for _, rr, pp in chosen:
            cov.update(rr)
            cov.update(pp)
        return cov
    for s in range(n_species):
        if s == bath or s in covered():
            continue
        for i in order:
            if i in used:
                continue
            kind, rr, pp = pool[i]
            if s in rr or s in pp:
                # replace the last elementary reaction whose removal keeps coverage
                for q in range(len(chosen) - 1, n_rec - 1, -1):
                    trial = chosen[:q] + chosen[q + 1:]
                    cov = set()
                    for _, r2, p2 in trial:
                        cov.update(r2)
                        cov.update(p2)
                    if all((t in cov) for t in covered() if t != s):
                        chosen[q] = (RT_ELEMENTARY, rr, pp)
                        used.add(i)
                        break
                break
    R = len(chosen)
    rtype = np.zeros(R, np.int32)
    reac = -np.ones((R, 3), np.int32)
    prod = -np.ones((R, 3), np.int32)
    A = np.zeros(R)
    beta = np.zeros(R)
    Ea = np.zeros(R)
    A0 = np.zeros(R)
    beta0 = np.zeros(R)
    Ea0 = np.zeros(R)
    troe = np.zeros((R, 4))
    eff = np.ones((R, n_species))
    for j, (t, rr, pp) in enumerate(chosen):
        dh = hf[pp].sum() - hf[rr].sum()
        if dh > 0.0:               # orient every reaction exothermic in the forward direction
            rr, pp = pp, rr
        rtype[j] = t
        reac[j, :len(rr)] = sorted(rr)
        prod[j, :len(pp)] = sorted(pp)
        order_f = len(rr)
        la = rng.uniform(8.0, 14.0)
        beta[j] = rng.uniform(-1.5, 1.5)
        Ea[j] = rng.uniform(0.0, 40.0) * 4184.0
        if t == RT_THREEBODY:
            A[j] = 10.0 ** la * 1e-6 ** order_f          # order_f + 1 with the third body
        else:
            A[j] = 10.0 ** la * 1e-6 ** (order_f - 1)
        if t == RT_TROE:
            A0[j] = 10.0 ** (la + rng.uniform(2.0, 5.0)) * 1e-6 ** order_f
            beta0[j] = rng.uniform(-1.5, 1.5)
            Ea0[j] = rng.uniform(0.0, 40.0) * 4184.0
            troe[j] = [rng.uniform(0.3, 0.8), rng.uniform(50.0, 300.0),
                       rng.uniform(500.0, 3000.0), rng.uniform(2000.0, 8000.0)]
        if t != RT_ELEMENTARY:
            sp = rng.choice(n_species, size=3, replace=False)
            eff[j, sp] = rng.uniform(0.5, 2.5, 3)
    return Mech(name=name, elements=list(elements), elem=elem, W=W, nasa_lo=nasa_lo, nasa_hi=nasa_hi,
                sigma=sigma, eps_k=eps_k, visc_fit=visc, diff_fit=diff, rtype=rtype, reac=reac, prod=prod,
                A=A, beta=beta, Ea=Ea, A0=A0, beta0=beta0, Ea0=Ea0, troe=troe, eff=eff, bath=bath,
                roles=roles, hf298=hf, s298=s298)


_MECH_CACHE: Dict[str, Mech] = {}


def mech_c1() -> Mech:
    """9 species H/O/N, 20 reactions, 4 three-body (seed 1001)."""
    if "c1" not in _MECH_CACHE:
        _MECH_CACHE["c1"] = make_mech("c1", 9, 20, 0, 4, ["H", "O", "N"], 1001)
    return _MECH_CACHE["c1"]


def mech_c2() -> Mech:
    """30 species C/H/O/N, 180 reactions: 18 Troe fall-off, 27 three-body (seed 1002)."""
    if "c2" not in _MECH_CACHE:
        _MECH_CACHE["c2"] = make_mech("c2", 30, 180, 18, 27, ["C", "H", "O", "N"], 1002)
    return _MECH_CACHE["c2"]


def mech_c5() -> Mech:
    """53 species C/H/O/N, 325 reactions: 33 Troe fall-off, 49 three-body (seed 1005)."""
    if "c5" not in _MECH_CACHE:
        _MECH_CACHE["c5"] = make_mech("c5", 53, 325, 33, 49, ["C", "H", "O", "N"], 1005)
    return _MECH_CACHE["c5"]


def get_mech(name: str) -> Mech:
    return {"c1": mech_c1, "c2": mech_c2, "c5": mech_c5}[name]()


# ----------------------------------------------------------------------------
# binary mechanism file (read by the C-ABI library's chem_mech_load)
# ----------------------------------------------------------------------------

def mech_to_bytes(m: Mech) -> bytes:
    """Serialise in the fixed little-endian layout documented in include/chemgb.h."""
    E = len(m.elements)
    parts = [MAGIC, struct.pack("<4i", m.N, m.R, E, m.bath),
             struct.pack("<4d", P_STD, T_LO, T_MID, T_HI)]
    f64 = lambda a: np.ascontiguousarray(a, dtype="<f8").tobytes()
    i32 = lambda a: np.ascontiguousarray(a, dtype="<i4").tobytes()
    parts += [f64(m.W), f64(m.nasa_lo), f64(m.nasa_hi), i32(m.elem), f64(m.sigma), f64(m.eps_k),
              f64(m.visc_fit), f64(m.diff_fit), i32(m.rtype), i32(m.reac), i32(m.prod),
              f64(m.A), f64(m.beta), f64(m.Ea), f64(m.A0), f64(m.beta0), f64(m.Ea0),
              f64(m.troe), f64(m.eff)]
    return b"".join(parts)


def write_mech(m: Mech, path: str) -> str:
    with open(path, "wb") as fh:
        fh.write(mech_to_bytes(m))
    return path


# ----------------------------------------------------------------------------
# cell states (structure of arrays: T[ld], p[ld], Y[N, ld])
# ----------------------------------------------------------------------------

def padded_ld(ncells: int, align: int = 4) -> int:
    return max(align, ((ncells + align - 1) // align) * align)


def states_dirichlet(m: Mech, ncells: int, seed: int, ld: int | None = None):
    """T ~ U[300, 2500] K, p = 1 atm, Y ~ Dirichlet(0.5) (small parity workload)."""
    rng = np.random.default_rng(seed)
    ld = ld or padded_ld(ncells)
    T = np.zeros(ld)
    p = np.zeros(ld)
    Y = np.zeros((m.N, ld))
    T[:ncells] = rng.uniform(300.0, 2500.0, ncells)
    p[:ncells] = P_ATM
    Y[:, :ncells] = rng.dirichlet(np.full(m.N, 0.5), size=ncells).T
    return T, p, Y


def _mole_to_mass(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    Y = X * W[:, None]
    return Y / Y.sum(axis=0, keepdims=True)


def states_profiles(m: Mech, ncells: int, seed: int, ld: int | None = None,
                    phi_range=(0.5, 1.2), noise: float = 0.05):
    """Cells sampled along algebraic 1-D stratified premixed profiles.

    Stand-in for flamelet data: a mixture-fraction coordinate s ~ U[0,1] sets the
    equivalence ratio phi = phi_lo + s (phi_hi - phi_lo); a progress variable
    c ~ U[0,1] blends the unburnt fuel/air mixture with its complete-combustion
    products, and each intermediate species gets a bump 4c(1-c) with a seeded
    amplitude (a fixed property of the mechanism, the same for every state
    seed). T rises from 300 K to a burnt value estimated from the seeded
    formation enthalpies with a constant cp of 1400 J/kg/K (the estimate only
    shapes the sample; it is not the method's thermodynamics). Mass fractions
    then get a log-normal perturbation exp(noise * xi) and are renormalised.
    """
    rng = np.random.default_rng(seed)
    ld = ld or padded_ld(ncells)
    N = m.N
    r = m.roles
    E = m.elements
    ce = m.elem
    iC = E.index("C") if "C" in E else None
    iH = E.index("H")
    iO = E.index("O")
    fuel = r.get("fuel", r["h2"])
    ox, bath, water = r["oxidizer"], r["bath"], r["water"]
    co2 = r.get("co2")
    nC = ce[fuel, iC] if iC is not None else 0
    nH = ce[fuel, iH]
    o2_st = nC + nH / 4.0            # mol O2 per mol fuel at stoichiometry
    s = rng.uniform(0.0, 1.0, ncells)
    phi = phi_range[0] + s * (phi_range[1] - phi_range[0])
    c = rng.uniform(0.0, 1.0, ncells)
    # unburnt mole numbers per mol O2
    Xu = np.zeros((N, ncells))
    Xu[fuel] = phi / o2_st
    Xu[ox] = 1.0
    Xu[bath] = 3.76
    # burnt: burn min(1, 1/phi) of the fuel completely
    burnt = np.minimum(1.0, 1.0 / phi) * Xu[fuel]
    Xb = Xu.copy()
    Xb[fuel] -= burnt
    Xb[ox] -= burnt * o2_st
    Xb[water] += burnt * nH / 2.0
    if co2 is not None:
        Xb[co2] += burnt * nC
    Xb[ox] = np.maximum(Xb[ox], 0.0)
    Yu = _mole_to_mass(Xu, m.W)
    Yb = _mole_to_mass(Xb, m.W)
    dh = -((Yb - Yu) * (m.hf298 / m.W)[:, None]).sum(axis=0)     # J/kg released
    Tb = np.clip(300.0 + dh / 1400.0, 1200.0, 2700.0)
    T = 300.0 + c * (Tb - 300.0)
    Y = (1.0 - c)[None, :] * Yu + c[None, :] * Yb
    majors = {fuel, ox, bath, water} | ({co2} if co2 is not None else set())
    # the intermediates' peak amplitudes belong to the mechanism (fixed per mechanism), so every
    # state seed samples the same distribution; only the per-cell draws depend on `seed`
    amp = 10.0 ** np.random.default_rng(7000 + N).uniform(-6.0, -2.0, N)
    bump = 4.0 * c * (1.0 - c)
    for k in range(N):
        if k not in majors:
            Y[k] += amp[k] * bump * rng.uniform(0.5, 1.5, ncells) + 1e-12
    Y *= np.exp(noise * rng.standard_normal((N, ncells)))
    Y /= Y.sum(axis=0, keepdims=True)
    To = np.zeros(ld)
    po = np.zeros(ld)
    Yo = np.zeros((N, ld))
    To[:ncells] = T
    po[:ncells] = P_ATM
    Yo[:, :ncells] = Y
    return To, po, Yo


def fuel_air(m: Mech, phi: float):
    """Mass fractions of the fuel / air mixture at equivalence ratio phi (1 mol O2 with 3.76 mol
    of the bath species) and of its complete-combustion products (min(1, 1/phi) of the fuel burnt
    to water and CO2): the unburnt and burnt ends of the profiles above, for one phi."""
    r = m.roles
    E = m.elements
    fuel = r.get("fuel", r["h2"])
    ox, bath, water, co2 = r["oxidizer"], r["bath"], r["water"], r.get("co2")
    nC = m.elem[fuel, E.index("C")] if "C" in E else 0
    nH = m.elem[fuel, E.index("H")]
    o2_st = nC + nH / 4.0
    Xu = np.zeros(m.N)
    Xu[fuel] = phi / o2_st
    Xu[ox] = 1.0
    Xu[bath] = 3.76
    burnt = min(1.0, 1.0 / phi) * Xu[fuel]
    Xb = Xu.copy()
    Xb[fuel] -= burnt
    Xb[ox] = max(Xb[ox] - burnt * o2_st, 0.0)
    Xb[water] += burnt * nH / 2.0
    if co2 is not None:
        Xb[co2] += burnt * nC
    return Xu * m.W / np.dot(Xu, m.W), Xb * m.W / np.dot(Xb, m.W)


def air(m: Mech):
    """Mass fractions of ambient air: 1 mol O2 with 3.76 mol of the bath species."""
    X = np.zeros(m.N)
    X[m.roles["oxidizer"]] = 1.0
    X[m.bath] = 3.76
    return X * m.W / np.dot(X, m.W)


def element_table(m: Mech, names=("C", "H", "O", "N")) -> np.ndarray:
    """[len(names)][N] int32 atom counts of the named elements (0 for an element the mechanism lacks)."""
    out = np.zeros((len(names), m.N), np.int32)
    for e, nm in enumerate(names):
        if nm in m.elements:
            out[e] = m.elem[:, m.elements.index(nm)]
    return out


def perturb_off_manifold(T: np.ndarray, Y: np.ndarray, ncells: int, frac: float, seed: int,
                         dT: float = 300.0, sigma: float = 0.2):
    """Move a seeded fraction of cells off the sampled manifold (T +/- dT with a
    fair sign, clipped to >= 250 K; Y * exp(sigma xi), renormalised). Returns the
    perturbed copies and the boolean mask of moved cells."""
    rng = np.random.default_rng(seed)
    T = T.copy()
    Y = Y.copy()
    mask = np.zeros(T.shape[0], bool)
    idx = rng.choice(ncells, size=int(round(frac * ncells)), replace=False)
    mask[idx] = True
    sign = np.where(rng.uniform(size=idx.size) < 0.5, -1.0, 1.0)
    T[idx] = np.maximum(T[idx] + sign * dT, 250.0)
    Y[:, idx] *= np.exp(sigma * rng.standard_normal((Y.shape[0], idx.size)))
    Y[:, idx] /= Y[:, idx].sum(axis=0, keepdims=True)
    return T, Y, mask


# ----------------------------------------------------------------------------
# network parameters for tests (seeded uniform draws; no arithmetic of the method)
# ----------------------------------------------------------------------------

def mlp_layers(widths, seed: int):
    """[(W [out, in], b [out])] with entries U(-1/sqrt(in), 1/sqrt(in)), float32-representable."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in zip(widths[:-1], widths[1:]):
        a = 1.0 / np.sqrt(fi)
        W = rng.uniform(-a, a, (fo, fi)).astype(np.float32).astype(np.float64)
        b = rng.uniform(-a, a, fo).astype(np.float32).astype(np.float64)
        out.append((W, b))
    return out


def mlp_ensemble(widths, seed: int):
    """G = widths[-1] networks of widths [n_in, h1, h2, h3, 1] (one per output, the per-species
    model), network g drawn as mlp_layers draws a network with seed + g."""
    return [mlp_layers(list(widths[:-1]) + [1], seed + g) for g in range(widths[-1])]


def stack_ensemble(nets):
    """Per-output networks in the C ABI's ensemble layout: per layer, the networks' weight
    matrices stacked row-wise (network g's rows follow network g - 1's) and their biases
    concatenated."""
    return [(np.concatenate([net[l][0] for net in nets], axis=0), np.concatenate([net[l][1] for net in nets]))
            for l in range(len(nets[0]))]


def unstack_ensemble(layers, G: int):
    """The inverse of stack_ensemble for G networks."""
    out = [[] for _ in range(G)]
    for W, b in layers:
        r = W.shape[0] // G
        for g in range(G):
            out[g].append((W[g * r:(g + 1) * r], b[g * r:(g + 1) * r]))
    return out


def flatten_layers(layers):
    """Layer-by-layer W (row-major) then b, as float32 (the C ABI's parameter layout)."""
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers]).astype(np.float32)


def unflatten(flat, widths):
    out, o = [], 0
    for fi, fo in zip(widths[:-1], widths[1:]):
        W = flat[o:o + fo * fi].reshape(fo, fi).astype(np.float64)
        o += fo * fi
        b = flat[o:o + fo].astype(np.float64)
        o += fo
        out.append((W, b))
    return out
