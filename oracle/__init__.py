"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` and
``--impl reference`` legs of ``bench.py`` may import this package. It shares
no code with the CUDA library (``paper_2312_05800_gb300``), and neither
imports the other; both take their inputs from ``paper_2312_05800_gb300.synth``.

``chem_oracle.c`` holds the thermo, transport, kinetics and Rosenbrock
integrator (plain C, FP64, OpenMP over cells); ``mlp.py`` holds the MLP
forward / backward / Adam and the Box-Cox / Z-score maps in numpy FP64;
``ann.py`` holds the ANN step that closes, clamps and renormalises the predicted
mass fractions and inverts the enthalpy for T.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libchem_oracle.so")
# ORACLE_SANITIZE=1 loads a build instrumented with AddressSanitizer and UndefinedBehaviorSanitizer
# (every finding aborts); the process must preload the ASan runtime (the tests do this)
_SAN_LIB = os.path.join(_BUILD, "libchem_oracle_san.so")
_lib = None


def _sanitized() -> bool:
    return os.environ.get("ORACLE_SANITIZE", "") == "1"


def build(force: bool = False, sanitize: bool = None) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP). Returns the library path."""
    if sanitize is None:
        sanitize = _sanitized()
    os.makedirs(_BUILD, exist_ok=True)
    out = _SAN_LIB if sanitize else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + ".tmp%d" % os.getpid()
        flags = (["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]
                 if sanitize else ["-O2"])
        cmd = ["gcc"] + flags + ["-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class _Mech(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("R", ctypes.c_int), ("E", ctypes.c_int), ("bath", ctypes.c_int),
                ("P_std", ctypes.c_double), ("T_lo", ctypes.c_double), ("T_mid", ctypes.c_double),
                ("T_hi", ctypes.c_double)] + [
        (nm, ctypes.c_void_p) for nm in ("W", "nasa_lo", "nasa_hi", "visc_fit", "diff_fit", "rtype", "reac",
                                         "prod", "A", "beta", "Ea", "A0", "beta0", "Ea0", "troe", "eff")]


class _Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol_Y", ctypes.c_double), ("atol_T", ctypes.c_double),
                ("h0", ctypes.c_double), ("max_steps", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        L = ctypes.c_long
        d = ctypes.c_double
        _lib.om_props.argtypes = [vp, L, L, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.om_rates.argtypes = [vp, d, d, vp, vp, vp]
        _lib.om_rate_constants.argtypes = [vp, d, d, vp, vp, vp]
        _lib.om_rhs.argtypes = [vp, d, vp, vp]
        _lib.om_jac.argtypes = [vp, d, vp, vp]
        _lib.om_species_thermo.argtypes = [vp, ctypes.c_int, d, vp, vp, vp, vp]
        _lib.om_integrate_cell.argtypes = [vp, d, d, vp, vp, vp]
        _lib.om_integrate_cell.restype = ctypes.c_int
        _lib.om_step_stiff.argtypes = [vp, L, L, d, vp, vp, vp, vp, vp, vp]
        _lib.om_rodas3_fixed.argtypes = [vp, d, d, ctypes.c_int, vp]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMech:
    """Keeps contiguous copies of a synth.Mech's arrays alive for the C oracle."""

    def __init__(self, mech):
        from paper_2312_05800_gb300 import synth
        self.mech = mech
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self._keep = dict(W=f(mech.W), nasa_lo=f(mech.nasa_lo), nasa_hi=f(mech.nasa_hi),
                          visc_fit=f(mech.visc_fit), diff_fit=f(mech.diff_fit), rtype=i(mech.rtype),
                          reac=i(mech.reac), prod=i(mech.prod), A=f(mech.A), beta=f(mech.beta), Ea=f(mech.Ea),
                          A0=f(mech.A0), beta0=f(mech.beta0), Ea0=f(mech.Ea0), troe=f(mech.troe), eff=f(mech.eff))
        self.s = _Mech(N=mech.N, R=mech.R, E=len(mech.elements), bath=mech.bath, P_std=synth.P_STD,
                       T_lo=synth.T_LO, T_mid=synth.T_MID, T_hi=synth.T_HI,
                       **{k: v.ctypes.data for k, v in self._keep.items()})
        self.N = mech.N
        self.R = mech.R

    @property
    def ref(self):
        return ctypes.byref(self.s)


_OM_CACHE = {}


def omech(mech) -> OracleMech:
    key = id(mech)
    if key not in _OM_CACHE:
        _OM_CACHE[key] = OracleMech(mech)
    return _OM_CACHE[key]


# ---------------------------------------------------------------------------
# thermo / transport
# ---------------------------------------------------------------------------

def species_thermo(mech, k: int, T: float):
    """(cp/R, H/RT, S/R, d(cp/R)/dT) of species k at T (NASA-7)."""
    om = omech(mech)
    out = [ctypes.c_double() for _ in range(4)]
    lib().om_species_thermo(om.ref, k, float(T), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def props(mech, T, p, Y, ncells=None):
    """Mixture cp (J/kg/K), h (J/kg), mu (Pa s), lambda (W/m/K), D_k (m^2/s, [N, ld]) of SoA cells."""
    om = omech(mech)
    T = np.ascontiguousarray(T, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    ld = T.shape[0]
    n = ld if ncells is None else ncells
    cp = np.zeros(ld); h = np.zeros(ld); mu = np.zeros(ld); lam = np.zeros(ld)
    Dk = np.zeros((mech.N, ld))
    lib().om_props(om.ref, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(cp), _ptr(h), _ptr(mu), _ptr(lam), _ptr(Dk))
    return cp, h, mu, lam, Dk


# ---------------------------------------------------------------------------
# kinetics
# ---------------------------------------------------------------------------

def rates(mech, T: float, p: float, Y):
    """(wdot [N] mol/m^3/s, q [R]) at one state."""
    om = omech(mech)
    Y = np.ascontiguousarray(Y, np.float64)
    w = np.zeros(mech.N)
    q = np.zeros(mech.R)
    lib().om_rates(om.ref, float(T), float(p), _ptr(Y), _ptr(w), _ptr(q))
    return w, q


def rate_constants(mech, T: float, p: float, Y):
    om = omech(mech)
    Y = np.ascontiguousarray(Y, np.float64)
    kf = np.zeros(mech.R)
    kr = np.zeros(mech.R)
    lib().om_rate_constants(om.ref, float(T), float(p), _ptr(Y), _ptr(kf), _ptr(kr))
    return kf, kr


def rhs(mech, p: float, y):
    om = omech(mech)
    y = np.ascontiguousarray(y, np.float64)
    f = np.zeros(mech.N + 1)
    lib().om_rhs(om.ref, float(p), _ptr(y), _ptr(f))
    return f


def jac(mech, p: float, y):
    om = omech(mech)
    y = np.ascontiguousarray(y, np.float64)
    J = np.zeros((mech.N + 1, mech.N + 1))
    lib().om_jac(om.ref, float(p), _ptr(y), _ptr(J))
    return J


DEFAULT_OPTS = dict(rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=10000)


def _opts(**kw):
    o = dict(DEFAULT_OPTS)
    o.update(kw)
    return _Opts(**o)


def integrate_cell(mech, p: float, dt: float, y0, **opts):
    """One cell over [0, dt]; returns (y, status, nsteps)."""
    om = omech(mech)
    y = np.array(y0, dtype=np.float64)
    ns = ctypes.c_int()
    o = _opts(**opts)
    st = lib().om_integrate_cell(om.ref, float(p), float(dt), ctypes.byref(o), _ptr(y), ctypes.byref(ns))
    return y, st, ns.value


def rodas3_fixed(mech, p: float, dt: float, nsub: int, y0):
    """nsub equal Rodas3 steps without error control (order observation)."""
    om = omech(mech)
    y = np.array(y0, dtype=np.float64)
    lib().om_rodas3_fixed(om.ref, float(p), float(dt), int(nsub), _ptr(y))
    return y


def step_stiff(mech, T, p, Y, dt: float, ncells=None, **opts):
    """Stiff step over SoA cells; returns (T, Y, status, nsteps) as new arrays."""
    om = omech(mech)
    T = np.array(T, dtype=np.float64)
    p = np.ascontiguousarray(p, np.float64)
    Y = np.array(Y, dtype=np.float64)
    ld = T.shape[0]
    n = ld if ncells is None else ncells
    st = np.zeros(ld, np.int32)
    ns = np.zeros(ld, np.int32)
    o = _opts(**opts)
    lib().om_step_stiff(om.ref, n, ld, float(dt), ctypes.byref(o), _ptr(T), _ptr(p), _ptr(Y), _ptr(st), _ptr(ns))
    return T, Y, st, ns
