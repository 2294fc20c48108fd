"""Helpers for the GPU parity tests: device copies of seeded SoA states and a
once-per-session mechanism handle cache."""
import numpy as np

_MECHS = {}


def dev_mech(name):
    from paper_2312_05800_gb300 import binding, synth
    if name not in _MECHS:
        _MECHS[name] = binding.Mech(synth.get_mech(name))
    return _MECHS[name]


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def h_scale(oracle, mech, T, Y, n):
    """sum_k Y_k |h_k| per cell: the scale of the mixture enthalpy, which crosses zero."""
    from paper_2312_05800_gb300 import synth
    s = np.zeros(n)
    for i in range(n):
        for k in range(mech.N):
            s[i] += abs(Y[k, i]) * abs(oracle.species_thermo(mech, k, T[i])[1] * synth.R_GAS * T[i] / mech.W[k])
    return s
