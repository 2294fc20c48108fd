"""ctypes binding of libchemgb.so: argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; device arrays are passed as raw pointers taken from
torch CUDA tensors (or integers). The library must be built first
(``paper_2312_05800_gb300.build.build()``); if it is missing, importing
this module's functions raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

from . import build as _build

CHEM_OK, CHEM_EINVAL, CHEM_ECUDA, CHEM_EUNSUPPORTED, CHEM_EIO = 0, -1, -2, -3, -4
CHEM_F32, CHEM_F64, CHEM_F64_IN_F32 = 0, 1, 2
CELL_OK, CELL_FALLBACK, CELL_MAXSTEPS, CELL_UNDERFLOW, CELL_NONFINITE = 0, 1, 2, 3, 4

_lib = None


class ChemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("chemgb error %d: %s" % (code, msg))
        self.code = code


class chem_ode_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol_Y", ctypes.c_double), ("atol_T", ctypes.c_double),
                ("h0", ctypes.c_double), ("max_steps", ctypes.c_int32), ("_pad", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Loads libchemgb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("libchemgb.so is not built (%s); run paper_2312_05800_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.chem_mech_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
    L.chem_mech_load_bytes.argtypes = [vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.chem_mech_free.argtypes = [vp]
    L.chem_mech_nspecies.argtypes = [vp]
    L.chem_mech_nreactions.argtypes = [vp]
    L.props_eval.argtypes = [vp, i64, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.chem_ode_opts_default.argtypes = [ctypes.POINTER(chem_ode_opts)]
    L.chem_ode_opts_default.restype = None
    L.chem_step_stiff.argtypes = [vp, i64, i64, d, ctypes.POINTER(chem_ode_opts), vp, vp, vp, vp, vp, vp]
    L.chem_step_stiff_noalloc.argtypes = [vp, i64, i64, d, ctypes.POINTER(chem_ode_opts), vp, vp, vp, vp, vp, vp]
    L.chem_last_error.restype = ctypes.c_char_p
    L.chem_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int):
    if rc != CHEM_OK:
        raise ChemError(rc, lib().chem_last_error().decode())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("device arrays must be CUDA tensors")
        if not x.is_contiguous():
            raise ValueError("device arrays must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a torch CUDA tensor or an integer pointer")


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Mech:
    """Library-owned mechanism handle (chem_mech_load / chem_mech_load_bytes)."""

    def __init__(self, source):
        h = ctypes.c_void_p()
        if isinstance(source, (bytes, bytearray)):
            buf = ctypes.create_string_buffer(bytes(source), len(source))
            _check(lib().chem_mech_load_bytes(buf, len(source), ctypes.byref(h)))
        elif isinstance(source, str):
            _check(lib().chem_mech_load(source.encode(), ctypes.byref(h)))
        else:   # a synth.Mech
            from . import synth
            data = synth.mech_to_bytes(source)
            buf = ctypes.create_string_buffer(data, len(data))
            _check(lib().chem_mech_load_bytes(buf, len(data), ctypes.byref(h)))
        self.handle = h.value
        self.N = lib().chem_mech_nspecies(self.handle)
        self.R = lib().chem_mech_nreactions(self.handle)

    def free(self):
        if self.handle:
            _check(lib().chem_mech_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def chem_mech_load(path: str) -> Mech:
    return Mech(path)


def chem_ode_opts_default() -> chem_ode_opts:
    o = chem_ode_opts()
    lib().chem_ode_opts_default(ctypes.byref(o))
    return o


def make_opts(**kw) -> chem_ode_opts:
    o = chem_ode_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def props_eval(mech: Mech, ncells: int, ld: int, dtype: int, T, p, Y, cp=None, h=None, mu=None, lam=None,
               Dk=None, stream=None):
    _check(lib().props_eval(mech.handle, ncells, ld, dtype, _ptr(T), _ptr(p), _ptr(Y), _ptr(cp), _ptr(h), _ptr(mu),
                            _ptr(lam), _ptr(Dk), _stream(stream)))


def chem_step_stiff(mech: Mech, ncells: int, ld: int, dt: float, opts: Optional[chem_ode_opts], T, p, Y, status,
                    nsteps=None, stream=None):
    _check(lib().chem_step_stiff(mech.handle, ncells, ld, float(dt), ctypes.byref(opts) if opts is not None else None,
                                 _ptr(T), _ptr(p), _ptr(Y), _ptr(status), _ptr(nsteps), _stream(stream)))


def chem_step_stiff_noalloc(mech: Mech, ncells: int, ld: int, dt: float, opts: Optional[chem_ode_opts], T, p, Y,
                            status, nsteps=None, stream=None):
    _check(lib().chem_step_stiff_noalloc(mech.handle, ncells, ld, float(dt),
                                         ctypes.byref(opts) if opts is not None else None, _ptr(T), _ptr(p), _ptr(Y),
                                         _ptr(status), _ptr(nsteps), _stream(stream)))


def chem_last_error() -> str:
    return lib().chem_last_error().decode()


def chem_version() -> str:
    return lib().chem_version().decode()
