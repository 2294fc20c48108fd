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

import numpy as np

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
                ("h0", ctypes.c_double), ("max_steps", ctypes.c_int32), ("mode", ctypes.c_int32)]


CHEM_ODE_FP64, CHEM_ODE_MIXED = 0, 1


class chem_mlp_desc(ctypes.Structure):
    _fields_ = [("n_hidden", ctypes.c_int32 * 3), ("chunk", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("ensemble", ctypes.c_int32), ("dt", ctypes.c_double)]


class chem_hfrd_params(ctypes.Structure):
    _fields_ = [(nm, ctypes.c_double) for nm in ("alpha", "beta", "gamma", "T_min", "T_max", "p_min", "p_max",
                                                 "Yb_min", "Yb_max", "hc_lo", "hc_hi", "on_lo", "on_hi", "phi_lo",
                                                 "phi_hi")]


CHEM_PREC_BF16, CHEM_PREC_FP8 = 0, 1
CHEM_FUSE_34 = 2


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
    L.chem_pasr.argtypes = [vp, i64, i64, d, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.chem_hfrd_params_default.argtypes = [ctypes.POINTER(chem_hfrd_params)]
    L.chem_hfrd_params_default.restype = None
    L.chem_hfrd_perturb.argtypes = [vp, ctypes.POINTER(chem_hfrd_params), vp, i64, i64, vp, vp, vp, vp, vp, vp, vp,
                                    vp, vp]
    L.chem_hfrd_blend.argtypes = [i32, i64, i64, vp, d, vp, d, vp, vp, vp, vp]
    L.chem_dense_bf16.argtypes = [i64, i32, i32, vp, i64, vp, i64, vp, i32, vp, i64, i32, vp, vp]
    L.chem_mlp_create.argtypes = [vp, ctypes.POINTER(chem_mlp_desc), ctypes.c_uint64, ctypes.POINTER(vp)]
    L.chem_mlp_free.argtypes = [vp]
    L.chem_mlp_dims.argtypes = [vp, vp]
    L.chem_mlp_groups.argtypes = [vp]
    L.chem_mlp_nparams.argtypes = [vp]
    L.chem_mlp_nparams.restype = ctypes.c_int64
    L.chem_mlp_set_params.argtypes = [vp, vp]
    L.chem_mlp_get_params.argtypes = [vp, vp]
    L.chem_mlp_get_grads.argtypes = [vp, vp]
    L.chem_mlp_set_norm.argtypes = [vp, vp, vp, vp, vp]
    L.chem_mlp_get_norm.argtypes = [vp, vp, vp, vp, vp]
    L.chem_mlp_fit_norm.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp]
    L.chem_mlp_forward.argtypes = [vp, i64, i64, vp, vp, vp, vp, i64, vp]
    L.chem_mlp_forward_prec.argtypes = [vp, i32, i64, i64, vp, vp, vp, vp, i64, vp]
    L.chem_mlp_set_fp8_scales.argtypes = [vp, vp]
    L.chem_mlp_get_fp8_scales.argtypes = [vp, vp]
    L.chem_mlp_calibrate_fp8.argtypes = [vp, i64, i64, vp, vp, vp, vp]
    L.chem_mlp_get_fp8_weights.argtypes = [vp, i32, vp, vp]
    L.chem_mlp_error.argtypes = [vp, vp]
    L.chem_mlp_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
    L.chem_mlp_set_fusion.argtypes = [vp, i32]
    L.chem_mlp_set_physics_loss.argtypes = [vp, d, d, d, d]
    L.chem_mlp_fit_physics_scales.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.chem_mlp_get_fusion.argtypes = [vp]
    L.chem_mlp_fit_ood.argtypes = [vp, vp, i64, i64, vp, vp, vp, i32, i32, i32, vp]
    L.chem_mlp_fit_ood_multi.argtypes = [vp, vp, i64, i64, vp, vp, vp, vp, i32, i32, i32, vp]
    L.chem_mlp_get_ood_grid.argtypes = [vp, i32, vp, vp, vp]
    L.chem_mlp_set_ood.argtypes = [vp, i32]
    L.chem_mlp_ood_flags.argtypes = [vp, vp, i64, i64, vp, vp, vp, vp, vp]
    L.chem_mlp_get_ood.argtypes = [vp, vp, vp, vp, vp, vp]
    L.chem_mlp_autotune.argtypes = [vp, i64, vp, vp]
    L.chem_mlp_save.argtypes = [vp, ctypes.c_char_p]
    L.chem_mlp_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(vp)]
    L.chem_step_ann.argtypes = [vp, vp, i64, i64, d, i32, ctypes.POINTER(chem_ode_opts), vp, vp, vp, vp, vp]
    L.chem_step_ann_props.argtypes = [vp, vp, i64, i64, d, i32, ctypes.POINTER(chem_ode_opts), vp, vp, vp, vp,
                                      vp, vp, vp, vp, vp, vp]
    L.mlp_train_step.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, ctypes.c_float, vp, vp]
    L.mlp_train_grads.argtypes = [vp, i64, vp, i64, vp, vp, vp, vp, vp, vp]
    L.mlp_adam_step.argtypes = [vp, ctypes.c_float, vp]
    L.chem_mlp_grad_buffers.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]
    L.chem_prof_enable.argtypes = [i32]
    L.chem_prof_read.argtypes = [ctypes.c_char_p, i64]
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


def chem_dense_bf16(M: int, N: int, K: int, x, ldx: int, W, ldw: int, b, act: int, y, ldy: int, tile_n: int = 0,
                    err=None, stream=None):
    _check(lib().chem_dense_bf16(M, N, K, _ptr(x), ldx, _ptr(W), ldw, _ptr(b), act, _ptr(y), ldy, tile_n, _ptr(err),
                                 _stream(stream)))


def hfrd_params(**kw) -> chem_hfrd_params:
    """chem_hfrd_params with the paper's defaults, then the given fields."""
    q = chem_hfrd_params()
    lib().chem_hfrd_params_default(ctypes.byref(q))
    for k, v in kw.items():
        setattr(q, k, float(v))
    return q


def chem_hfrd_perturb(mech: Mech, params: chem_hfrd_params, chon, n: int, ld: int, T, p, Y, c, T2, p2, Y2, keep,
                      stream=None):
    a = np.ascontiguousarray(chon, dtype=np.int32)
    _check(lib().chem_hfrd_perturb(mech.handle, ctypes.byref(params), a.ctypes.data_as(ctypes.c_void_p), n, ld,
                                   _ptr(T), _ptr(p), _ptr(Y), _ptr(c), _ptr(T2), _ptr(p2), _ptr(Y2), _ptr(keep),
                                   _stream(stream)))


def chem_hfrd_blend(N: int, n: int, ld: int, s, Ta: float, Ya, Tb: float, Yb, T, Y, stream=None):
    ya = np.ascontiguousarray(Ya, dtype=np.float64)
    yb = np.ascontiguousarray(Yb, dtype=np.float64)
    _check(lib().chem_hfrd_blend(N, n, ld, _ptr(s), float(Ta), ya.ctypes.data_as(ctypes.c_void_p), float(Tb),
                                 yb.ctypes.data_as(ctypes.c_void_p), _ptr(T), _ptr(Y), _stream(stream)))


def chem_pasr(mech: Mech, ncells: int, ld: int, y_min: float, T0, p, Y0, tau_taylor, tau_kolmogorov, T=None, Y=None,
              tau_c=None, kappa=None, stream=None):
    _check(lib().chem_pasr(mech.handle, ncells, ld, float(y_min), _ptr(T0), _ptr(p), _ptr(Y0), _ptr(tau_taylor),
                           _ptr(tau_kolmogorov), _ptr(T), _ptr(Y), _ptr(tau_c), _ptr(kappa), _stream(stream)))


class Mlp:
    """Library-owned network handle (chem_mlp_create / chem_mlp_free)."""

    def __init__(self, mech: Mech, hidden=(1600, 800, 400), dt=1e-6, seed=0, chunk=0, max_batch=0, ensemble=False):
        d = chem_mlp_desc()
        for i in range(3):
            d.n_hidden[i] = int(hidden[i])
        d.chunk, d.max_batch, d.dt, d.ensemble = int(chunk), int(max_batch), float(dt), int(bool(ensemble))
        h = ctypes.c_void_p()
        _check(lib().chem_mlp_create(mech.handle, ctypes.byref(d), ctypes.c_uint64(seed), ctypes.byref(h)))
        self.handle = h.value
        self._describe()

    def _describe(self):
        import numpy as np
        w = np.zeros(5, np.int32)
        _check(lib().chem_mlp_dims(self.handle, w.ctypes.data))
        self.widths = [int(v) for v in w]
        self.nparams = int(lib().chem_mlp_nparams(self.handle))
        self.groups = int(lib().chem_mlp_groups(self.handle))
        self.ensemble = self.groups > 1

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        _check(lib().chem_mlp_set_params(self.handle, a.ctypes.data))

    def get_params(self):
        import numpy as np
        a = np.zeros(self.nparams, np.float32)
        _check(lib().chem_mlp_get_params(self.handle, a.ctypes.data))
        return a

    def get_grads(self):
        import numpy as np
        a = np.zeros(self.nparams, np.float32)
        _check(lib().chem_mlp_get_grads(self.handle, a.ctypes.data))
        return a

    def set_norm(self, mu_x, sd_x, mu_u, sd_u):
        import numpy as np
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (mu_x, sd_x, mu_u, sd_u)]
        _check(lib().chem_mlp_set_norm(self.handle, *[a.ctypes.data for a in arrs]))

    def get_norm(self):
        import numpy as np
        nin, nout = self.widths[0], self.widths[4]
        arrs = [np.zeros(nin), np.zeros(nin), np.zeros(nout), np.zeros(nout)]
        _check(lib().chem_mlp_get_norm(self.handle, *[a.ctypes.data for a in arrs]))
        return arrs

    def save(self, path: str):
        _check(lib().chem_mlp_save(self.handle, path.encode()))

    @classmethod
    def load(cls, mech: Mech, path: str) -> "Mlp":
        h = ctypes.c_void_p()
        _check(lib().chem_mlp_load(mech.handle, path.encode(), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.handle = h.value
        self._describe()
        return self

    def error(self) -> int:
        e = ctypes.c_int()
        _check(lib().chem_mlp_error(self.handle, ctypes.byref(e)))
        return e.value

    def set_wait_limit(self, tries: int):
        _check(lib().chem_mlp_set_wait_limit(self.handle, int(tries)))

    def set_physics_loss(self, lam_m: float, lam_q: float, s_m: float = 1.0, s_q: float = 1.0):
        _check(lib().chem_mlp_set_physics_loss(self.handle, float(lam_m), float(lam_q), float(s_m), float(s_q)))

    def fit_physics_scales(self, n: int, ld: int, T, Y, Y1, stream=None):
        sm, sq = ctypes.c_double(), ctypes.c_double()
        _check(lib().chem_mlp_fit_physics_scales(self.handle, n, ld, _ptr(T), _ptr(Y), _ptr(Y1), ctypes.byref(sm),
                                                 ctypes.byref(sq), _stream(stream)))
        return sm.value, sq.value

    def set_fusion(self, mask):
        """0 or CHEM_FUSE_34 (True: CHEM_FUSE_34, False: none)."""
        if mask is True:
            mask = CHEM_FUSE_34
        elif mask is False:
            mask = 0
        _check(lib().chem_mlp_set_fusion(self.handle, int(mask)))

    @property
    def fusion(self) -> int:
        r = lib().chem_mlp_get_fusion(self.handle)
        if r < 0:
            _check(r)
        return r

    @property
    def fused(self) -> bool:
        return self.fusion != 0

    def free(self):
        if self.handle:
            _check(lib().chem_mlp_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def chem_mlp_fit_ood(mlp: Mlp, mech: Mech, n: int, ld: int, T, p, Y, species: int, nbins: int = 64,
                     min_count: int = 4, stream=None):
    _check(lib().chem_mlp_fit_ood(mlp.handle, mech.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), species, nbins,
                                  min_count, _stream(stream)))


def chem_mlp_fit_ood_multi(mlp: Mlp, mech: Mech, n: int, ld: int, T, p, Y, species, nbins: int = 64,
                           min_count: int = 4, stream=None):
    import numpy as np
    sp = np.ascontiguousarray(species, dtype=np.int32)
    _check(lib().chem_mlp_fit_ood_multi(mlp.handle, mech.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), sp.ctypes.data,
                                        int(sp.size), nbins, min_count, _stream(stream)))


def chem_mlp_get_ood_grid(mlp: Mlp, grid: int):
    import numpy as np
    lo, hi = np.zeros(3, np.float32), np.zeros(3, np.float32)
    sp = ctypes.c_int32()
    _check(lib().chem_mlp_get_ood_grid(mlp.handle, grid, lo.ctypes.data, hi.ctypes.data, ctypes.byref(sp)))
    return lo, hi, sp.value


def chem_mlp_set_ood(mlp: Mlp, enable: bool):
    _check(lib().chem_mlp_set_ood(mlp.handle, 1 if enable else 0))


def chem_mlp_ood_flags(mlp: Mlp, mech: Mech, ncells: int, ld: int, T, p, Y, flags, stream=None):
    _check(lib().chem_mlp_ood_flags(mlp.handle, mech.handle, ncells, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(flags),
                                    _stream(stream)))


def chem_mlp_get_ood(mlp: Mlp):
    import numpy as np
    lo, hi = np.zeros(3, np.float32), np.zeros(3, np.float32)
    nb, sp, km = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().chem_mlp_get_ood(mlp.handle, lo.ctypes.data, hi.ctypes.data, ctypes.byref(nb), ctypes.byref(sp),
                                  ctypes.byref(km)))
    return lo, hi, nb.value, sp.value, km.value


def chem_mlp_autotune(mlp: Mlp, rows: int = 262144, stream=None):
    import numpy as np
    t = np.zeros(4, np.int32)
    _check(lib().chem_mlp_autotune(mlp.handle, rows, t.ctypes.data, _stream(stream)))
    return [int(v) for v in t]


def chem_mlp_fit_norm(mlp: Mlp, n: int, ld: int, T, p, Y, Y1, stream=None):
    _check(lib().chem_mlp_fit_norm(mlp.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(Y1), _stream(stream)))


def chem_mlp_forward(mlp: Mlp, ncells: int, ld: int, T, p, Y, u, ldu: int, stream=None):
    _check(lib().chem_mlp_forward(mlp.handle, ncells, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(u), ldu, _stream(stream)))


def chem_mlp_forward_prec(mlp: Mlp, prec: int, ncells: int, ld: int, T, p, Y, u, ldu: int, stream=None):
    _check(lib().chem_mlp_forward_prec(mlp.handle, prec, ncells, ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(u), ldu,
                                       _stream(stream)))


def chem_mlp_set_fp8_scales(mlp: Mlp, scales):
    import numpy as np
    a = np.ascontiguousarray(scales, dtype=np.float32)
    assert a.size == 2
    _check(lib().chem_mlp_set_fp8_scales(mlp.handle, a.ctypes.data))


def chem_mlp_get_fp8_scales(mlp: Mlp):
    import numpy as np
    a = np.zeros(2, np.float32)
    _check(lib().chem_mlp_get_fp8_scales(mlp.handle, a.ctypes.data))
    return a


def chem_mlp_calibrate_fp8(mlp: Mlp, n: int, ld: int, T, p, Y, stream=None):
    _check(lib().chem_mlp_calibrate_fp8(mlp.handle, n, ld, _ptr(T), _ptr(p), _ptr(Y), _stream(stream)))


def chem_mlp_get_fp8_weights(mlp: Mlp, layer: int):
    """(Wq [out][in] uint8 E4M3 codes, sw [out] float32) of hidden-to-hidden layer 1 or 2."""
    import numpy as np
    fo, fi = mlp.widths[layer + 1], mlp.widths[layer]
    Wq = np.zeros((fo, fi), np.uint8)
    sw = np.zeros(fo, np.float32)
    _check(lib().chem_mlp_get_fp8_weights(mlp.handle, layer, Wq.ctypes.data, sw.ctypes.data))
    return Wq, sw


def chem_step_ann(mech: Mech, mlp: Mlp, ncells: int, ld: int, dt: float, prec: int, fallback, T, p, Y, status=None,
                  stream=None):
    _check(lib().chem_step_ann(mech.handle, mlp.handle, ncells, ld, float(dt), prec,
                               ctypes.byref(fallback) if fallback is not None else None, _ptr(T), _ptr(p), _ptr(Y),
                               _ptr(status), _stream(stream)))


def chem_step_ann_props(mech: Mech, mlp: Mlp, ncells: int, ld: int, dt: float, prec: int, fallback, T, p, Y,
                        status=None, cp=None, h=None, mu=None, lam=None, Dk=None, stream=None):
    _check(lib().chem_step_ann_props(mech.handle, mlp.handle, ncells, ld, float(dt), prec,
                                     ctypes.byref(fallback) if fallback is not None else None, _ptr(T), _ptr(p),
                                     _ptr(Y), _ptr(status), _ptr(cp), _ptr(h), _ptr(mu), _ptr(lam), _ptr(Dk),
                                     _stream(stream)))


def mlp_train_step(mlp: Mlp, batch: int, idx, ld: int, T, p, Y, Y1, lr: float, loss=None, stream=None):
    _check(lib().mlp_train_step(mlp.handle, batch, _ptr(idx), ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(Y1),
                                ctypes.c_float(lr), _ptr(loss), _stream(stream)))


def mlp_train_grads(mlp: Mlp, batch: int, idx, ld: int, T, p, Y, Y1, loss=None, stream=None):
    """The forward, loss and back-propagation of mlp_train_step: the batch's gradients in the handle."""
    _check(lib().mlp_train_grads(mlp.handle, batch, _ptr(idx), ld, _ptr(T), _ptr(p), _ptr(Y), _ptr(Y1), _ptr(loss),
                                 _stream(stream)))


def mlp_adam_step(mlp: Mlp, lr: float, stream=None):
    """The Adam update of mlp_train_step from the handle's current gradients."""
    _check(lib().mlp_adam_step(mlp.handle, ctypes.c_float(lr), _stream(stream)))


class _DeviceF32:
    """A float32 device array at a library-owned address (__cuda_array_interface__, no copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False), "version": 3,
                                         "strides": None}


def grad_buffers(mlp: Mlp):
    """The handle's gradient buffers as float32 CUDA tensors aliasing its memory, layer by layer
    [gW_0, gb_0, ..., gW_3, gb_3]: a collective may reduce them in place between mlp_train_grads and
    mlp_adam_step."""
    import torch
    out = []
    for layer in range(4):
        gw, nw, gb, nb = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_int64()
        _check(lib().chem_mlp_grad_buffers(mlp.handle, layer, ctypes.byref(gw), ctypes.byref(nw), ctypes.byref(gb),
                                           ctypes.byref(nb)))
        out.append(torch.as_tensor(_DeviceF32(gw.value, nw.value), device="cuda"))
        out.append(torch.as_tensor(_DeviceF32(gb.value, nb.value), device="cuda"))
    return out


def chem_prof_enable(on: bool):
    _check(lib().chem_prof_enable(1 if on else 0))


def chem_prof_read():
    """{tag: (launches, ms, flops, bytes)} accumulated since chem_prof_enable."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().chem_prof_read(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        tag, n, ms, fl, by = line.split("\t")
        out[tag] = (int(n), float(ms), float(fl), float(by))
    return out


def chem_last_error() -> str:
    return lib().chem_last_error().decode()


def chem_version() -> str:
    return lib().chem_version().decode()
