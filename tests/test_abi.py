"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                                src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2312_05800_gb300 import build
    return build.build()


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("props_eval", "chem_step_stiff", "chem_mech_load", "chem_last_error"):
        assert must in names, names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_compute_calls_fail_loudly_without_a_gpu(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2312_05800_gb300 import binding, synth
    with pytest.raises(binding.ChemError) as e:
        binding.Mech(synth.mech_c1())
    assert e.value.code in (binding.CHEM_EUNSUPPORTED, binding.CHEM_ECUDA)


def test_bad_arguments_are_rejected_before_any_device_work(libpath):
    from paper_2312_05800_gb300 import binding
    L = binding.lib()
    assert L.props_eval(None, 10, 12, 0, None, None, None, None, None, None, None, None, None) == binding.CHEM_EINVAL
    h = ctypes.c_void_p()
    assert L.chem_mech_load_bytes(b"XXXXXXXX", 8, ctypes.byref(h)) == binding.CHEM_EIO
    assert "magic" in binding.chem_last_error()


def test_host_defaults_fill_the_structs_the_binding_declares(libpath):
    """The two host-only default calls write exactly the ctypes layouts of the binding: the header's
    documented values land in the right fields, and bytes past the end of each struct stay untouched
    (a C struct larger than its ctypes twin would overwrite them)."""
    from paper_2312_05800_gb300 import binding
    L = ctypes.CDLL(libpath)
    for cls, fn in ((binding.chem_ode_opts, L.chem_ode_opts_default),
                    (binding.chem_hfrd_params, L.chem_hfrd_params_default)):
        size = ctypes.sizeof(cls)
        buf = (ctypes.c_ubyte * (size + 64))(*([0xA5] * (size + 64)))
        fn.restype = None
        fn(ctypes.byref(buf))
        assert bytes(buf[size:]) == b"\xa5" * 64, cls.__name__
    o = binding.chem_ode_opts()
    L.chem_ode_opts_default(ctypes.byref(o))
    # chem_ode_opts' documented defaults
    assert (o.rtol, o.atol_Y, o.atol_T, o.h0, o.max_steps, o.mode) == (1e-6, 1e-12, 1e-6, 1e-9, 10000, 0)


def test_binding_calls_every_declared_entry_point():
    """The Python binding has a call for every entry point the header declares (no C function is
    reachable only from C)."""
    src = open(os.path.join(ROOT, "paper_2312_05800_gb300", "binding.py")).read()
    missing = [n for n in _declared() if ("lib()." + n) not in src and ("L." + n) not in src]
    assert not missing, missing
