"""The C-ABI library loads and exports every entry point its header declares (CPU only).

No compute call is made here; only calls that return before touching the device (argument
validation, error strings) are exercised.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dcdft.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_21125_b300 import build, load
    build.build()
    return load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dc_init", "dc_hpsi", "dc_subspace", "dc_chefsi", "dc_density", "dc_scf_step",
                     "dc_eb_adjoint", "dc_finalize", "dc_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2606_21125_b300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dc_[a-z_0-9]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)
        assert n in _lib.PROTOTYPES, f"binding lacks a prototype for {n}"


def test_error_strings(lib):
    assert lib.dc_error_string(0) == b"DC_OK"
    assert lib.dc_error_string(-4) == b"DC_ERR_NOCONV"
    assert lib.dc_error_string(-5) == b"DC_ERR_TIMEOUT"
    assert lib.dc_error_string(123) == b"DC_ERR_UNKNOWN"


def _structs(n=(10, 10, 10), F=(2, 2, 2), b=(2, 2, 2), prec=0, kT=0.01, cheb=8):
    from paper_2606_21125_b300 import _lib
    import numpy as np
    g = _lib.dc_grid_t((C.c_int * 3)(*n), (C.c_double * 3)(6.0, 6.0, 6.0))
    fr = _lib.dc_fragments_t((C.c_int * 3)(*F), 0, 4)
    bu = _lib.dc_buffers_t((C.c_int * 3)(*b))
    keep = [np.zeros(3), np.zeros(1, dtype=np.int32), np.ones(1), np.ones(1), np.ones(1), np.ones(1)]
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    at = _lib.dc_atoms_t(1, dp(keep[0]), keep[1].ctypes.data_as(C.POINTER(C.c_int)), 1, dp(keep[2]), dp(keep[3]),
                         dp(keep[4]), dp(keep[5]))
    pa = _lib.dc_params_t(prec, cheb, 1, 0, 1, kT, 0.3, 1)
    return g, fr, bu, at, pa, keep


@pytest.mark.parametrize("bad", ["null", "kT", "precision", "fragments", "cheb", "xc_fragment_no_hxc", "xi",
                                 "xc_fragment_value", "rank", "nranks"])
def test_invalid_configuration_is_rejected_before_device_work(lib, bad):
    """dc_init validates its arguments on the host and returns DC_ERR_ARG with a message."""
    kw = {}
    if bad == "kT":
        kw["kT"] = 0.0
    elif bad == "precision":
        kw["prec"] = 7
    elif bad == "fragments":
        kw["F"] = (11, 2, 2)
    elif bad == "cheb":
        kw["cheb"] = 0
    g, fr, bu, at, pa, keep = _structs(**kw)
    if bad == "xc_fragment_no_hxc":
        pa.xc_fragment, pa.hxc = 1, 0
    elif bad == "xi":
        pa.xi = -1.0
    elif bad == "xc_fragment_value":
        pa.xc_fragment = 2
    elif bad == "rank":
        pa.rank, pa.nranks = 2, 2
    elif bad == "nranks":
        pa.nranks = 9  # more ranks than the 8 fragments
    ctx = C.c_void_p(123)
    if bad == "null":
        st = lib.dc_init(C.byref(g), None, C.byref(bu), C.byref(at), C.byref(pa), C.byref(ctx))
    else:
        st = lib.dc_init(C.byref(g), C.byref(fr), C.byref(bu), C.byref(at), C.byref(pa), C.byref(ctx))
    assert st == -1
    assert not ctx.value
    assert len(lib.dc_last_error()) > 0


def test_null_context_calls_fail_cleanly(lib):
    assert lib.dc_query(None, None) == -1
    assert lib.dc_hpsi(None, None, None, 0, None) == -1
    assert lib.dc_scf_step(None, None, 0, None, None) == -1
    lib.dc_finalize(None)
