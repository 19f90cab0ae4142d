"""ctypes declarations of the C ABI in ``include/dcdft.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdcdft.so")

DC_OK = 0
DC_FP64, DC_FP32, DC_MIXED = 0, 1, 2
DC_BC_ZERO, DC_BC_PERIODIC = 0, 1
DC_HXC_NONE, DC_HXC_HARTREE_X = 0, 1
ERRORS = {-1: "DC_ERR_ARG", -2: "DC_ERR_CUDA", -3: "DC_ERR_OOM", -4: "DC_ERR_NOCONV", -5: "DC_ERR_TIMEOUT",
          -6: "DC_ERR_NONFINITE", -7: "DC_ERR_STATE"}


class dc_grid_t(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("L", C.c_double * 3)]


class dc_fragments_t(C.Structure):
    _fields_ = [("num_fragment", C.c_int * 3), ("bc", C.c_int), ("nstate_frag", C.c_int)]


class dc_buffers_t(C.Structure):
    _fields_ = [("num_rgrid_buffer", C.c_int * 3)]


class dc_atoms_t(C.Structure):
    _fields_ = [("natom", C.c_int), ("pos", C.POINTER(C.c_double)), ("species", C.POINTER(C.c_int)),
                ("nspecies", C.c_int), ("Z", C.POINTER(C.c_double)), ("sigma_loc", C.POINTER(C.c_double)),
                ("sigma_proj", C.POINTER(C.c_double)), ("D", C.POINTER(C.c_double))]


class dc_params_t(C.Structure):
    _fields_ = [("precision", C.c_int), ("cheb_degree", C.c_int), ("n_pass", C.c_int), ("n_warmup", C.c_int),
                ("hxc", C.c_int), ("kT", C.c_double), ("mix_alpha", C.c_double), ("seed", C.c_uint64),
                ("kerker_q0", C.c_double), ("rank", C.c_int), ("nranks", C.c_int),
                ("xc_fragment", C.c_int), ("xi", C.c_double)]


class dc_layout_t(C.Structure):
    _fields_ = [("nfrag", C.c_int), ("natom", C.c_int), ("npts", C.c_int64), ("psi_elems", C.c_int64),
                ("frag_points", C.c_int64), ("nstates", C.c_int64), ("natom_frag", C.c_int64),
                ("max_norb", C.c_int), ("element_bytes", C.c_int), ("frag_lo", C.c_int), ("frag_hi", C.c_int),
                ("state_lo", C.c_int64), ("state_hi", C.c_int64)]


class dc_stats_t(C.Structure):
    _fields_ = [("E", C.c_double), ("F", C.c_double), ("eband", C.c_double), ("mu", C.c_double),
                ("drho", C.c_double), ("ne", C.c_double), ("step", C.c_int), ("status", C.c_int)]


class DCError(RuntimeError):
    def __init__(self, fn, status, detail):
        super().__init__(f"{fn}: {ERRORS.get(status, status)}: {detail}")
        self.status = status


VP = C.c_void_p
PD = C.POINTER(C.c_double)
PI32 = C.POINTER(C.c_int32)

# name -> (restype, argtypes); the names are those of include/dcdft.h
PROTOTYPES = {
    "dc_init": (C.c_int, [C.POINTER(dc_grid_t), C.POINTER(dc_fragments_t), C.POINTER(dc_buffers_t),
                          C.POINTER(dc_atoms_t), C.POINTER(dc_params_t), C.POINTER(VP)]),
    "dc_finalize": (None, [VP]),
    "dc_error_string": (C.c_char_p, [C.c_int]),
    "dc_last_error": (C.c_char_p, []),
    "dc_query": (C.c_int, [VP, C.POINTER(dc_layout_t)]),
    "dc_get_maps": (C.c_int, [VP, PI32, PI32, PI32, PI32, PI32]),
    "dc_get_initial": (C.c_int, [VP, VP, VP, VP]),
    "dc_potential": (C.c_int, [VP, VP, VP, VP]),
    "dc_set_potential": (C.c_int, [VP, VP, VP]),
    "dc_hpsi": (C.c_int, [VP, VP, VP, C.c_int, VP]),
    "dc_subspace": (C.c_int, [VP, VP, C.c_int, VP, VP]),
    "dc_chefsi": (C.c_int, [VP, C.c_int, VP]),
    "dc_warmup": (C.c_int, [VP, VP]),
    "dc_get_state": (C.c_int, [VP, VP, VP, VP]),
    "dc_set_state": (C.c_int, [VP, VP, VP, VP]),
    "dc_density": (C.c_int, [VP, VP, C.c_int, VP, VP, VP, VP, VP]),
    "dc_step_local": (C.c_int, [VP, VP, VP, VP, VP]),
    "dc_step_density": (C.c_int, [VP, VP, VP, VP, VP, VP]),
    "dc_step_finish": (C.c_int, [VP, VP, VP, C.POINTER(dc_stats_t), VP]),
    "dc_selftest_wait": (C.c_int, [VP, VP]),
    "dc_lcfo_query": (C.c_int, [VP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "dc_lcfo_basis": (C.c_int, [VP, VP, C.c_int, VP, C.c_double, C.c_double, VP, VP, VP, VP]),
    "dc_fermi_level_noalloc": (C.c_int, [VP, VP, C.c_int64, C.c_double, C.c_double, VP, VP, VP]),
    "dc_scf_step": (C.c_int, [VP, VP, C.c_int, C.POINTER(dc_stats_t), VP]),
    "dc_get_rho_out": (C.c_int, [VP, VP, VP]),
    "dc_eb_adjoint": (C.c_int, [VP, VP, C.c_int, VP, VP, VP, PD, VP, VP, VP, VP]),
    "dc_tuning": (C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "dc_set_tuning": (C.c_int, [VP, C.c_int, C.c_int, C.c_int, C.c_int]),
    "dc_profile": (C.c_int, [VP, C.c_int]),
    "dc_profile_read": (C.c_int, [VP, PD, C.POINTER(C.c_int64), PD]),
    "dc_fp64_fma_probe": (C.c_int, [C.c_int64, VP, C.POINTER(C.c_int64), VP]),
}

STAGES = ["potential", "gather", "project", "hpsi", "gram", "subspace", "rotate", "density", "energy"]

_lib = None


def load():
    """Load libdcdft.so (built in-tree).  Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"native library {LIB_PATH} is missing; run paper_2606_21125_b300/build.py")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(fn_name, status):
    if status != DC_OK:
        detail = load().dc_last_error().decode(errors="replace")
        raise DCError(fn_name, status, detail)
    return status
