"""B300-native divide-and-conquer DFT fragment solver (Python binding).

The compute path is the native library ``libdcdft.so`` (C ABI declared in ``include/dcdft.h``);
this module only marshals arguments.  PyTorch provides device memory and streams.  There is no
CPU fallback: if the library is missing, importing ``DCSolver`` works but constructing one raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (DC_BC_PERIODIC, DC_BC_ZERO, DC_FP32, DC_FP64, DC_HXC_HARTREE_X, DC_HXC_NONE, DC_MIXED,
                   DCError, check, load)

__all__ = ["DCSolver", "Eb", "DCError", "load", "fermi_level_noalloc", "DC_FP64", "DC_FP32", "DC_MIXED"]

PRECISIONS = {"fp64": DC_FP64, "fp32": DC_FP32, "mixed": DC_MIXED}
BCS = {"zero": DC_BC_ZERO, "periodic": DC_BC_PERIODIC}
HXCS = {"none": DC_HXC_NONE, "hartree_x": DC_HXC_HARTREE_X}


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


class DCSolver:
    """One DC-DFT system on the current CUDA device (a ``dc_ctx``).

    ``cfg`` uses the keys of the workload generator: n, L, num_fragment, num_rgrid_buffer,
    nstate_frag, bc, pos, species, spec (Z, sigma_loc, sigma_proj, D), precision, cheb_degree,
    n_pass, n_warmup, hxc, kT, mix_alpha, seed.
    """

    def __init__(self, cfg):
        lib = load()
        self.lib = lib
        self.cfg = cfg
        g = _lib.dc_grid_t((C.c_int * 3)(*cfg["n"]), (C.c_double * 3)(*cfg["L"]))
        fr = _lib.dc_fragments_t((C.c_int * 3)(*cfg["num_fragment"]), BCS[cfg["bc"]], int(cfg["nstate_frag"]))
        bu = _lib.dc_buffers_t((C.c_int * 3)(*cfg["num_rgrid_buffer"]))
        self._pos = np.ascontiguousarray(np.asarray(cfg["pos"], dtype=np.float64).reshape(-1))
        self._spc = np.ascontiguousarray(np.asarray(cfg["species"], dtype=np.int32))
        sp = cfg["spec"]
        self._tabs = [np.ascontiguousarray(np.asarray(sp[k], dtype=np.float64)) for k in ("Z", "sigma_loc",
                                                                                         "sigma_proj", "D")]
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        at = _lib.dc_atoms_t(len(self._spc), dp(self._pos), self._spc.ctypes.data_as(C.POINTER(C.c_int)),
                             len(self._tabs[0]), *[dp(t) for t in self._tabs])
        self.precision = PRECISIONS[cfg["precision"]]
        pa = _lib.dc_params_t(self.precision, int(cfg["cheb_degree"]), int(cfg["n_pass"]), int(cfg["n_warmup"]),
                              HXCS[cfg["hxc"]], float(cfg["kT"]), float(cfg["mix_alpha"]), int(cfg["seed"]),
                              float(cfg.get("kerker_q0", 0.0)), int(cfg.get("rank", 0)),
                              int(cfg.get("nranks", 1)), int(bool(cfg.get("xc_fragment", False))),
                              float(cfg.get("xi", 0.0)))
        ctx = C.c_void_p()
        check("dc_init", lib.dc_init(C.byref(g), C.byref(fr), C.byref(bu), C.byref(at), C.byref(pa), C.byref(ctx)))
        self.ctx = ctx
        lay = _lib.dc_layout_t()
        check("dc_query", lib.dc_query(self.ctx, C.byref(lay)))
        self.layout = lay
        self.shape = (int(cfg["n"][2]), int(cfg["n"][1]), int(cfg["n"][0]))
        torch = _torch()
        self.dtype = torch.float64 if self.precision == DC_FP64 else torch.float32

    # ---- lifecycle ------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dc_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- maps ------------------------------------------------------------------------------
    def maps(self):
        L = self.layout
        frag = np.zeros((L.nfrag, 12), dtype=np.int32)
        idx = np.zeros(L.frag_points, dtype=np.int32)
        owner = np.zeros(L.npts, dtype=np.int32)
        core = np.zeros(L.npts, dtype=np.int32)
        atoms = np.zeros(max(1, L.natom_frag), dtype=np.int32)
        p = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))  # noqa: E731
        check("dc_get_maps", self.lib.dc_get_maps(self.ctx, p(frag), p(idx), p(owner), p(core), p(atoms)))
        return dict(frag=frag, idx_map=idx, owner=owner, core_local=core, atoms=atoms[:L.natom_frag])

    # ---- tensors ---------------------------------------------------------------------------
    def empty_psi(self, dtype=None):
        torch = _torch()
        return torch.empty(self.layout.psi_elems, dtype=dtype or self.dtype, device="cuda")

    def grid_tensor(self):
        torch = _torch()
        return torch.empty(self.layout.npts, dtype=torch.float64, device="cuda")

    def initial(self, stream=None):
        vion, rho0 = self.grid_tensor(), self.grid_tensor()
        check("dc_get_initial", self.lib.dc_get_initial(self.ctx, _ptr(vion), _ptr(rho0), _stream(stream)))
        return vion, rho0

    # ---- calls -----------------------------------------------------------------------------
    def potential(self, rho, stream=None):
        veff = self.grid_tensor()
        check("dc_potential", self.lib.dc_potential(self.ctx, _ptr(rho), _ptr(veff), _stream(stream)))
        return veff

    def set_potential(self, veff, stream=None):
        check("dc_set_potential", self.lib.dc_set_potential(self.ctx, _ptr(veff), _stream(stream)))

    def hpsi(self, psi, out=None, stream=None):
        torch = _torch()
        out = torch.empty_like(psi) if out is None else out
        dt = DC_FP64 if psi.dtype == torch.float64 else DC_FP32
        check("dc_hpsi", self.lib.dc_hpsi(self.ctx, _ptr(psi), _ptr(out), dt, _stream(stream)))
        return out

    def lcfo_basis(self, psi, eps, eps_cut, lambda_cut=1e-7, stream=None):
        """DC-LCFO basis of every fragment (Sec. 2.3, Eqs. 6-7) from the orbital block ``psi`` and its
        eigenvalues ``eps`` (device tensors in the context's layout).  Returns (basis, nbasis, s,
        offsets): basis FP64 with fragment f's row k at offsets[f] + k |core_f| (rows k >= nbasis[f]
        zero), nbasis int32 per fragment, s the overlap eigenvalues per fragment in descending order,
        offsets a host list."""
        torch = _torch()
        nel = C.c_int64(0)
        offs = (C.c_int64 * self.layout.nfrag)()
        check("dc_lcfo_query", self.lib.dc_lcfo_query(self.ctx, C.byref(nel), offs))
        basis = torch.empty(nel.value, dtype=torch.float64, device=psi.device)
        nbasis = torch.empty(self.layout.nfrag, dtype=torch.int32, device=psi.device)
        sv = torch.empty(self.layout.nstates, dtype=torch.float64, device=psi.device)
        dt = DC_FP64 if psi.dtype == torch.float64 else DC_FP32
        check("dc_lcfo_basis", self.lib.dc_lcfo_basis(self.ctx, _ptr(psi), dt, _ptr(eps), float(eps_cut),
                                                       float(lambda_cut), _ptr(basis), _ptr(nbasis), _ptr(sv),
                                                       _stream(stream)))
        return basis, nbasis, sv, list(offs)

    def subspace(self, psi=None, eps=None, stream=None):
        """Rayleigh-Ritz without filtering.  ``psi=None``: of the context's own state.  Otherwise of the
        caller block ``psi`` (rotated in place); the Ritz values go to ``eps`` (allocated if None) and
        are returned."""
        torch = _torch()
        if psi is None:
            check("dc_subspace", self.lib.dc_subspace(self.ctx, None, 0, _ptr(eps), _stream(stream)))
            return eps
        eps = torch.empty(self.layout.nstates, dtype=torch.float64, device=psi.device) if eps is None else eps
        dt = DC_FP64 if psi.dtype == torch.float64 else DC_FP32
        check("dc_subspace", self.lib.dc_subspace(self.ctx, _ptr(psi), dt, _ptr(eps), _stream(stream)))
        return eps

    def chefsi(self, n_pass=1, stream=None):
        check("dc_chefsi", self.lib.dc_chefsi(self.ctx, int(n_pass), _stream(stream)))

    def warmup(self, stream=None):
        check("dc_warmup", self.lib.dc_warmup(self.ctx, _stream(stream)))

    def get_state(self, stream=None):
        torch = _torch()
        psi = self.empty_psi()
        eps = torch.empty(self.layout.nstates, dtype=torch.float64, device="cuda")
        check("dc_get_state", self.lib.dc_get_state(self.ctx, _ptr(psi), _ptr(eps), _stream(stream)))
        return psi, eps

    def set_state(self, psi=None, eps=None, stream=None):
        check("dc_set_state", self.lib.dc_set_state(self.ctx, _ptr(psi), _ptr(eps), _stream(stream)))

    def density(self, psi=None, eps=None, stream=None):
        """(rho, q, mu) from the context's own state (``psi=None``) or from a caller block ``psi`` with its
        eigenvalues ``eps``."""
        torch = _torch()
        rho = self.grid_tensor()
        q = torch.empty(self.layout.nstates, dtype=torch.float64, device="cuda")
        mu = torch.empty(1, dtype=torch.float64, device="cuda")
        dt = 0 if psi is None else (DC_FP64 if psi.dtype == torch.float64 else DC_FP32)
        check("dc_density", self.lib.dc_density(self.ctx, _ptr(psi), dt, _ptr(eps), _ptr(rho), _ptr(q), _ptr(mu),
                                                _stream(stream)))
        return rho, q, mu

    # ---- fragment-sharded step (Sec. 2.5) ----------------------------------------------------
    def step_local(self, rho_in, eps, q, stream=None):
        check("dc_step_local", self.lib.dc_step_local(self.ctx, _ptr(rho_in), _ptr(eps), _ptr(q), _stream(stream)))

    def step_density(self, eps, q, rho_part, mu=None, stream=None):
        check("dc_step_density", self.lib.dc_step_density(self.ctx, _ptr(eps), _ptr(q), _ptr(rho_part), _ptr(mu),
                                                          _stream(stream)))

    def step_finish(self, rho_in, rho_out, stream=None):
        st = _lib.dc_stats_t()
        check("dc_step_finish", self.lib.dc_step_finish(self.ctx, _ptr(rho_in), _ptr(rho_out), C.byref(st),
                                                        _stream(stream)))
        return dict(E=st.E, F=st.F, eband=st.eband, mu=st.mu, drho=st.drho, ne=st.ne, step=st.step)

    def scf_step(self, rho, stream=None):
        """One SCF step; ``rho`` is a CUDA float64 tensor (updated in place) or a host numpy array."""
        st = _lib.dc_stats_t()
        if isinstance(rho, np.ndarray):
            if rho.dtype != np.float64 or not rho.flags.c_contiguous or rho.size != self.layout.npts:
                raise ValueError("host rho must be a contiguous float64 array of npts values")
            ptr, host = C.c_void_p(rho.ctypes.data), 1
        else:
            ptr, host = _ptr(rho), 0
        status = self.lib.dc_scf_step(self.ctx, ptr, host, C.byref(st), _stream(stream))
        check("dc_scf_step", status)
        return dict(E=st.E, F=st.F, eband=st.eband, mu=st.mu, drho=st.drho, ne=st.ne, step=st.step)

    def rho_out(self, stream=None):
        rho = self.grid_tensor()
        check("dc_get_rho_out", self.lib.dc_get_rho_out(self.ctx, _ptr(rho), _stream(stream)))
        return rho

    def eb_adjoint(self, psi, occ, V, D, need_psi=True, need_V=True, need_D=True, stream=None):
        """E_b and its gradients (dpsi, dV, dD) through the native adjoint."""
        torch = _torch()
        dt = DC_FP64 if psi.dtype == torch.float64 else DC_FP32
        dpsi = torch.empty_like(psi) if need_psi else None
        dV = self.grid_tensor() if need_V else None
        dD = torch.empty(self.layout.natom, dtype=torch.float64, device="cuda") if need_D else None
        Eb = C.c_double(0.0)
        check("dc_eb_adjoint", self.lib.dc_eb_adjoint(self.ctx, _ptr(psi), dt, _ptr(occ), _ptr(V), _ptr(D),
                                                      C.byref(Eb), _ptr(dpsi), _ptr(dV), _ptr(dD),
                                                      _stream(stream)))
        return Eb.value, dpsi, dV, dD


def fermi_level_noalloc(eps, q, n_elec, kT, mu, occ, stream=None):
    """``dc_fermi_level_noalloc``: mu and occupations from eigenvalues ``eps`` and core weights ``q``
    (CUDA float64 tensors of one length) into the caller's tensors ``mu`` (1 element, read as the
    starting guess) and ``occ``.  The library allocates nothing; this wrapper creates no tensors."""
    torch = _torch()
    for name, t in (("eps", eps), ("q", q), ("occ", occ), ("mu", mu)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"fermi_level_noalloc: {name} must be a contiguous CUDA float64 tensor")
    if not (eps.device == q.device == occ.device == mu.device):
        raise ValueError("fermi_level_noalloc: eps, q, occ and mu must be on one device")
    if q.numel() != eps.numel() or occ.numel() != eps.numel():
        raise ValueError("fermi_level_noalloc: eps, q and occ must have the same number of elements")
    if mu.numel() < 1:
        raise ValueError("fermi_level_noalloc: mu needs one element")
    lib = load()
    check("dc_fermi_level_noalloc", lib.dc_fermi_level_noalloc(_ptr(eps), _ptr(q), int(eps.numel()), float(n_elec),
                                                               float(kT), _ptr(mu), _ptr(occ), _stream(stream)))


def _profile_methods():
    def profile(self, enable=True):
        check("dc_profile", self.lib.dc_profile(self.ctx, 1 if enable else 0))

    def profile_read(self):
        n = len(_lib.STAGES)
        ms = (C.c_double * n)()
        nl = (C.c_int64 * n)()
        by = (C.c_double * n)()
        check("dc_profile_read", self.lib.dc_profile_read(self.ctx, ms, nl, by))
        return {name: dict(ms=ms[i], launches=int(nl[i]), bytes=by[i]) for i, name in enumerate(_lib.STAGES)}

    def tuning(self):
        shp = (C.c_int * 6)()
        ms = (C.c_float * 40)()
        check("dc_tuning", self.lib.dc_tuning(self.ctx, shp, ms))
        return dict(fp32=dict(kind=shp[0], threads=shp[1], pairs=shp[2], candidates_ms=list(ms[0:20])),
                    fp64=dict(kind=shp[3], threads=shp[4], pairs=shp[5], candidates_ms=list(ms[20:40])))

    def set_tuning(self, dtype, kind, threads, pairs):
        """Pin the stencil launch shape for ``dtype`` ("fp64" or "fp32"); False if it does not fit."""
        st = self.lib.dc_set_tuning(self.ctx, PRECISIONS[dtype], int(kind), int(threads), int(pairs))
        if st == _lib.DC_OK:
            return True
        if st == -1:
            return False
        check("dc_set_tuning", st)

    DCSolver.profile = profile
    DCSolver.set_tuning = set_tuning
    DCSolver.profile_read = profile_read
    DCSolver.tuning = tuning


_profile_methods()


def _make_eb():
    torch = _torch()

    class EbFunction(torch.autograd.Function):
        """E_b = sum_f sum_i occ_i <psi_i|H_f[V, D]|psi_i> with a hand-written adjoint.

        The backward pass calls the native adjoint, which recomputes H psi (nothing is stored
        between forward and backward except the inputs).
        """

        @staticmethod
        def forward(ctx, psi, V, D, occ, solver):
            Eb, _, _, _ = solver.eb_adjoint(psi, occ, V, D, need_psi=False, need_V=False, need_D=False)
            ctx.save_for_backward(psi, V, D, occ)
            ctx.solver = solver
            return torch.tensor(Eb, dtype=torch.float64, device=psi.device)

        @staticmethod
        def backward(ctx, g):
            psi, V, D, occ = ctx.saved_tensors
            _, dpsi, dV, dD = ctx.solver.eb_adjoint(psi, occ, V, D, need_psi=ctx.needs_input_grad[0],
                                                    need_V=ctx.needs_input_grad[1], need_D=ctx.needs_input_grad[2])
            gs = g.to(torch.float64)
            out_psi = None if dpsi is None else dpsi * gs.to(dpsi.dtype)
            out_V = None if dV is None else dV * gs
            out_D = None if dD is None else dD * gs
            return out_psi, out_V, out_D, None, None

    return EbFunction


class _EbProxy:
    _fn = None

    def apply(self, psi, V, D, occ, solver):
        if _EbProxy._fn is None:
            _EbProxy._fn = _make_eb()
        return _EbProxy._fn.apply(psi, V, D, occ, solver)


Eb = _EbProxy()
