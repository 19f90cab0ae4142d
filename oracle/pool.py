"""The oracle's fragment solves spread over host processes (test infrastructure; FP64 oracle).

Within an SCF step the fragments are independent until the chemical potential is found (Sec. 2.2), so
their CheFSI passes, core weights and core densities can run in separate processes without changing
any arithmetic: each worker holds a ``scf.DCState`` restricted to its own fragments, and the global
stages (potential, Fermi level, energy, mixing) stay with the caller.  Workers are started with
``spawn`` and run one BLAS thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys

import numpy as np

_ST = None
_KEYS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _init(root, cfg, frags):
    global _ST
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import scf
    _ST = scf.DCState(cfg, fragments_subset=frags)


def _warm(V, n_pass, round_fp32):
    """Rayleigh-Ritz of the starting block, then n_pass CheFSI passes in V; with round_fp32 the orbitals
    are rounded to FP32 afterwards.  Returns {f: (orbitals, Ritz values)}."""
    st = _ST
    st.initial_rr(V)
    st.solve(V, n_pass)
    out = {}
    for f in st.active:
        if round_fp32:
            st.psi[f] = st.psi[f].astype(np.float32).astype(np.float64)
        out[f] = (st.psi[f].astype(np.float32) if round_fp32 else st.psi[f].copy(), st.eps[f].copy())
    return out


def _initial_rr(V):
    _ST.initial_rr(V)
    return {}


def _solve(V, n_pass):
    """n_pass CheFSI passes; returns {f: (Ritz values, core weights)}."""
    from oracle import density
    st = _ST
    st.solve(V, n_pass)
    return {f: (st.eps[f].copy(), density.core_weights(st.frags, f, st.psi[f], st.grid.dV)) for f in st.active}


def _core_density(mu):
    """{f: (global indices of the core, rho_out there)} with occupations at mu (Eqs. 2-4)."""
    from oracle import density, fermi
    st = _ST
    out = {}
    for f in st.active:
        occ = fermi.occupation(st.eps[f], mu, st.kT)
        out[f] = density.core_density(st.frags, f, st.psi[f], occ)
    return out


def _core_squares():
    """{f: (|psi_i|^2 on the core [n][core points], their global indices)}."""
    st = _ST
    out = {}
    for f in st.active:
        cm = st.frags.core_mask(f)
        out[f] = (st.psi[f][:, cm] ** 2, st.frags.idx_map(f)[cm.reshape(-1)])
    return out


class FragmentPool:
    """Worker processes, each owning a contiguous chunk of the fragments ``frags``."""

    def __init__(self, cfg, frags, nproc=None):
        frags = [int(f) for f in frags]
        nproc = max(1, min(len(frags), nproc or os.cpu_count() or 1))
        self.nproc = nproc
        chunks = [list(map(int, c)) for c in np.array_split(np.asarray(frags, dtype=np.int64), nproc) if len(c)]
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in _KEYS}
        os.environ.update({k: "1" for k in _KEYS})
        try:
            self.pools = [ctx.Pool(1, initializer=_init, initargs=(root, cfg, c)) for c in chunks]
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def _map(self, fn, *args):
        res = [p.apply_async(fn, args) for p in self.pools]
        out = {}
        for r in res:
            out.update(r.get(timeout=3600))
        return out

    def warm(self, V, n_pass, round_fp32=False):
        return self._map(_warm, V, n_pass, round_fp32)

    def initial_rr(self, V):
        self._map(_initial_rr, V)

    def solve(self, V, n_pass):
        return self._map(_solve, V, n_pass)

    def core_density(self, mu):
        return self._map(_core_density, mu)

    def core_squares(self):
        return self._map(_core_squares)

    def close(self):
        for p in self.pools:
            p.close()
            p.join()
