"""DC-LCFO basis construction (test infrastructure; FP64 oracle).

Only tests/, the package's smoke entry and the bench's CPU-baseline leg may use this module.

Sec. 2.3, Eqs. 6-7: after the SCF loop, each fragment keeps its orbitals whose
eigenvalue lies below the cutoff energy eps_cut, projects them onto its core
Omega_0^alpha (zero outside it, the same projection as Eq. 3), forms their overlap
matrix S_ij = <phibar_i|phibar_j>, and diagonalises it.  Eigenvectors whose
eigenvalue falls below lambda_cut are dropped; the others define basis functions
localised on the core and orthonormal there (and therefore across fragments,
whose cores do not overlap).

Readings where the paper leaves a choice open:
- "lower than eps_cut" is strict: orbital i is selected when eps_i < eps_cut.
- lambda_cut is an absolute threshold on the eigenvalues s of S (core projections of
  normalised orbitals give 0 <= s <= 1); direction k is kept when s_k > lambda_cut.
- The basis is lambda_k = sum_i phibar_i U_ik / sqrt(s_k) over the kept eigenpairs
  (s_k, U_k) of S, ordered by descending s_k.  Any orthonormal basis of the kept span
  is equally valid; tests compare the span (its projector), the kept eigenvalues and
  the count, which are unique.

Inner products carry the volume element: <u|v> = dV sum_j u_j v_j.
"""
from __future__ import annotations

import numpy as np


def selected(eps, eps_cut):
    """Indices of the orbitals with eps_i < eps_cut, in orbital order (Sec. 2.3)."""
    return np.nonzero(np.asarray(eps) < eps_cut)[0]


def core_projected(frags, f, psi, sel):
    """phibar_i restricted to the core of fragment f: [len(sel)][core points], points in
    fragment order (z slowest, x fastest) -- the projection onto Omega_0^alpha (Eq. 3 form)."""
    cm = frags.core_mask(f)
    return psi[sel][:, cm]


def overlap(phibar, dV):
    """S_ij = <phibar_i|phibar_j> (Eq. 6)."""
    return dV * (phibar @ phibar.T)


def basis(phibar, dV, lambda_cut):
    """Eigenvalues of S in descending order and the kept basis functions [m][core points]."""
    s, U = np.linalg.eigh(overlap(phibar, dV))
    order = np.argsort(-s, kind="stable")
    s, U = s[order], U[:, order]
    keep = s > lambda_cut
    B = (U[:, keep] / np.sqrt(s[keep])).T @ phibar
    return s, B


def fragment_basis(frags, f, psi, eps, dV, eps_cut, lambda_cut):
    """The whole step for fragment f: (eigenvalues of S descending, basis [m][core points])."""
    sel = selected(eps, eps_cut)
    return basis(core_projected(frags, f, psi, sel), dV, lambda_cut)


def span_projector(B, dV):
    """dV sum_k lambda_k lambda_k^T on the core points: the orthogonal projector onto the span."""
    return dV * (B.T @ B)
