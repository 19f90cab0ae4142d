"""Core weights and the core-projected density (test infrastructure; FP64 oracle).

Eqs. 2-4: rho_alpha = sum_i f(eps_i - mu) |phi_i|^2 on the fragment, projected
onto the core Omega_0^alpha, and rho_tot = sum_alpha of the projections.  The
cores partition the cell, so each global point takes the density of exactly
one fragment (its owner).  Spin degeneracy gives the factor 2.
"""
from __future__ import annotations

import numpy as np


def core_weights(frags, f, psi, dV):
    """q_i = <psi_i|1_core|psi_i> for the block psi [n][Ez][Ey][Ex]."""
    cm = frags.core_mask(f)
    return dV * np.sum(psi[:, cm] ** 2, axis=1)


def core_density(frags, f, psi, occ):
    """Values of rho_tot on the core of fragment f: sum_i 2 occ_i psi_i^2, and their global indices."""
    cm = frags.core_mask(f)
    vals = np.einsum("i,ip->p", 2.0 * occ, psi[:, cm] ** 2)
    g = frags.idx_map(f)[cm.reshape(-1)]
    return g, vals
