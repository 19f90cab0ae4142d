"""Band energy and its gradients (test infrastructure; FP64 oracle).

The band energy of the fragment problems (Eqs. 1 and 5) with fixed
occupations occ_i in [0, 2] and orbitals that need not be normalised:

    E_b = sum_f sum_i occ_i <psi_i^f|H_f|psi_i^f>,

where H_f depends on the global potential V (restricted to the fragment) and
the projector strengths D_a.  Its gradients:

    dE_b/dpsi_i^f(j) = 2 occ_i dV (H_f psi_i^f)(j)
    dE_b/dV(g)       = dV sum_f sum_{j: idx_map[f][j] = g} sum_i occ_i psi_i^f(j)^2
    dE_b/dD_a        = sum_f sum_i occ_i <p_a|psi_i^f>^2       (a in A_f)

dE_b/dV is the unweighted scatter-sum of the fragment densities (every
fragment that covers g contributes, not only the owner).
"""
from __future__ import annotations

import numpy as np

from . import model


def band_energy(state, psi, V, D, occ):
    """E_b for orbital blocks psi[f], global potential V, per-atom strengths D, occupations occ[f]."""
    E = 0.0
    for f in state.active:
        H = model.FragmentHamiltonian(state.frags, f, state.grid, V, state.proj[f], state.bc,
                                      D=np.asarray(D)[state.proj[f].atoms])
        Hpsi = H.apply(psi[f])
        E += state.grid.dV * float(np.sum(occ[f][:, None, None, None] * psi[f] * Hpsi))
    return E


def band_energy_grad(state, psi, V, D, occ):
    """(dE/dpsi per fragment, dE/dV global, dE/dD per atom)."""
    dV = state.grid.dV
    gpsi = {}
    gV = np.zeros(state.grid.npts)
    gD = np.zeros(len(D))
    for f in state.active:
        P = state.proj[f]
        H = model.FragmentHamiltonian(state.frags, f, state.grid, V, P, state.bc, D=np.asarray(D)[P.atoms])
        gpsi[f] = 2.0 * dV * occ[f][:, None, None, None] * H.apply(psi[f])
        dens = np.einsum("i,ip->p", occ[f], psi[f].reshape(psi[f].shape[0], -1) ** 2)
        np.add.at(gV, state.frags.idx_map(f), dV * dens)
        if len(P.atoms):
            c = H.projections(psi[f])  # [n][A]
            np.add.at(gD, P.atoms, np.einsum("i,ia->a", occ[f], c * c))
    return gpsi, gV.reshape(state.grid.shape()), gD
