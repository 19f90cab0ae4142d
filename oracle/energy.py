"""Total energy, mixing and convergence measure (test infrastructure; FP64 oracle).

The paper gives no DC total-energy expression.  Reading: the band sum uses
core-weighted eigenvalues, and the double counting is removed with the input
potential, so that the result is the Kohn-Sham energy T + E_NL + E_es + E_x
evaluated at rho_out (for one fragment spanning the cell this is the plain
Kohn-Sham functional):

    E = sum_f sum_i 2 f_i eps_i q_i - int V_in rho_out + E_es[rho_out] + E_x[rho_out]

with V_in = V_loc + V_H[rho_in] + v_x[rho_in].  With hxc = "none" the model is
non-interacting and E is the band sum alone.  The free energy is E - kT S.
The SCF residual is int |rho_out - rho_in| / N_e (Sec. 3.3 convergence
criterion), and the next input density is the linear mix
rho_in + alpha (rho_out - rho_in).
"""
from __future__ import annotations

import numpy as np

from . import model


def band_sum(eps, q, occ):
    return float(np.sum(2.0 * occ * eps * q))


def total_energy(grid, hxc, eband, V_in, rho_out, rhoiG):
    if hxc == "none":
        return eband
    return (eband - grid.dV * float(np.sum(V_in * rho_out))
            + model.es_energy(grid, rho_out, rhoiG) + model.ex_energy(grid, rho_out))


def residual(grid, rho_out, rho_in, ne):
    return grid.dV * float(np.sum(np.abs(rho_out - rho_in))) / ne


def mix(rho_in, rho_out, alpha, grid=None, q0=0.0):
    """Next input density.  q0 = 0: plain linear mixing rho_in + alpha (rho_out - rho_in).  q0 > 0:
    Kerker-preconditioned linear mixing, each Fourier component of the residual weighted by
    alpha G^2/(G^2 + q0^2) (long wavelengths damped; G = 0 carries no charge change)."""
    if q0 <= 0.0:
        return rho_in + alpha * (rho_out - rho_in)
    g2 = grid.g2()
    w = alpha * g2 / (g2 + q0 * q0)
    return rho_in + np.real(np.fft.ifftn(w * np.fft.fftn(rho_out - rho_in)))
