"""Global chemical potential (test infrastructure; FP64 oracle).

Sec. 2.2: mu is determined globally so that the core-projected density
integrates to N_e, with Fermi-Dirac occupations at a finite electronic
temperature (Eq. 4).  With spin degeneracy and the core weights
q_i^f = <psi_i^f|1_core|psi_i^f>, the condition reads

    N(mu) = sum_f sum_i 2 f_FD((eps_i^f - mu)/kT) q_i^f = N_e,
    f_FD(x) = 1/(1+e^x) = (1 - tanh(x/2))/2.

Solved by bisection on [min eps - 40 kT, max eps + 40 kT] until the bracket
is below 1e-13 Ha or after 200 halvings.
"""
from __future__ import annotations

import numpy as np


def occupation(eps, mu, kT):
    """Fermi-Dirac f in [0,1] (per spin)."""
    return 0.5 * (1.0 - np.tanh(0.5 * (np.asarray(eps) - mu) / kT))


def electron_count(eps, q, mu, kT):
    return float(np.sum(2.0 * occupation(eps, mu, kT) * q))


def find_mu(eps, q, ne, kT, tol=1e-13, maxit=200):
    lo = float(np.min(eps)) - 40.0 * kT
    hi = float(np.max(eps)) + 40.0 * kT
    for _ in range(maxit):
        if hi - lo < tol:
            break
        mid = 0.5 * (lo + hi)
        if electron_count(eps, q, mid, kT) < ne:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def entropy(eps, q, mu, kT):
    """S = -sum 2 q [f ln f + (1-f) ln(1-f)] (0 ln 0 = 0)."""
    f = occupation(eps, mu, kT)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(f > 0, f * np.log(f), 0.0) + np.where(f < 1, (1 - f) * np.log1p(-f), 0.0)
    return float(-np.sum(2.0 * q * t))
