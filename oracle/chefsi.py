"""Chebyshev-filtered subspace iteration on one fragment (test infrastructure; FP64 oracle).

Eq. 1 asks for the lowest ``nstate_frag`` eigenpairs of each fragment
Hamiltonian; the paper's inner solver is "the same procedure as conventional
DFT" (Sec. 2.2) and names no algorithm.  Reading: one pass of
Chebyshev-filtered subspace iteration (Zhou, Saad, Tiago & Chelikowsky,
J. Comput. Phys. 219, 172 (2006), scaled three-term filter), followed by
Cholesky orthonormalisation and a Rayleigh-Ritz step:

  1. bounds: a = largest and a_L = smallest Ritz value of the previous pass,
     b = the fragment's rigorous spectral upper bound;
  2. Y = p_m(H) X, the degree-m filter damping [a, b] and scaled to 1 at a_L;
  3. S = <Y|Y>, S = L L^T;
  4. Hs = L^-1 <Y|H Y> L^-T, Hs = Q diag(eps) Q^T (ascending);
  5. Psi = Y L^-T Q.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def filter_coefficients(m: int, a: float, b: float, aL: float):
    """Per-step (alpha_k, beta_k, c) of Y_k = alpha_k (H - c) Y_{k-1} + beta_k Y_{k-2}, k = 1..m."""
    e = (b - a) / 2.0
    c = (b + a) / 2.0
    sigma = e / (aL - c)
    tau = 2.0 / sigma
    coefs = [(sigma / e, 0.0)]
    for _ in range(2, m + 1):
        sigma_new = 1.0 / (tau - sigma)
        coefs.append((2.0 * sigma_new / e, -sigma * sigma_new))
        sigma = sigma_new
    return coefs, c


def chebyshev_filter(H, X, m: int, a: float, b: float, aL: float):
    """Scaled Chebyshev filter of degree m applied to the block X (Zhou et al. 2006)."""
    coefs, c = filter_coefficients(m, a, b, aL)
    alpha, _ = coefs[0]
    Yprev = X
    Y = alpha * (H.apply(X) - c * X)
    for alpha, beta in coefs[1:]:
        Ynew = alpha * (H.apply(Y) - c * Y) + beta * Yprev
        Yprev, Y = Y, Ynew
    return Y


def rayleigh_ritz(H, Y):
    """Cholesky orthonormalisation and Rayleigh-Ritz of the block Y.  Returns (eps, Psi, C)."""
    n = Y.shape[0]
    flat = Y.reshape(n, -1)
    S = H.dV * (flat @ flat.T)
    HY = H.apply(Y).reshape(n, -1)
    A = H.dV * (flat @ HY.T)
    L = np.linalg.cholesky(S)
    Linv = sla.solve_triangular(L, np.eye(n), lower=True)
    Hs = Linv @ A @ Linv.T
    Hs = 0.5 * (Hs + Hs.T)
    eps, Q = sla.eigh(Hs)
    C = Linv.T @ Q
    Psi = (C.T @ flat).reshape(Y.shape)
    return eps, Psi, C


def chefsi_pass(H, X, m: int, eps_prev):
    """One CheFSI pass: filter with bounds from the previous Ritz values, then Rayleigh-Ritz."""
    a = float(np.max(eps_prev))
    aL = float(np.min(eps_prev))
    b = H.upper_bound()
    Y = chebyshev_filter(H, X, m, a, b, aL)
    return rayleigh_ritz(H, Y)
