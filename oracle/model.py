"""Model fragment Hamiltonian (test infrastructure; FP64 oracle).

Eq. 5 gives H^alpha = -1/2 nabla^2 + V_loc + V_NL + V_H[rho_tot] + V_xc + V^alpha.
The paper uses a real-space finite-difference kinetic operator, norm-conserving
pseudopotentials and LDA (Sec. 2.2); it does not print the stencil order, the
pseudopotentials or the functional.  Readings used here:

* Kinetic: 8th-order central finite differences (25 points), coefficients
  derived in exact rational arithmetic from polynomial exactness.
* V_loc: the periodic potential of Gaussian ion charges Z (width sigma_loc),
  evaluated in reciprocal space with G=0 dropped.
* V_NL: one separable s-projector per atom, D_a |p_a><p_a|, with a Gaussian
  p_a of width sigma_proj normalised to 1 in the continuum, summed over
  periodic images and truncated per axis at |x - X_a| < 5 sigma_proj (a cubic
  support, so p_a is exactly a product of three 1-D factors).
* V_H: global FFT Poisson solve on rho_tot, exact G^2, G=0 dropped (Eq. 5).
* V_xc: Slater exchange v_x = -(3 rho/pi)^(1/3) on rho_tot (correlation and
  the fragment-density argument are left out; V^alpha = 0, the paper's default).
* Fragment boundary: ghost points are zero (bc="zero") or wrap within the
  fragment extent (bc="periodic", Sec. 2.2).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fd_second_derivative_coefficients(order: int = 8):
    """Central-difference weights c_0..c_{order/2} of d^2/dx^2 (h = 1), as exact Fractions.

    Solves sum_n c_n (n^k + (-n)^k) = k! [k == 2] for even k <= order, the
    conditions that the stencil differentiates x^k exactly (Fornberg 1988).
    """
    r = order // 2
    # unknowns c_0..c_r; equations for k = 0, 2, 4, ..., 2r
    A = [[Fraction(0)] * (r + 1) for _ in range(r + 1)]
    rhs = [Fraction(0)] * (r + 1)
    for row, k in enumerate(range(0, 2 * r + 1, 2)):
        A[row][0] = Fraction(1 if k == 0 else 0)
        for n in range(1, r + 1):
            A[row][n] = Fraction(2 * n ** k)
        rhs[row] = Fraction(2) if k == 2 else Fraction(0)
    # Gaussian elimination in exact arithmetic
    m = r + 1
    for c in range(m):
        p = next(i for i in range(c, m) if A[i][c] != 0)
        A[c], A[p] = A[p], A[c]
        rhs[c], rhs[p] = rhs[p], rhs[c]
        for i in range(m):
            if i != c and A[i][c] != 0:
                fac = A[i][c] / A[c][c]
                A[i] = [A[i][j] - fac * A[c][j] for j in range(m)]
                rhs[i] = rhs[i] - fac * rhs[c]
    return [rhs[i] / A[i][i] for i in range(m)]


FD8 = fd_second_derivative_coefficients(8)
FD8_F = np.array([float(c) for c in FD8])


class Grid:
    """Periodic orthorhombic grid: n points, cell lengths L (bohr), spacing h = L/n."""

    def __init__(self, n, L):
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in L)
        self.h = tuple(self.L[d] / self.n[d] for d in range(3))
        self.dV = self.h[0] * self.h[1] * self.h[2]
        self.volume = self.L[0] * self.L[1] * self.L[2]
        self.npts = self.n[0] * self.n[1] * self.n[2]

    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def gvectors(self):
        """G components on the FFT grid (numpy frequency order), arrays shaped [Nz][Ny][Nx]."""
        g = [2.0 * np.pi * np.fft.fftfreq(self.n[d], d=1.0 / self.n[d]) / self.L[d] for d in range(3)]
        gx = g[0][None, None, :]
        gy = g[1][None, :, None]
        gz = g[2][:, None, None]
        return gx, gy, gz

    def g2(self):
        gx, gy, gz = self.gvectors()
        return gx * gx + gy * gy + gz * gz


# ----------------------------------------------------------------------------------------------
# Kinetic operator
# ----------------------------------------------------------------------------------------------

def _shift(psi, axis, n, bc):
    """psi evaluated at local index j+n along ``axis``: zero ghosts or periodic wrap in the fragment."""
    if bc == "periodic":
        return np.roll(psi, -n, axis=axis)
    out = np.zeros_like(psi)
    E = psi.shape[axis]
    if abs(n) >= E:
        return out
    src = [slice(None)] * psi.ndim
    dst = [slice(None)] * psi.ndim
    if n > 0:
        src[axis] = slice(n, E)
        dst[axis] = slice(0, E - n)
    else:
        src[axis] = slice(0, E + n)
        dst[axis] = slice(-n, E)
    out[tuple(dst)] = psi[tuple(src)]
    return out


def laplacian(psi, h, bc):
    """8th-order FD Laplacian of psi[..., z, y, x] with the fragment boundary condition."""
    out = np.zeros_like(psi)
    nd = psi.ndim
    for d, axis in ((0, nd - 1), (1, nd - 2), (2, nd - 3)):
        w = 1.0 / (h[d] * h[d])
        out += (FD8_F[0] * w) * psi
        for n in range(1, 5):
            out += (FD8_F[n] * w) * (_shift(psi, axis, n, bc) + _shift(psi, axis, -n, bc))
    return out


def kinetic_symbol_max(h):
    """Largest eigenvalue of -1/2 L_8 on any periodic grid: sum_d -(c0 + 2 sum_n c_n (-1)^n)/(2 h_d^2)."""
    s = FD8_F[0] + 2.0 * sum(FD8_F[n] * (-1) ** n for n in range(1, 5))
    return sum(-s / (2.0 * h[d] * h[d]) for d in range(3))


# ----------------------------------------------------------------------------------------------
# Local ionic potential, Hartree, exchange (global grid)
# ----------------------------------------------------------------------------------------------

def rho_ion_G(grid: Grid, pos, species, spec):
    """rho_ion(G) = (1/Omega) sum_a Z_a exp(-G^2 sigma_a^2/2) exp(-i G.R_a) on the FFT grid."""
    gx, gy, gz = grid.gvectors()
    g2 = gx * gx + gy * gy + gz * gz
    out = np.zeros(grid.shape(), dtype=np.complex128)
    for a in range(len(pos)):
        s = species[a]
        Z = spec["Z"][s]
        sig = spec["sigma_loc"][s]
        phase = np.exp(-1j * gx * pos[a, 0]) * np.exp(-1j * gy * pos[a, 1]) * np.exp(-1j * gz * pos[a, 2])
        out += Z * np.exp(-0.5 * g2 * sig * sig) * phase
    return out / grid.volume


def v_ion(grid: Grid, pos, species, spec):
    """V_loc(r) = Re sum_G [-4 pi rho_ion(G)/G^2] e^{iG.r}, G=0 dropped (Gaussian ions, Eq. 5 V_loc)."""
    g2 = grid.g2()
    rG = rho_ion_G(grid, pos, species, spec)
    vG = np.zeros_like(rG)
    nz = g2 > 0
    vG[nz] = -4.0 * np.pi * rG[nz] / g2[nz]
    return np.real(np.fft.ifftn(vG)) * grid.npts


def hartree(grid: Grid, rho):
    """V_H[rho] = Re IFFT(4 pi rho(G)/G^2), G=0 dropped (Eq. 5, global Poisson equation)."""
    g2 = grid.g2()
    rG = np.fft.fftn(rho)
    vG = np.zeros_like(rG)
    nz = g2 > 0
    vG[nz] = 4.0 * np.pi * rG[nz] / g2[nz]
    return np.real(np.fft.ifftn(vG))


def vx(rho):
    """Slater exchange potential v_x = -(3 rho/pi)^(1/3) (LDA exchange only)."""
    return -np.cbrt(3.0 * np.maximum(rho, 0.0) / np.pi)


def ex_energy(grid: Grid, rho):
    """E_x = -3/4 (3/pi)^(1/3) int rho^(4/3)."""
    r = np.maximum(rho, 0.0)
    return -0.75 * np.cbrt(3.0 / np.pi) * grid.dV * np.sum(r * np.cbrt(r))


def es_energy(grid: Grid, rho, rhoiG):
    """Electrostatic energy of rho - rho_ion: (Omega/2) sum_{G!=0} 4 pi |rho(G)-rho_ion(G)|^2/G^2."""
    g2 = grid.g2()
    rG = np.fft.fftn(rho) / grid.npts - rhoiG
    nz = g2 > 0
    return 0.5 * grid.volume * np.sum(4.0 * np.pi * np.abs(rG[nz]) ** 2 / g2[nz])


def periodic_gaussian_1d(x, X, sigma, cut, L):
    """sum over images n of exp(-(x - X - nL)^2/(2 sigma^2)) for |x - X - nL| < cut.

    Returns (values, in_support) for an array of coordinates x.
    """
    K = int(np.ceil(cut / L)) + 1
    val = np.zeros_like(x, dtype=np.float64)
    sup = np.zeros(x.shape, dtype=bool)
    t = x - X
    for n in range(-K, K + 1):
        d = t - n * L
        m = np.abs(d) < cut
        val += np.where(m, np.exp(-(d * d) / (2.0 * sigma * sigma)), 0.0)
        sup |= m
    return val, sup


def initial_density(grid: Grid, pos, species, spec):
    """Starting density: the Gaussian ion charges band-limited to the FFT grid, clamped at 0, scaled to N_e.

    rho_0(r) = max(Re sum_G rho_ion(G) e^{iG.r}, 0) * N_e / int(...).  (The paper does not state its
    starting density; this reading costs one inverse FFT on either side.)
    """
    rho = np.maximum(np.real(np.fft.ifftn(rho_ion_G(grid, pos, species, spec))) * grid.npts, 0.0)
    ne = float(np.sum(spec["Z"][species]))
    return rho * (ne / (grid.dV * np.sum(rho)))


# ----------------------------------------------------------------------------------------------
# Separable projectors restricted to a fragment
# ----------------------------------------------------------------------------------------------

PROJ_CUT_SIGMAS = 5.0


class FragmentProjectors:
    """Projector factors of the atoms that touch fragment f.

    atoms[k] is a global atom index (ascending); gx[k], gy[k], gz[k] are the
    1-D factors on the fragment's local axes; coef[k] = (pi sigma^2)^(-3/4);
    D[k] the strength.  p_k(j) = coef[k] gx[k][jx] gy[k][jy] gz[k][jz].
    """

    def __init__(self, frags, f, grid: Grid, pos, species, spec):
        self.atoms = []
        facs = []
        for a in range(len(pos)):
            s = species[a]
            sig = spec["sigma_proj"][s]
            cut = PROJ_CUT_SIGMAS * sig
            per_axis = []
            ok = True
            for d in range(3):
                x = frags.local_global_axis(f, d) * grid.h[d]
                v, sup = periodic_gaussian_1d(x, pos[a, d], sig, cut, grid.L[d])
                if not np.any(sup):
                    ok = False
                    break
                per_axis.append(v)
            if ok:
                self.atoms.append(a)
                facs.append((per_axis, (np.pi * sig * sig) ** (-0.75), spec["D"][s]))
        self.atoms = np.array(self.atoms, dtype=np.int64)
        self.gx = [p[0][0] for p in facs]
        self.gy = [p[0][1] for p in facs]
        self.gz = [p[0][2] for p in facs]
        self.coef = np.array([p[1] for p in facs])
        self.D = np.array([p[2] for p in facs])

    def dense(self):
        """P[k][j]: projector k on the fragment's flat points (x fastest)."""
        rows = []
        for k in range(len(self.atoms)):
            p = self.coef[k] * (self.gz[k][:, None, None] * self.gy[k][None, :, None] * self.gx[k][None, None, :])
            rows.append(p.reshape(-1))
        if not rows:
            return np.zeros((0, 0))
        return np.array(rows)


class FragmentHamiltonian:
    """H_f psi = -1/2 L8 psi + V_f psi + sum_a D_a p_a <p_a|psi>, <u|v> = dV sum u v (Eq. 5, model)."""

    def __init__(self, frags, f, grid: Grid, V_global, proj: FragmentProjectors, bc, D=None, V_frag=None):
        """V_global: the global potential, restricted to the fragment; or V_frag: the fragment's own
        potential on its points ([Ez][Ey][Ex], Eq. 5 with per-fragment terms)."""
        self.f = f
        self.shape = (int(frags.extent[f, 2]), int(frags.extent[f, 1]), int(frags.extent[f, 0]))
        self.h = grid.h
        self.dV = grid.dV
        self.bc = bc
        if V_frag is not None:
            self.V = np.asarray(V_frag, dtype=np.float64).reshape(self.shape)
        else:
            idx = frags.idx_map(f)
            self.V = V_global.reshape(-1)[idx].reshape(self.shape)
        self.P = proj.dense()
        self.D = proj.D.copy() if D is None else np.asarray(D, dtype=np.float64)

    def apply(self, psi):
        """psi shaped [n][Ez][Ey][Ex] (or one orbital [Ez][Ey][Ex])."""
        single = psi.ndim == 3
        X = psi[None] if single else psi
        out = -0.5 * laplacian(X, self.h, self.bc) + self.V[None] * X
        if len(self.D):
            flat = X.reshape(X.shape[0], -1)
            c = self.dV * (flat @ self.P.T)  # <p_a|psi_i>
            out += ((c * self.D[None, :]) @ self.P).reshape(X.shape)
        return out[0] if single else out

    def projections(self, psi):
        flat = psi.reshape(psi.shape[0], -1)
        return self.dV * (flat @ self.P.T)

    def upper_bound(self):
        """Rigorous spectral upper bound: kinetic symbol max + max V_f + sum_a max(D_a,0) <p_a|p_a>."""
        nl = 0.0
        if len(self.D):
            pp = self.dV * np.sum(self.P * self.P, axis=1)
            nl = float(np.sum(np.maximum(self.D, 0.0) * pp))
        return kinetic_symbol_max(self.h) + float(np.max(self.V)) + nl

    def dense(self):
        """Dense matrix of H_f (small fragments only), columns = apply to unit vectors."""
        n = int(np.prod(self.shape))
        eye = np.eye(n).reshape((n,) + self.shape)
        return self.apply(eye).reshape(n, n).T
