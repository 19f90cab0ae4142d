"""Pins of the FP64 oracle against the mathematics it follows (CPU only).

Each test ties an oracle function to something other than its own formula:
polynomial exactness, published coefficient tables, closed forms, analytic
potentials, dense brute force, library routines (eigh, chebval, brentq) and
finite differences.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import brentq
from scipy.special import erf

import workloads
from oracle import adjoint, chefsi, density, energy, fermi, maps, model, rng, scf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------------------------
# Finite-difference Laplacian
# ---------------------------------------------------------------------------------------------

def test_fd8_matches_published_table():
    """FD8 weights derived in the oracle equal Fornberg (1988) Table 1 exactly."""
    for off, num, den in _read_golden("fd8_fornberg1988.txt"):
        assert model.FD8[int(off)] == Fraction(int(num), int(den))


def test_fd8_polynomial_exactness_and_order():
    """The 9-point stencil differentiates x^k exactly for k <= 9 and fails at k = 10."""
    c = model.FD8
    for k in range(0, 12):
        # second derivative of x^k at x = 3 with h = 1, in exact arithmetic
        x0 = Fraction(3)
        approx = c[0] * x0 ** k + sum(c[n] * ((x0 + n) ** k + (x0 - n) ** k) for n in range(1, 5))
        exact = Fraction(k * (k - 1)) * x0 ** (k - 2) if k >= 2 else Fraction(0)
        if k <= 9:
            assert approx == exact, k
        else:
            assert approx != exact, k
    # convergence order 8 on a smooth periodic function
    errs = []
    for N in (16, 32):
        L = 2 * np.pi
        h = L / N
        x = np.arange(N) * h
        f = np.sin(x)[None, None, :] * np.ones((4, 4, 1))
        lap = model.laplacian(f, (h, 1e9, 1e9), "periodic")
        errs.append(np.max(np.abs(lap[0, 0] + np.sin(x))))
    assert 2 ** 7.5 < errs[0] / errs[1] < 2 ** 8.5


def _symbol(h, m, N):
    c = model.FD8_F
    return -0.5 * sum((c[0] + 2 * sum(c[n] * math.cos(2 * math.pi * n * m[d] / N[d]) for n in range(1, 5))) / h[d] ** 2
                      for d in range(3))


def test_laplacian_plane_wave_symbol():
    """-1/2 L8 cos(G.r) = eps(m) cos(G.r) on a periodic box, eps from the stencil's symbol."""
    N = (10, 12, 14)
    L = (5.0, 6.6, 7.4)
    h = [L[d] / N[d] for d in range(3)]
    z, y, x = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
    for m in [(1, 0, 0), (0, 2, 0), (0, 0, 3), (2, 3, 1), (5, 6, 7)]:
        phase = 2 * np.pi * (m[0] * x / N[0] + m[1] * y / N[1] + m[2] * z / N[2])
        psi = np.cos(phase)
        out = -0.5 * model.laplacian(psi, h, "periodic")
        np.testing.assert_allclose(out, _symbol(h, m, N) * psi, atol=1e-11)


def test_kinetic_symbol_max():
    h = (0.4, 0.5, 0.6)
    worst = max(_symbol(h, (mx, my, mz), (8, 8, 8)) for mx in range(8) for my in range(8) for mz in range(8))
    assert abs(model.kinetic_symbol_max(h) - worst) < 1e-12


def _empty_box_hamiltonian(N, L, bc="periodic"):
    grid = model.Grid(N, L)
    frags = maps.Fragments(N, (1, 1, 1), (0, 0, 0))

    class NoProj:
        atoms = np.zeros(0, dtype=np.int64)
        D = np.zeros(0)

        def dense(self):
            return np.zeros((0, grid.npts))

    return model.FragmentHamiltonian(frags, 0, grid, np.zeros(grid.shape()), NoProj(), bc), grid


def _converge(H, n, passes, m=12, seed=3):
    shape = (n,) + H.shape
    X = rng.orbital_block(seed, 0, n, int(np.prod(H.shape))).reshape(shape)
    eps, X, _ = chefsi.rayleigh_ritz(H, X)
    for _ in range(passes):
        eps, X, _ = chefsi.chefsi_pass(H, X, m, eps)
    return eps, X


def test_chefsi_empty_periodic_box_closed_form():
    """P1: lowest CheFSI eigenvalues of an empty periodic box equal the closed-form FD spectrum."""
    N = (10, 11, 12)
    L = (6.0, 6.6, 7.4)
    H, grid = _empty_box_hamiltonian(N, L)
    spec = sorted(_symbol(grid.h, (mx, my, mz), N) for mx in range(N[0]) for my in range(N[1]) for mz in range(N[2]))
    eps, _ = _converge(H, 12, 25)
    np.testing.assert_allclose(eps[:7], spec[:7], atol=1e-10)


# ---------------------------------------------------------------------------------------------
# Dense brute force, Hermiticity
# ---------------------------------------------------------------------------------------------

def _kron_laplacian(E, h, bc):
    """Independent dense FD Laplacian as a Kronecker sum of 1-D banded matrices (x fastest)."""
    c = model.FD8_F
    mats = []
    for d in range(3):
        n = E[d]
        D2 = np.zeros((n, n))
        for j in range(n):
            for k in range(-4, 5):
                jj = j + k
                if bc == "periodic":
                    D2[j, jj % n] += c[abs(k)] / h[d] ** 2
                elif 0 <= jj < n:
                    D2[j, jj] += c[abs(k)] / h[d] ** 2
        mats.append(D2)
    Ix, Iy, Iz = (np.eye(E[0]), np.eye(E[1]), np.eye(E[2]))
    return (np.kron(Iz, np.kron(Iy, mats[0])) + np.kron(Iz, np.kron(mats[1], Ix)) + np.kron(mats[2], np.kron(Iy, Ix)))


def _direct_projector(frags, f, grid, R, sigma):
    """p(r) at the fragment points, evaluated directly in 3-D (cubic cut per axis, images summed)."""
    cut = model.PROJ_CUT_SIGMAS * sigma
    coords = [frags.local_global_axis(f, d) * grid.h[d] for d in range(3)]
    z, y, x = np.meshgrid(coords[2], coords[1], coords[0], indexing="ij")
    pts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    val = np.zeros(len(pts))
    K = [int(np.ceil(cut / grid.L[d])) + 1 for d in range(3)]
    for nx in range(-K[0], K[0] + 1):
        for ny in range(-K[1], K[1] + 1):
            for nz in range(-K[2], K[2] + 1):
                dvec = pts - (R + np.array([nx * grid.L[0], ny * grid.L[1], nz * grid.L[2]]))
                inside = np.all(np.abs(dvec) < cut, axis=1)
                val += np.where(inside, np.exp(-np.sum(dvec * dvec, axis=1) / (2 * sigma ** 2)), 0.0)
    return (np.pi * sigma ** 2) ** -0.75 * val


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_dense_bruteforce_fragment(bc):
    """P2: oracle H_f equals an independently built dense matrix, and converged CheFSI gives its eigenvalues."""
    cfg = workloads.small_config(n=(12, 12, 12), L=(7.2, 7.2, 7.2), num_fragment=(2, 2, 2), buffer=(2, 2, 2),
                                 natom=3, bc=bc)
    st = scf.DCState(cfg)
    V = st.veff(st.rho_in)
    f = 5
    H = st.hamiltonian(f, V)
    E = tuple(int(v) for v in st.frags.extent[f])
    Hk = -0.5 * _kron_laplacian(E, st.grid.h, bc)
    Hk += np.diag(V.reshape(-1)[st.frags.idx_map(f)])
    for k, a in enumerate(st.proj[f].atoms):
        s = st.species[a]
        p = _direct_projector(st.frags, f, st.grid, st.pos[a], st.spec["sigma_proj"][s])
        Hk += st.spec["D"][s] * st.grid.dV * np.outer(p, p)
    Hd = H.dense()
    assert np.max(np.abs(Hd - Hk)) < 1e-11 * np.max(np.abs(Hk))
    w = sla.eigh(Hk, eigvals_only=True)
    eps, _ = _converge(H, 10, 30)
    np.testing.assert_allclose(eps[:6], w[:6], atol=1e-9)


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_hermiticity(bc):
    """P3: <phi|H psi> = <H phi|psi> to FP64 rounding."""
    cfg = workloads.small_config(bc=bc, natom=4)
    st = scf.DCState(cfg)
    V = st.veff(st.rho_in)
    r = np.random.default_rng(0)
    for f in (0, 3, 7):
        H = st.hamiltonian(f, V)
        a = r.standard_normal((1,) + H.shape)
        b = r.standard_normal((1,) + H.shape)
        lhs = np.sum(a * H.apply(b))
        rhs = np.sum(H.apply(a) * b)
        assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(a * H.apply(b)))


# ---------------------------------------------------------------------------------------------
# Maps
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,F,b", [((20, 20, 20), (2, 2, 2), (4, 4, 4)), ((21, 13, 8), (2, 3, 4), (3, 2, 1)),
                                   ((6, 6, 6), (1, 2, 3), (4, 4, 4)), ((9, 7, 5), (1, 1, 1), (0, 0, 0))])
def test_partition_of_unity(n, F, b):
    """P4: cores partition the cell: sum_f w_f(g) = 1 at every point, owner/core_local consistent."""
    fr = maps.Fragments(n, F, b)
    assert np.all(fr.weight_sum() == 1)
    owner, core_local = fr.owner()
    assert np.all(owner >= 0)
    for g in range(0, int(np.prod(n)), 7):
        assert fr.idx_map(owner[g])[core_local[g]] == g
    # cores differ by at most one point per axis (floor partition)
    for d in range(3):
        lens = np.diff(fr.starts[d])
        assert lens.max() - lens.min() <= 1 and lens.sum() == n[d]


def test_orbital_count_rule():
    """Auto orbital count n_f = ceil(Ne/2) + max(4, ceil(0.2 ceil(Ne/2))) from atoms with an image in the box."""
    fr = maps.Fragments((10, 10, 10), (2, 1, 1), (1, 0, 0))
    pos = np.array([[0.5, 5.0, 5.0], [2.0, 5.0, 5.0], [9.5, 5.0, 5.0]])
    n = maps.orbital_counts(fr, 0, (10.0, 10.0, 10.0), pos, np.zeros(3, dtype=np.int64), np.array([4.0]))
    assert list(n) == [10, 8]


# ---------------------------------------------------------------------------------------------
# Potentials and energies against analytic forms
# ---------------------------------------------------------------------------------------------

def _one_atom(L, N, sigma, Z=4.0):
    grid = model.Grid((N, N, N), (L, L, L))
    R = np.array([[L / 2, L / 2, L / 2]])
    spec = dict(Z=np.array([Z]), sigma_loc=np.array([sigma]), sigma_proj=np.array([0.6]), D=np.array([0.5]))
    return grid, R, np.zeros(1, dtype=np.int64), spec


def _sampled_gaussian(grid, R, sigma, Z):
    """Z (2 pi sigma^2)^(-3/2) exp(-|r-R|^2/(2 sigma^2)) sampled on the grid (nearest image; box >> sigma)."""
    coords = [np.arange(grid.n[d]) * grid.h[d] for d in range(3)]
    d = [coords[k] - R[k] for k in range(3)]
    d = [v - grid.L[k] * np.round(v / grid.L[k]) for k, v in enumerate(d)]
    r2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
    return Z * (2 * np.pi * sigma * sigma) ** -1.5 * np.exp(-r2 / (2 * sigma * sigma))


def test_vion_matches_gaussian_charge_potential():
    """V_loc near a Gaussian ion = -Z erf(r/(sqrt2 sigma))/r - (2 pi Z/3 Omega) r^2 + const (cubic images).

    The r^2 term is the neutralising background -Z/Omega that dropping G=0 implies; V is the electron's
    potential energy, -phi.
    """
    L, N, sig, Z = 30.0, 60, 0.8, 4.0
    grid, R, spc, spec = _one_atom(L, N, sig, Z)
    V = model.v_ion(grid, R, spc, spec)
    c = N // 2
    h = L / N
    pts, rs = [], []
    for k in (1, 2, 3):
        for off in ((k, 0, 0), (0, k, 0), (k, k, 0), (1, k, 1)):
            r = h * math.sqrt(sum(o * o for o in off))
            if r <= 1.6:
                pts.append(V[c + off[2], c + off[1], c + off[0]])
                rs.append(r)
    rs = np.array(rs)
    ana = -Z * erf(rs / (math.sqrt(2) * sig)) / rs - 2 * math.pi * Z / (3 * grid.volume) * rs ** 2
    v0 = V[c, c, c]
    ana0 = -Z * math.sqrt(2.0 / math.pi) / sig
    np.testing.assert_allclose(np.array(pts) - v0, ana - ana0, atol=2e-5)


def test_hartree_cancels_ion_potential():
    """V_H of the Gaussian ion charge sampled on the grid cancels V_loc up to a constant."""
    L, N, sig = 16.0, 40, 0.8
    grid, R, spc, spec = _one_atom(L, N, sig)
    rho = _sampled_gaussian(grid, R[0], sig, 4.0)
    tot = model.hartree(grid, rho) + model.v_ion(grid, R, spc, spec)
    assert np.ptp(tot) < 1e-6


def test_hartree_solves_fd_poisson():
    """-L8 V_H = 4 pi (rho - mean rho) for a smooth periodic density (independent operator)."""
    grid = model.Grid((32, 36, 40), (12.0, 13.0, 14.0))
    z, y, x = np.meshgrid(*[np.arange(grid.n[d]) * grid.h[d] for d in (2, 1, 0)], indexing="ij")
    L = grid.L
    rho = np.exp(np.cos(2 * np.pi * x / L[0]) + 0.5 * np.sin(2 * np.pi * y / L[1])
                 + 0.7 * np.cos(2 * np.pi * z / L[2] + 1.0))  # smooth and periodic
    V = model.hartree(grid, rho)
    lhs = -model.laplacian(V, grid.h, "periodic")
    rhs = 4 * np.pi * (rho - rho.mean())
    assert np.max(np.abs(lhs - rhs)) < 1e-5 * np.max(np.abs(rhs))  # FD truncation of high harmonics


def test_es_energy_neutral_pair():
    """E_es of ion + displaced electron Gaussian = 2 self energies - Z^2 erf(d/2s)/d - 2 pi p^2/(3 Omega)."""
    L, N, sig, Z = 30.0, 64, 0.8, 4.0
    grid, R, spc, spec = _one_atom(L, N, sig, Z)
    d = 1.875  # four grid spacings... any value; the electron cloud is sampled at an offset centre
    Re = R + np.array([[d, 0.0, 0.0]])
    rho = _sampled_gaussian(grid, Re[0], sig, Z)
    E = model.es_energy(grid, rho, model.rho_ion_G(grid, R, spc, spec))
    ana = 2 * Z * Z / (2 * sig * math.sqrt(math.pi)) - Z * Z * erf(d / (2 * sig)) / d - 2 * math.pi * (Z * d) ** 2 / (
        3 * grid.volume)
    assert abs(E - ana) < 5e-5
    # an electron cloud identical to the ion gives zero
    rho0 = _sampled_gaussian(grid, R[0], sig, Z)
    assert abs(model.es_energy(grid, rho0, model.rho_ion_G(grid, R, spc, spec))) < 1e-8


def test_initial_density_is_band_limited_ion_charge():
    """Starting density integrates to N_e and matches a sampled Gaussian where the latter is resolved."""
    L, N, sig = 16.0, 40, 0.8
    grid, R, spc, spec = _one_atom(L, N, sig)
    rho = model.initial_density(grid, R, spc, spec)
    assert abs(grid.dV * rho.sum() - 4.0) < 1e-12
    ref = _sampled_gaussian(grid, R[0], sig, 4.0)
    assert np.max(np.abs(rho - ref)) < 1e-6 * np.max(ref)


def test_kerker_mixing_plane_wave_and_charge():
    """Kerker mixing scales a plane-wave residual by alpha G^2/(G^2+q0^2) and keeps the charge; q0=0 is linear."""
    grid = model.Grid((12, 10, 8), (6.0, 5.0, 4.0))
    z, y, x = np.meshgrid(*[np.arange(grid.n[d]) * grid.h[d] for d in (2, 1, 0)], indexing="ij")
    G = np.array([2 * np.pi * 2 / 6.0, 2 * np.pi * 1 / 5.0, 0.0])
    res = 0.05 * np.cos(G[0] * x + G[1] * y)
    rho_in = np.full(grid.shape(), 0.1)
    alpha, q0 = 0.3, 0.8
    out = energy.mix(rho_in, rho_in + res, alpha, grid, q0)
    g2 = float(G @ G)
    np.testing.assert_allclose(out - rho_in, alpha * g2 / (g2 + q0 * q0) * res, atol=1e-14)
    r = np.random.default_rng(3).uniform(0.0, 0.2, grid.shape())
    assert abs(energy.mix(rho_in, r, alpha, grid, q0).sum() - rho_in.sum()) < 1e-12
    np.testing.assert_allclose(energy.mix(rho_in, r, alpha, grid, 0.0), rho_in + alpha * (r - rho_in))


def test_exchange_uniform_gas():
    grid = model.Grid((6, 6, 6), (5.0, 5.0, 5.0))
    rho = np.full(grid.shape(), 0.03)
    assert abs(model.ex_energy(grid, rho) - (-0.75 * (3 / np.pi) ** (1 / 3) * 0.03 ** (4 / 3) * 125.0)) < 1e-13
    assert np.allclose(model.vx(rho), -(3 * 0.03 / np.pi) ** (1 / 3))


def test_projector_normalisation_and_separability():
    """p_a is continuum-normalised (<p|p> = 1 on a fine grid) and equals the direct 3-D evaluation."""
    cfg = workloads.small_config(n=(40, 40, 40), L=(10.0, 10.0, 10.0), num_fragment=(1, 1, 1), buffer=(0, 0, 0),
                                 natom=1, bc="periodic")
    st = scf.DCState(cfg)
    P = st.proj[0]
    p = P.dense()[0]
    assert abs(st.grid.dV * np.sum(p * p) - 1.0) < 1e-9
    pd = _direct_projector(st.frags, 0, st.grid, st.pos[0], st.spec["sigma_proj"][0])
    assert np.max(np.abs(p - pd)) < 1e-13 * np.max(p)


# ---------------------------------------------------------------------------------------------
# Chebyshev filter and Rayleigh-Ritz
# ---------------------------------------------------------------------------------------------

class _DiagH:
    def __init__(self, lam):
        self.lam = lam
        self.dV = 1.0

    def apply(self, X):
        return X * self.lam[None, :, None, None]


def test_chebyshev_filter_is_scaled_chebyshev_polynomial():
    """Filter output on eigen-components = T_m((l-c)/e)/T_m((aL-c)/e) (numpy chebval)."""
    lam = np.linspace(-1.5, 30.0, 57)
    H = _DiagH(lam)
    X = np.ones((1, lam.size, 1, 1))
    m, a, b, aL = 10, 0.4, 31.0, -1.2
    Y = chefsi.chebyshev_filter(H, X, m, a, b, aL)[0, :, 0, 0]
    e, c = (b - a) / 2, (b + a) / 2
    coeff = [0] * m + [1]
    ref = np.polynomial.chebyshev.chebval((lam - c) / e, coeff) / np.polynomial.chebyshev.chebval((aL - c) / e, coeff)
    np.testing.assert_allclose(Y, ref, rtol=1e-11, atol=1e-13)


class _DenseH:
    def __init__(self, A, dV):
        self.A = A
        self.dV = dV

    def apply(self, X):
        flat = X.reshape(X.shape[0], -1)
        return (flat @ self.A.T).reshape(X.shape)


def test_rayleigh_ritz_exact_on_invariant_subspace():
    r = np.random.default_rng(1)
    n = 30
    M = r.standard_normal((n, n))
    A = M + M.T
    w, U = np.linalg.eigh(A)
    k = 5
    dV = 0.37
    Y = (r.standard_normal((k, k)) @ U[:, :k].T).reshape(k, n, 1, 1)
    eps, Psi, C = chefsi.rayleigh_ritz(_DenseH(A, dV), Y)
    np.testing.assert_allclose(eps, w[:k], atol=1e-11)
    G = dV * Psi.reshape(k, -1) @ Psi.reshape(k, -1).T
    np.testing.assert_allclose(G, np.eye(k), atol=1e-11)


# ---------------------------------------------------------------------------------------------
# Fermi level, electron count
# ---------------------------------------------------------------------------------------------

def test_fermi_two_level_symmetric():
    """P8: levels -D, +D with two electrons: mu = 0 by f(-x) = 1 - f(x)."""
    mu = fermi.find_mu(np.array([-0.3, 0.3]), np.array([1.0, 1.0]), 2.0, 0.05)
    assert abs(mu) < 1e-13


def test_fermi_low_temperature_aufbau():
    eps = np.array([-1.0, -0.7, -0.5, -0.2, 0.1, 0.4])
    q = np.ones(6)
    mu = fermi.find_mu(eps, q, 6.0, 1e-4)
    occ = fermi.occupation(eps, mu, 1e-4)
    np.testing.assert_allclose(occ, [1, 1, 1, 0, 0, 0], atol=1e-12)
    assert -0.5 < mu < -0.2


def test_fermi_matches_brentq_and_is_monotone():
    r = np.random.default_rng(4)
    eps = r.uniform(-1, 1, 200)
    q = r.uniform(0.05, 0.3, 200)
    mus = []
    for ne in (5.0, 10.0, 20.0):
        mu = fermi.find_mu(eps, q, ne, 0.01)
        ref = brentq(lambda m: fermi.electron_count(eps, q, m, 0.01) - ne, -3, 3, xtol=1e-15)
        assert abs(mu - ref) < 1e-11
        mus.append(mu)
    assert mus[0] < mus[1] < mus[2]


def test_entropy_is_minus_temperature_derivative_of_grand_potential():
    """The smearing entropy equals -dOmega/dT at fixed mu, Omega(T) = -T sum_i 2 q_i ln(1 + e^{-(eps_i - mu)/T})
    the grand potential of independent spin-degenerate fermionic levels weighted by q (k_B = 1).  A
    central difference in T checks the oracle's S, including its factor 2, its q weighting and its sign."""
    r = np.random.default_rng(11)
    eps = r.uniform(-0.3, 0.3, 64)
    q = r.uniform(0.05, 1.0, 64)
    mu = 0.017

    def omega(T):
        return -T * float(np.sum(2.0 * q * np.logaddexp(0.0, -(eps - mu) / T)))

    for kT in (0.01, 0.03, 0.1):
        dT = 1e-5 * kT
        s_fd = -(omega(kT + dT) - omega(kT - dT)) / (2.0 * dT)
        s = fermi.entropy(eps, q, mu, kT)
        assert s > 0.0
        assert abs(s - s_fd) < 1e-7 * s, (kT, s, s_fd)


def test_entropy_closed_forms():
    """A level at mu is half filled: 2 ln 2 per unit weight; a level far from mu carries none; the
    entropy of a level at eps - mu = x kT is 2 [ln(1 + e^x) - x e^x/(1 + e^x)] (here x = ln 3, f = 1/4:
    2 [ln 4 - (3/4) ln 3])."""
    kT = 0.02
    assert abs(fermi.entropy(np.array([0.5]), np.array([1.0]), 0.5, kT) - 2.0 * math.log(2.0)) < 1e-15
    assert abs(fermi.entropy(np.array([0.5]), np.array([0.25]), 0.5, kT) - 0.5 * math.log(2.0)) < 1e-15
    assert fermi.entropy(np.array([-5.0, 5.0]), np.array([1.0, 1.0]), 0.0, kT) < 1e-100
    x = math.log(3.0)
    want = 2.0 * (math.log(4.0) - 0.75 * math.log(3.0))
    assert abs(fermi.entropy(np.array([x * kT]), np.array([1.0]), 0.0, kT) - want) < 1e-14


def test_density_residual_hand_computed():
    """int |rho_out - rho_in| dV / N_e on a 4x2x2 grid (dV = 0.125 bohr^3, 16 points): half the points
    differ by +0.3, four by -0.2, four agree, so the integral is 0.125 (8 * 0.3 + 4 * 0.2) = 0.4 and, for
    N_e = 2, the residual is 0.2 whatever the values of rho_in (Sec. 3.3 convergence measure)."""
    grid = model.Grid((4, 2, 2), (2.0, 1.0, 1.0))
    assert grid.dV == 0.125
    r = np.random.default_rng(3)
    rho_in = r.uniform(0.5, 2.0, grid.shape())
    d = np.zeros(16)
    d[:8] = 0.3
    d[8:12] = -0.2
    rho_out = rho_in + r.permutation(d).reshape(grid.shape())
    assert abs(energy.residual(grid, rho_out, rho_in, 2.0) - 0.2) < 1e-14
    assert energy.residual(grid, rho_in, rho_in, 2.0) == 0.0


def test_electron_count_conserved():
    """P6: int rho_out = N_e after mu is found."""
    cfg = workloads.small_config(natom=3, n_warmup=2)
    st = scf.DCState(cfg)
    st.warmup()
    q, mu, occ, rho = st.density_stage()
    assert abs(st.grid.dV * rho.sum() - st.ne) < 1e-10 * st.ne


# ---------------------------------------------------------------------------------------------
# Single fragment = conventional DFT
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("xc_fragment,xi", [(False, 0.0), (True, 0.0), (True, 0.7)])
def test_single_fragment_equals_conventional_dft(xc_fragment, xi):
    """P5: F=1, b=0, periodic DC reduces to a dense-diagonalisation Kohn-Sham SCF (per-step energies).

    With the per-fragment exchange-correlation and density-template potential (Eq. 5), the one fragment's
    density is the previous step's output density, so the reference SCF takes v_x of the previous output
    density (of the starting potential's eigenstates before step 1) and, for xi > 0, adds
    (rho_prev_out - rho_in)/xi; its energy is still the direct Kohn-Sham energy of the output orbitals."""
    natom, nst = 2, 8
    cfg = workloads.small_config(n=(10, 10, 10), L=(6.0, 6.0, 6.0), num_fragment=(1, 1, 1), buffer=(0, 0, 0),
                                 nstate=nst, natom=natom, bc="periodic", cheb_degree=14, n_pass=25, n_warmup=40,
                                 seed=11, xc_fragment=xc_fragment, xi=xi)
    st = scf.DCState(cfg)
    st.warmup()
    dc = [st.scf_step() for _ in range(3)]

    # conventional: dense matrices, full diagonalisation, q = 1, direct energy terms
    grid = model.Grid(cfg["n"], cfg["L"])
    fr = maps.Fragments(cfg["n"], (1, 1, 1), (0, 0, 0))
    E = grid.n
    Lap = _kron_laplacian(E, grid.h, "periodic")
    P = []
    D = []
    for a in range(natom):
        s = cfg["species"][a]
        P.append(_direct_projector(fr, 0, grid, cfg["pos"][a], cfg["spec"]["sigma_proj"][s]))
        D.append(cfg["spec"]["D"][s])
    P = np.array(P)
    D = np.array(D)
    vion = model.v_ion(grid, cfg["pos"], cfg["species"], cfg["spec"])
    rhoiG = model.rho_ion_G(grid, cfg["pos"], cfg["species"], cfg["spec"])
    rho_in = model.initial_density(grid, cfg["pos"], cfg["species"], cfg["spec"])
    ne = float(np.sum(cfg["spec"]["Z"][cfg["species"]]))

    def solve(V):
        H = -0.5 * Lap + np.diag(V.reshape(-1)) + grid.dV * (P.T * D) @ P
        w, U = np.linalg.eigh(H)
        w, U = w[:nst], U[:, :nst] / math.sqrt(grid.dV)
        mu = brentq(lambda m: np.sum(2 * 0.5 * (1 - np.tanh(0.5 * (w - m) / cfg["kT"]))) - ne, -5, 5, xtol=1e-15)
        occ = 0.5 * (1 - np.tanh(0.5 * (w - mu) / cfg["kT"]))
        return w, U, mu, occ, ((U * U) @ (2 * occ)).reshape(grid.shape())

    rho_prev = solve(vion + model.hartree(grid, rho_in) + model.vx(rho_in))[4]  # the warm state's density
    for step in range(3):
        if xc_fragment:
            V = vion + model.hartree(grid, rho_in) + model.vx(rho_prev)
            if xi > 0.0:
                V = V + (rho_prev - rho_in) / xi
        else:
            V = vion + model.hartree(grid, rho_in) + model.vx(rho_in)
        w, U, mu, occ, rho_out = solve(V)
        rho_prev = rho_out
        T = np.sum(2 * occ * np.einsum("pi,pq,qi->i", U, -0.5 * Lap, U)) * grid.dV
        c = grid.dV * P @ U
        Enl = np.sum(2 * occ[None, :] * D[:, None] * c * c)
        Etot = T + Enl + model.es_energy(grid, rho_out, rhoiG) + model.ex_energy(grid, rho_out)
        assert abs(dc[step]["E"] - Etot) / natom < 1e-10, (step, dc[step]["E"], Etot)
        assert abs(dc[step]["mu"] - mu) < 1e-9
        assert np.max(np.abs(dc[step]["rho_out"] - rho_out)) < 1e-9
        rho_in = rho_in + cfg["mix_alpha"] * (rho_out - rho_in)


# ---------------------------------------------------------------------------------------------
# Band-energy gradient, random orbitals
# ---------------------------------------------------------------------------------------------

def test_band_energy_gradient_finite_differences():
    """P7: analytic dE_b/dpsi, dE_b/dV, dE_b/dD against central differences (E_b is at most quadratic)."""
    cfg = workloads.small_config(natom=3, nstate=4)
    st = scf.DCState(cfg)
    r = np.random.default_rng(5)
    V = st.veff(st.rho_in) + 0.1 * r.standard_normal(st.grid.shape())
    D = np.array([st.spec["D"][s] for s in st.species]) + 0.1
    psi = {f: r.standard_normal(st.psi[f].shape) for f in st.active}
    occ = {f: r.uniform(0, 2, st.norb[f]) for f in st.active}
    gpsi, gV, gD = adjoint.band_energy_grad(st, psi, V, D, occ)
    dpsi = {f: r.standard_normal(psi[f].shape) for f in st.active}
    dVv = r.standard_normal(V.shape)
    dD = r.standard_normal(D.shape)
    t = 1e-3

    def E(ps, vv, dd):
        return adjoint.band_energy(st, ps, vv, dd, occ)

    fd = (E({f: psi[f] + t * dpsi[f] for f in psi}, V, D) - E({f: psi[f] - t * dpsi[f] for f in psi}, V, D)) / (2 * t)
    an = sum(np.sum(gpsi[f] * dpsi[f]) for f in psi)
    assert abs(fd - an) < 1e-8 * abs(an)
    fd = (E(psi, V + t * dVv, D) - E(psi, V - t * dVv, D)) / (2 * t)
    assert abs(fd - np.sum(gV * dVv)) < 1e-8 * abs(fd)
    fd = (E(psi, V, D + t * dD) - E(psi, V, D - t * dD)) / (2 * t)
    assert abs(fd - np.sum(gD * dD)) < 1e-8 * abs(fd)


# ---------------------------------------------------------------------------------------------
# Counter-based generator
# ---------------------------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    for key, out in _read_golden("splitmix64_seed0.txt"):
        assert int(rng.splitmix64(np.array([int(key, 16)], dtype=np.uint64))[0]) == int(out, 16)


def test_orbital_block_range_and_layout():
    blk = rng.orbital_block(99, 3, 4, 1000)
    assert blk.shape == (4, 1000) and blk.min() >= -1.0 and blk.max() < 1.0
    key = 99 ^ (((3 << 20) | 2) << 32) ^ 17
    z = int(rng.splitmix64(np.array([key], dtype=np.uint64))[0])
    assert blk[2, 17] == (z >> 11) * 2.0 ** -52 - 1.0


# ---------------------------------------------------------------------------------------------
# Buffer-thickness convergence (Sec. 3: DC accuracy improves monotonically with the buffer)
# ---------------------------------------------------------------------------------------------
def test_dc_energy_converges_with_buffer_thickness():
    """Fixed-density DC (mix_alpha = 0) on 2x2x2 fragments approaches the single-fragment solve of the
    same cell as the buffer b grows, monotonically, and by two orders of magnitude over b = 1..4."""
    base = dict(n=(20, 20, 20), L=(10.26, 10.26, 10.26), nstate=10, natom=6, seed=21, mix_alpha=0.0,
                n_warmup=12, cheb_degree=12, n_pass=4)
    ref_cfg = workloads.small_config(num_fragment=(1, 1, 1), buffer=(0, 0, 0), bc="periodic",
                                     **dict(base, nstate=20))
    st = scf.DCState(ref_cfg)
    st.warmup()
    E_ref = [st.scf_step() for _ in range(2)][-1]["E"]
    err = []
    for b in (1, 2, 3, 4):
        cfg = workloads.small_config(num_fragment=(2, 2, 2), buffer=(b, b, b), bc="zero", **base)
        st = scf.DCState(cfg)
        st.warmup()
        E = [st.scf_step() for _ in range(2)][-1]["E"]
        err.append(abs(E - E_ref) / 6)
    assert all(err[k + 1] < err[k] for k in range(3)), err
    assert err[-1] < 0.01 and err[0] / err[-1] > 20, err
