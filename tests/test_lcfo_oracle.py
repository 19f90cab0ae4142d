"""Pins of the DC-LCFO basis oracle (Sec. 2.3, Eqs. 6-7) against the mathematics (CPU only).

The overlap and its eigenpairs are checked against a closed-form 2 x 2 eigenproblem, the basis
against orthonormality, reconstruction of the selected orbitals and a QR factorisation of the
selected core vectors (a library routine), and the truncation against a planted linear
dependence.  Orbital values outside the core are set to large numbers throughout, so a basis
or overlap that leaks the buffer region fails.
"""
import math

import numpy as np
import pytest

from oracle import lcfo, maps

DV = 0.37  # a volume element far from 1, so a dropped dV shows


@pytest.fixture(scope="module")
def frags():
    return maps.Fragments((8, 8, 8), (2, 2, 2), (1, 1, 1))  # 6^3 fragments with 4^3 cores


def _block(frags, f, core_rows, rng):
    """Orbitals [n][Ez][Ey][Ex] with the given core values and large random buffer values."""
    E = tuple(int(v) for v in frags.extent[f][::-1])
    cm = frags.core_mask(f)
    psi = 50.0 * rng.standard_normal((core_rows.shape[0],) + E)
    psi[:, cm] = core_rows
    return psi


def test_two_orbitals_closed_form(frags):
    """S = dV [[u.u, u.v], [u.v, v.v]]: eigenvalues (a+b)/2 +- sqrt(((a-b)/2)^2 + c^2), descending."""
    r = np.random.default_rng(1)
    f = 5
    ncore = int(frags.core_mask(f).sum())
    u, v = r.standard_normal(ncore), r.standard_normal(ncore)
    psi = _block(frags, f, np.stack([u, v]), r)
    s, B = lcfo.fragment_basis(frags, f, psi, np.array([-1.0, -0.5]), DV, 0.0, 1e-7)
    a, b, c = DV * u @ u, DV * v @ v, DV * u @ v
    mid, rad = 0.5 * (a + b), math.sqrt((0.5 * (a - b)) ** 2 + c * c)
    assert s[0] == pytest.approx(mid + rad, rel=1e-13)
    assert s[1] == pytest.approx(mid - rad, rel=1e-13)
    assert B.shape == (2, ncore)


def test_basis_is_orthonormal_and_reproduces_the_selected_orbitals(frags):
    r = np.random.default_rng(2)
    f = 3
    cm = frags.core_mask(f)
    ncore = int(cm.sum())
    n = 12
    psi = _block(frags, f, r.standard_normal((n, ncore)), r)
    eps = np.sort(r.uniform(-1.0, 1.0, n))
    eps_cut = 0.5 * (eps[7] + eps[8])  # 8 selected
    s, B = lcfo.fragment_basis(frags, f, psi, eps, DV, eps_cut, 1e-7)
    assert B.shape == (8, ncore) and len(s) == 8
    assert np.all(np.diff(s) <= 0.0)
    np.testing.assert_allclose(DV * B @ B.T, np.eye(8), atol=1e-12)
    P = lcfo.span_projector(B, DV)
    for i in range(n):
        x = psi[i][cm]
        res = x - P @ x
        if i < 8:
            assert DV * res @ res < 1e-20 * (DV * x @ x)  # selected: inside the span
        else:
            assert DV * res @ res > 1e-3 * (DV * x @ x)  # not selected: generic, outside it


def test_projector_equals_qr_of_the_selected_core_vectors(frags):
    r = np.random.default_rng(3)
    f = 0
    cm = frags.core_mask(f)
    X = r.standard_normal((6, int(cm.sum())))
    psi = _block(frags, f, X, r)
    _, B = lcfo.fragment_basis(frags, f, psi, np.linspace(-1, 0, 6), DV, 10.0, 1e-7)
    Q, _ = np.linalg.qr(X.T)
    np.testing.assert_allclose(lcfo.span_projector(B, DV), Q @ Q.T, atol=1e-12)


def test_planted_dependence_is_dropped(frags):
    """phibar_2 = 0.3 phibar_0 - 0.7 phibar_1 on the core (the buffer differs): S is singular,
    one direction falls below lambda_cut and the span is that of phibar_0, phibar_1."""
    r = np.random.default_rng(4)
    f = 6
    cm = frags.core_mask(f)
    u, v = r.standard_normal((2, int(cm.sum())))
    psi = _block(frags, f, np.stack([u, v, 0.3 * u - 0.7 * v]), r)
    s, B = lcfo.fragment_basis(frags, f, psi, np.array([-3.0, -2.0, -1.0]), DV, 0.0, 1e-7)
    assert B.shape[0] == 2
    assert abs(s[2]) < 1e-13 * s[0]
    Q, _ = np.linalg.qr(np.stack([u, v]).T)
    np.testing.assert_allclose(lcfo.span_projector(B, DV), Q @ Q.T, atol=1e-12)


def test_core_orthonormal_input_keeps_every_direction(frags):
    """Orbitals orthonormal on the core: S = I, every s = 1, and the span is theirs."""
    r = np.random.default_rng(5)
    f = 7
    cm = frags.core_mask(f)
    Q, _ = np.linalg.qr(r.standard_normal((int(cm.sum()), 5)))
    X = Q.T / math.sqrt(DV)
    psi = _block(frags, f, X, r)
    s, B = lcfo.fragment_basis(frags, f, psi, np.zeros(5) - 1.0, DV, 0.0, 1e-7)
    np.testing.assert_allclose(s, np.ones(5), atol=1e-13)
    np.testing.assert_allclose(lcfo.span_projector(B, DV), DV * X.T @ X, atol=1e-12)


def test_selection_is_strict_and_in_orbital_order():
    eps = np.array([-0.2, -0.1, 0.0, 0.1])
    assert list(lcfo.selected(eps, 0.0)) == [0, 1]
    assert list(lcfo.selected(eps, 0.0 + 1e-15)) == [0, 1, 2]
    assert list(lcfo.selected(np.array([0.3, -0.3, 0.1]), 0.2)) == [1, 2]
