"""Pins of the FP64 oracle's SH transforms against facts fixed outside the oracle.

Each test checks the oracle against a closed form, a textbook identity, an
independent library routine (scipy's complex spherical harmonics) or an exact
quadrature, so that a dropped term, a wrong sign or index, or a transposed
operand in ``oracle/sh.py`` fails at least one of them.
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import sh as osh
from paper_1808_01517_gb300 import synth

PHI = (1 + 5 ** 0.5) / 2
# six icosahedron vertices, one of each antipodal pair: an equal-weight quadrature
# (spherical 5-design) for even functions of degree <= 4
ICOSA_HALF = np.array([[0, 1, PHI], [0, -1, PHI], [1, PHI, 0], [-1, PHI, 0], [PHI, 0, 1], [-PHI, 0, 1]],
                      np.float64)
ICOSA_HALF /= np.linalg.norm(ICOSA_HALF, axis=1, keepdims=True)


def product_quadrature(L):
    """Gauss-Legendre in cos(theta) x uniform phi, exact for polynomials of degree <= 2L+1."""
    x, wx = leggauss(L + 2)
    nphi = 2 * L + 3
    phi = 2 * np.pi * np.arange(nphi) / nphi
    X, P = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - X ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), X], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return dirs, w


def test_t1_index_table_is_bijective():
    for L in (0, 2, 4, 8, 12):
        l, m = osh.sh_lm(L)
        assert len(l) == osh.n_coef(L) == (L + 1) * (L + 2) // 2
        assert all(osh.sh_index(a, b) == j for j, (a, b) in enumerate(zip(l, m)))
        assert np.all(l % 2 == 0) and np.all(np.abs(m) <= l)


@pytest.mark.parametrize("L", [2, 4, 8, 10])
def test_basis_orthonormal_under_exact_quadrature(L):
    dirs, w = product_quadrature(L)
    B = osh.real_sh(L, dirs)
    G = B.T @ (w[:, None] * B)
    assert np.max(np.abs(G - np.eye(B.shape[1]))) < 1e-13


def test_basis_matches_scipy_complex_harmonics():
    from scipy.special import sph_harm_y
    g = synth.hemisphere_directions(50, seed=7)
    g[0] = [0, 0, 1]
    theta = np.arccos(np.clip(g[:, 2], -1, 1))
    phi = np.arctan2(g[:, 1], g[:, 0])
    B = osh.real_sh(8, g)
    for l in range(0, 9, 2):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            ref = Y.real if m == 0 else (np.sqrt(2) * Y.real if m < 0 else np.sqrt(2) * Y.imag)
            np.testing.assert_allclose(B[:, osh.sh_index(l, m)], ref, rtol=0, atol=1e-13)


def test_addition_theorem_and_y0():
    g = synth.hemisphere_directions(40, seed=3)
    B = osh.real_sh(8, g)
    np.testing.assert_allclose(B[:, 0], 1 / np.sqrt(4 * np.pi), atol=1e-15)
    l, _ = osh.sh_lm(8)
    for band in range(0, 9, 2):
        np.testing.assert_allclose((B[:, l == band] ** 2).sum(1), (2 * band + 1) / (4 * np.pi), atol=1e-13)


def test_pinv_routes_agree():
    g = synth.hemisphere_directions(60, seed=11)
    B = osh.real_sh(8, g)
    for lam in (0.0, 0.006, 0.06, 1.0):
        np.testing.assert_allclose(osh.pinv_normal(B, 8, lam), osh.pinv_qr(B, 8, lam), atol=1e-11, rtol=0)


def test_exact_recovery_of_band_limited_signal():
    g = synth.hemisphere_directions(60, seed=12)
    B = osh.real_sh(8, g)
    c = synth.gaussian(45, 1.0, seed=5, tag="coeffs")
    c_hat = osh.pinv_normal(B, 8, 0.0) @ (B @ c)
    assert np.linalg.norm(c_hat - c) / np.linalg.norm(c) < 1e-12


def test_constant_signal_recovered_for_any_lambda():
    g = synth.hemisphere_directions(30, seed=13)
    B = osh.real_sh(4, g)
    e0 = np.zeros(15)
    e0[0] = np.sqrt(4 * np.pi)
    for lam in (0.0, 0.006, 0.06, 5.0):
        np.testing.assert_allclose(osh.pinv_normal(B, 4, lam) @ np.ones(30), e0, atol=1e-12)


def test_projector_properties():
    g = synth.hemisphere_directions(60, seed=14)
    B = osh.real_sh(8, g)
    H = B @ osh.pinv_normal(B, 8, 0.0)
    np.testing.assert_allclose(H @ H, H, atol=1e-12)
    np.testing.assert_allclose(H, H.T, atol=1e-12)
    assert abs(np.trace(H) - 45) < 1e-10
    Hl = B @ osh.pinv_normal(B, 8, 0.006)
    np.testing.assert_allclose(Hl, Hl.T, atol=1e-12)
    ev = np.linalg.eigvalsh(Hl)
    assert ev.min() > -1e-12 and ev.max() <= 1 + 1e-12
    nz = ev[ev > 1e-9]
    assert len(nz) == 45 and np.all(nz <= 1 + 1e-12) and np.trace(Hl) < 45 - 1e-3


def test_penalty_closed_form_on_equal_weight_design():
    """Six half-icosahedron directions integrate even degree-4 products exactly, so
    B^T B = (6/4pi) I at order 2 and P B = diag((6/4pi) / (6/4pi + lambda l^2 (l+1)^2))."""
    B = osh.real_sh(2, ICOSA_HALF)
    a = 6 / (4 * np.pi)
    np.testing.assert_allclose(B.T @ B, a * np.eye(6), atol=1e-13)
    for lam in (0.006, 0.06, 0.5):
        expect = np.array([a / (a + lam * (l * (l + 1)) ** 2) for l in (0, 2, 2, 2, 2, 2)])
        np.testing.assert_allclose(osh.pinv_normal(B, 2, lam) @ B, np.diag(expect), atol=1e-13)


def test_rotation_invariance_of_band_power():
    g = synth.hemisphere_directions(60, seed=15)
    s = synth.gaussian(60, 1.0, seed=2, tag="coeffs")
    R = synth.random_rotation(1.0, seed=9)
    l, _ = osh.sh_lm(8)
    for lam in (0.0, 0.006, 0.06):
        c = osh.pinv_normal(osh.real_sh(8, g), 8, lam) @ s
        c2 = osh.pinv_normal(osh.real_sh(8, g @ R.T), 8, lam) @ s
        for band in range(0, 9, 2):
            np.testing.assert_allclose((c[l == band] ** 2).sum(), (c2[l == band] ** 2).sum(), rtol=1e-11)
        # and the rotated fit is not trivially the same coefficient vector
        assert np.linalg.norm(c - c2) > 1e-3


def test_antipodal_doubling_halves_lambda():
    g = synth.hemisphere_directions(40, seed=16)
    s = synth.gaussian(40, 1.0, seed=3, tag="coeffs")
    B = osh.real_sh(6, g)
    B2 = osh.real_sh(6, np.vstack([g, -g]))
    for lam in (0.0, 0.006, 0.2):
        np.testing.assert_allclose(osh.pinv_normal(B2, 6, lam) @ np.concatenate([s, s]),
                                   osh.pinv_normal(B, 6, lam / 2) @ s, atol=1e-12)


def test_shell_grouping_and_round_trips():
    dirs, bvals = synth.multishell_table([20, 30, 25], [3000, 1000, 2000], seed=4)
    ob = osh.SHBasisOracle(dirs, bvals, 4, 0.0)
    assert list(ob.shell_b) == [1000, 2000, 3000] and ob.m == [30, 25, 20]
    assert list(ob.rows[0]) == list(range(20, 50))
    c = synth.gaussian((3, 3, 15), 1.0, seed=1, tag="coeffs")
    # Signal2SH o SH2Signal = identity at lambda = 0 on the same directions
    np.testing.assert_allclose(ob.signal2sh(ob.sh2signal(c)), c, atol=1e-11)
    # SH2Signal o Signal2SH = H (the hat matrix) per shell
    s = synth.fibre_signal(dirs, bvals, 3, seed=2).astype(np.float64)
    back = ob.sh2signal(ob.signal2sh(s))
    for r, B, P in zip(ob.rows, ob.B, ob.P):
        np.testing.assert_allclose(back[:, r], s[:, r] @ (B @ P).T, atol=1e-12)
    with pytest.raises(ValueError):
        osh.group_shells(np.array([0.0, 1000.0]))


def test_transform_adjoints():
    dirs, bvals = synth.multishell_table([40, 40], [1000, 2000], seed=5)
    ob = osh.SHBasisOracle(dirs, bvals, 6, 0.006)
    x = synth.gaussian((4, 80), 1.0, seed=1, tag="coeffs")
    y = synth.gaussian((4, 2, 28), 1.0, seed=2, tag="coeffs")
    assert abs(np.sum(ob.signal2sh(x) * y) - np.sum(x * ob.signal2sh_backward(y))) < 1e-11
    assert abs(np.sum(ob.sh2signal(y) * x) - np.sum(y * ob.sh2signal_backward(x))) < 1e-11
