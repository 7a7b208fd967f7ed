"""Pins of the FP64 LSC oracle against facts fixed outside the oracle.

* geometry: unit norm, exact polar angles and azimuth spacing, frame rule;
* identity: a centre-only delta kernel reproduces the input (Sec. 2.3 layer with
  the output projection of the same table);
* Funk-Hecke: a ring-uniform kernel acts per band as multiplication by
  w_0 + sum_r w_r P_l(cos theta_r) (Legendre polynomials from numpy), which
  includes the paper's moving-average example (n = 5, alpha = pi/5, weights 1/6);
* order 0: the layer reduces to a kernel sum plus sqrt(4 pi) times the bias, for any lambda;
* brute force: kernel-point sums of a closed-form band-limited function;
* the algebraically collapsed route equals the literal route;
* gradients against central finite differences and the adjoint identity.
"""
import json
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import lsc as olsc
from oracle import sh as osh
from paper_1808_01517_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def legendre_p(l, x):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return npleg.legval(x, c)


def test_kernel_geometry():
    g = synth.hemisphere_directions(30, seed=21)
    R, Sec, alpha = 4, 12, np.deg2rad(25)
    P = olsc.kernel_points(g, alpha, R, Sec)
    assert P.shape == (30, 49, 3)
    np.testing.assert_allclose(np.linalg.norm(P, axis=2), 1.0, atol=1e-14)
    np.testing.assert_allclose(P[:, 0], g, atol=0)
    for i in range(30):
        e1, e2 = olsc.tangent_frame(g[i])
        k = int(np.argmin(np.abs(g[i])))
        # e1 is orthogonal to g and lies in the plane of g and the chosen axis
        assert abs(e1 @ g[i]) < 1e-15 and abs(np.cross(g[i], np.eye(3)[k]) @ e1) < 1e-14
        for r in range(1, R + 1):
            ring = P[i, 1 + (r - 1) * Sec: 1 + r * Sec]
            np.testing.assert_allclose(ring @ g[i], np.cos(r * alpha / R), atol=1e-14)
            t = ring - np.outer(ring @ g[i], g[i])
            az = np.arctan2(t @ e2, t @ e1)
            diff = az - 2 * np.pi * np.arange(Sec) / Sec
            np.testing.assert_allclose(np.sin(diff), 0.0, atol=1e-12)
            np.testing.assert_allclose(np.cos(diff), 1.0, atol=1e-12)


def test_tables_t2_t3_t4():
    np.testing.assert_array_equal(olsc.shell_window(3, 3, "adjacent"),
                                  [[1, 1, 0], [1, 1, 1], [0, 1, 1]])
    np.testing.assert_array_equal(olsc.shell_window(2, 2, "same"), np.eye(2, dtype=bool))
    assert olsc.shell_window(3, 1, "all").shape == (3, 1)
    with pytest.raises(ValueError):
        olsc.shell_window(3, 1, "adjacent")
    # octahedron axes + a diagonal: hand-checked neighbour sets
    g = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1] / np.sqrt(3)])
    ip, ix = olsc.neighbour_csr(g, np.deg2rad(30))
    assert list(ip) == [0, 1, 2, 3, 4] and list(ix) == [0, 1, 2, 3]
    ip, ix = olsc.neighbour_csr(g, np.deg2rad(60))  # axis-to-diagonal angle is 54.7 deg
    assert list(ix[ip[0]:ip[1]]) == [0, 3] and list(ix[ip[3]:ip[4]]) == [0, 1, 2, 3]
    # antipodal awareness: -g counts as g
    ip, ix = olsc.neighbour_csr(np.array([[0, 0, 1.0], [0, 0.1, -1.0] / np.linalg.norm([0, .1, -1])]),
                                np.deg2rad(10))
    assert list(ix) == [0, 1, 0, 1]
    T4 = olsc.kernel_row_index([3, 2], 5)
    assert T4.shape == (5, 5) and T4[3, 2] == 17
    m = np.zeros((3, 4, 5), bool)
    m[1, 2, 3] = m[0, 0, 1] = True
    np.testing.assert_array_equal(olsc.mask_to_index(m), [1, 1 * 20 + 2 * 5 + 3])


def _single_shell(m, order, lam, seed):
    g = synth.hemisphere_directions(m, seed=seed)
    return osh.SHBasisOracle(g, np.full(m, 1000.0), order, lam)


def test_identity_for_centre_only_kernel():
    ob = _single_shell(60, 8, 0.0, 31)
    L = olsc.LSCOracle(ob, 8, 1, np.deg2rad(30), 3, 8)
    c = synth.gaussian((5, 1, 1, 45), 1.0, seed=1, tag="coeffs")
    w = np.zeros((1, 1, 1, 1, 25))
    w[..., 0] = 1.0
    np.testing.assert_allclose(L.forward(c, w, np.zeros((1, 1))), c, atol=1e-11)
    # with lambda > 0 the delta kernel is SH2Signal followed by Signal2SH
    ob2 = osh.SHBasisOracle(ob.dirs, np.full(60, 1000.0), 8, 0.006)
    L2 = olsc.LSCOracle(ob2, 8, 1, np.deg2rad(30), 3, 8)
    np.testing.assert_allclose(L2.forward(c, w, np.zeros((1, 1))), ob2.signal2sh(ob2.sh2signal(c)),
                               atol=1e-11)


def test_order_zero_is_a_kernel_sum_for_any_lambda():
    """Order 0 (one coefficient per shell): the interpolant is the constant c / sqrt(4 pi) at
    every kernel point, so each output direction carries sum_k w c / sqrt(4 pi) + b, and the
    projection of a constant recovers it exactly for any lambda (the penalty vanishes on
    l = 0).  Closed form: c_out = sum_{ci, s' in win(s), k} w c + sqrt(4 pi) b."""
    dirs, bvals = synth.multishell_table([20, 30], [1000, 2000], seed=7)
    for lam in (0.0, 0.06):
        ob = osh.SHBasisOracle(dirs, bvals, 0, lam)
        lsc = olsc.LSCOracle(ob, 0, 2, np.deg2rad(20), 2, 6, "adjacent")
        c = synth.gaussian((4, 3, 2, 1), 1.0, seed=3, tag="coeffs")
        w = synth.gaussian((5, 2, 3, 2, lsc.K), 0.1, seed=4)
        b = synth.gaussian((5, 2), 0.1, seed=5)
        want = np.einsum("osipk,vip->vos", w, c[..., 0])[..., None] + np.sqrt(4 * np.pi) * b[None, :, :, None]
        np.testing.assert_allclose(lsc.forward(c, w, b), want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("R,Sec,alpha,L", [(1, 5, np.pi / 5, 4), (3, 9, np.deg2rad(30), 8),
                                           (4, 12, np.deg2rad(25), 8)])
def test_funk_hecke_ring_uniform_kernel(R, Sec, alpha, L):
    ob = _single_shell(90, L, 0.0, 32)
    lsc = olsc.LSCOracle(ob, L, 1, alpha, R, Sec)
    w0 = 0.3
    wr = np.linspace(0.5, -0.2, R)
    w = np.zeros((1, 1, 1, 1, lsc.K))
    w[..., 0] = w0
    for r in range(R):
        w[..., 1 + r * Sec: 1 + (r + 1) * Sec] = wr[r] / Sec
    lvals, _ = osh.sh_lm(L)
    mu = np.array([w0 + sum(wr[r] * legendre_p(l, np.cos((r + 1) * alpha / R)) for r in range(R))
                   for l in lvals])
    c = synth.gaussian((3, 1, 1, osh.n_coef(L)), 1.0, seed=2, tag="coeffs")
    np.testing.assert_allclose(lsc.forward(c, w, np.zeros((1, 1))), c * mu, atol=1e-11)


def test_paper_moving_average_example():
    """The paper's LSC example (Sec. 2.3): order 4, kernel_sizes [5], alpha = pi/5,
    uniform weights 1/6, bias 0.  On a table dense enough to be exact at lambda = 0
    the layer scales band l by 1/6 + 5/6 P_l(cos pi/5): a low-pass ("blurred") filter."""
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        ex = json.load(f)["lsc_moving_average"]
    assert ex["kernel_sizes"] == [5] and ex["weights"] == [1, 1, 1, 1, 1, 1]
    ob = _single_shell(60, ex["sh_order"], 0.0, 33)
    lsc = olsc.LSCOracle(ob, ex["sh_order"], 1, np.pi * ex["angular_distance_over_pi"], 1,
                         ex["kernel_sizes"][0])
    w = np.array(ex["weights"], np.float64).reshape(1, 1, 1, 1, 6)
    w /= w.sum()
    mu = {l: 1 / 6 + 5 / 6 * legendre_p(l, np.cos(np.pi / 5)) for l in (0, 2, 4)}
    assert mu[0] == pytest.approx(1.0) and 1 > mu[2] > abs(mu[4])
    lvals, _ = osh.sh_lm(4)
    c = synth.gaussian((2, 1, 1, 15), 1.0, seed=3, tag="coeffs")
    out = lsc.forward(c, w, np.array([[ex["bias"]]], np.float64))
    np.testing.assert_allclose(out, c * np.array([mu[l] for l in lvals]), atol=1e-12)


def test_brute_force_kernel_sums_on_tiny_sphere():
    """Resampling equals exact evaluation of a closed-form band-limited function."""
    g = synth.hemisphere_directions(8, seed=34)
    ob = osh.SHBasisOracle(g, np.full(8, 1000.0), 2, 0.05)
    lsc = olsc.LSCOracle(ob, 2, 1, np.deg2rad(20), 2, 3)
    funcs = [lambda p: p[..., 0] ** 2, lambda p: p[..., 0] * p[..., 1], lambda p: 1 + p[..., 2] ** 2 - p[..., 1] * p[..., 2]]
    # SH coefficients of each f by exact quadrature (independent of the pseudo-inverse)
    from tests.test_oracle_sh import product_quadrature
    qd, qw = product_quadrature(2)
    Bq = osh.real_sh(2, qd)
    c = np.stack([Bq.T @ (qw * f(qd)) for f in funcs])[:, None, None, :]  # [3, 1, 1, 6]
    w = synth.gaussian((1, 1, 1, 1, 7), 0.5, seed=4)
    b = np.array([[0.25]])
    y = lsc.direction_space(c, w, b)[0]  # [v, 1, i]
    for v, f in enumerate(funcs):
        for i in range(8):
            manual = sum(w[0, 0, 0, 0, k] * f(lsc.kpts[0][i, k]) for k in range(7)) + 0.25
            assert abs(y[v, 0, i] - manual) < 1e-12
    np.testing.assert_allclose(lsc.forward(c, w, b)[:, 0, 0], y[:, 0] @ ob.P[0].T, atol=1e-13)


def _multishell_lsc(window="adjacent", order_in=4, order_out=4, lam=0.006, m=(30, 30, 30), seed=40):
    dirs, bvals = synth.multishell_table(list(m), [1000, 2000, 3000][:len(m)], seed=seed)
    ob = osh.SHBasisOracle(dirs, bvals, order_out, lam)
    s_in = len(m) if window != "all" else 2
    return olsc.LSCOracle(ob, order_in, s_in, np.deg2rad(25), 2, 6, window)


@pytest.mark.parametrize("window,order_in", [("adjacent", 4), ("same", 4), ("all", 2), ("all", 6)])
def test_collapsed_route_equals_literal(window, order_in):
    lsc = _multishell_lsc(window, order_in=order_in)
    Ci, Co = 3, 2
    c = synth.gaussian((4, Ci, lsc.s_in, lsc.n_in), 1.0, seed=5, tag="coeffs")
    w = synth.gaussian((Co, lsc.s_out, Ci, lsc.s_in, lsc.K), 0.1, seed=6)
    b = synth.gaussian((Co, lsc.s_out), 0.1, seed=7)
    np.testing.assert_allclose(lsc.forward_collapsed(c, w, b), lsc.forward(c, w, b), atol=1e-12)


def test_shell_window_masks_weights():
    lsc = _multishell_lsc("adjacent")
    c = synth.gaussian((3, 2, 3, 15), 1.0, seed=8, tag="coeffs")
    w = synth.gaussian((2, 3, 2, 3, lsc.K), 0.1, seed=9)
    b = np.zeros((2, 3))
    w2 = w.copy()
    w2[:, 0, :, 2] = 5.0  # outside the window: must not matter
    w2[:, 2, :, 0] = -3.0
    np.testing.assert_allclose(lsc.forward(c, w2, b), lsc.forward(c, w, b), atol=0)
    # only the (s=1, s'=2) block active: output shells 0 and 2 see just the bias (0)
    w3 = np.zeros_like(w)
    w3[:, 1, :, 2] = w[:, 1, :, 2]
    out = lsc.forward(c, w3, b)
    assert np.all(out[:, :, [0, 2]] == 0) and np.linalg.norm(out[:, :, 1]) > 0
    c2 = c.copy()
    c2[:, :, [0, 1]] = 0
    np.testing.assert_allclose(lsc.forward(c2, w3, b), out, atol=1e-13)


def test_backward_matches_finite_differences_and_adjoint():
    lsc = _multishell_lsc("adjacent", order_in=4, order_out=6)
    Ci, Co, V = 2, 3, 4
    c = synth.gaussian((V, Ci, 3, 15), 1.0, seed=10, tag="coeffs")
    w = synth.gaussian((Co, 3, Ci, 3, lsc.K), 0.1, seed=11)
    b = synth.gaussian((Co, 3), 0.1, seed=12)
    d = synth.gaussian((V, Co, 3, 28), 1.0, seed=13, tag="grads")
    dc, dw, db = lsc.backward(c, w, d)

    def loss(c_, w_, b_):
        return float(np.sum(lsc.forward(c_, w_, b_) * d))

    rng = np.random.default_rng(0)
    for _ in range(3):
        for name, x, g in (("c", c, dc), ("w", w, dw), ("b", b, db)):
            dx = rng.standard_normal(x.shape)
            if name == "w":
                dx *= lsc.win[None, :, None, :, None]
            h = 1e-6 * np.linalg.norm(x) / np.linalg.norm(dx)
            args_p = {"c": c, "w": w, "b": b}
            args_m = dict(args_p)
            args_p[name] = x + h * dx
            args_m[name] = x - h * dx
            fd = (loss(args_p["c"], args_p["w"], args_p["b"]) - loss(args_m["c"], args_m["w"], args_m["b"])) / (2 * h)
            an = float(np.sum(g * dx))
            assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (name, fd, an)
    # adjoint in the input: <LSC_0 c, d> = <c, dc> with the bias off
    lin = float(np.sum(lsc.forward(c, w, np.zeros_like(b)) * d))
    assert abs(lin - float(np.sum(c * dc))) < 1e-10 * max(1.0, abs(lin))
    # outside-window weight gradients are exactly zero
    assert np.all(dw[:, 0, :, 2] == 0) and np.all(dw[:, 2, :, 0] == 0)


@pytest.mark.parametrize("R,Sec,alpha,L", [(2, 9, np.deg2rad(30), 8), (4, 12, np.deg2rad(25), 8),
                                           (1, 5, np.pi / 5, 4)])
def test_ring_tied_kernel_is_band_scaling(R, Sec, alpha, L):
    """Ring-tied weights (origin + one per ring) through the literal LSC equal the band
    multipliers w0 + Sec sum_r w_r P_l(cos theta_r) at lambda = 0 when Sec > L, for
    several channels and a random table: the layer does not see the tangent frames."""
    ob = _single_shell(90, L, 0.0, 35)
    lsc = olsc.LSCOracle(ob, L, 1, alpha, R, Sec)
    w_ring = synth.gaussian((2, 1, 3, 1, R + 1), 0.2, seed=11)
    w = olsc.ring_expand(w_ring, R, Sec)
    assert w.shape[-1] == lsc.K
    c = synth.gaussian((5, 3, 1, osh.n_coef(L)), 1.0, seed=12, tag="coeffs")
    mu = olsc.ring_band_multipliers(w_ring, L, alpha, R, Sec)  # [co, s, ci, s', j]
    ref = np.einsum("oscpj,vcpj->vosj", mu, c)
    np.testing.assert_allclose(lsc.forward(c, w, np.zeros((2, 1))), ref, atol=1e-10)


def test_ring_expand_reduce_adjoint():
    w_ring = synth.gaussian((3, 2, 4, 2, 5), 1.0, seed=13)
    dw = synth.gaussian((3, 2, 4, 2, 1 + 4 * 7), 1.0, seed=14)
    lhs = np.sum(olsc.ring_expand(w_ring, 4, 7) * dw)
    rhs = np.sum(w_ring * olsc.ring_reduce(dw, 4, 7))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # each ring's points carry the ring's weight
    w = olsc.ring_expand(w_ring, 4, 7)
    assert np.all(w[..., 0] == w_ring[..., 0]) and np.all(w[..., 1 + 7 * 2: 1 + 7 * 3] == w_ring[..., 3:4])
