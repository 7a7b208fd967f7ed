"""Pins of the resampling-free LSC oracle (acquired neighbours binned to the nearest
kernel point, the alternative Sec. 2.3 argues against) against facts fixed outside it.

* bins: every neighbour's kernel point is the nearest one on the sphere, found here by
  a second route (polar coordinates in the tangent frame and the spherical law of
  cosines) with the neighbour test written as an angle;
* identity: with a radius below the table's smallest inter-direction angle every
  direction is its own only neighbour, so a centre-only kernel reproduces the input
  at lambda = 0;
* a constant signal with all-ones weights yields, per direction, the number of
  non-empty kernel points (a mean, not a sum, of the neighbours in each);
* brute force on a tiny table: neighbourhood means of a closed-form quadratic
  evaluated at the acquired directions;
* the collapsed route equals the literal route; gradients against central finite
  differences and the adjoint identity.
"""
import numpy as np
import pytest

from oracle import lsc as olsc
from oracle import sh as osh
from paper_1808_01517_gb300 import synth


def _polar_bins(g_i, dirs_in, radius, rings, sectors):
    """Second route: neighbours by angle, bins by spherical distance in polar form.
    Returns (indices, bins, margin) with margin the gap between the two nearest
    kernel points' cosines (ties would make the bin ambiguous)."""
    e1, e2 = olsc.tangent_frame(g_i)
    idx, bins, margin = [], [], np.inf
    for j, gj in enumerate(dirs_in):
        ang = np.arccos(np.clip(abs(float(np.dot(g_i, gj))), -1.0, 1.0))
        if ang > radius:
            continue
        u = gj * np.sign(np.dot(g_i, gj) or 1.0)
        th = np.arccos(np.clip(np.dot(g_i, u), -1.0, 1.0))
        ph = np.arctan2(np.dot(u, e2), np.dot(u, e1))
        cosd = [np.cos(th)]  # distance to the origin is th itself
        for r in range(1, rings + 1):
            tr = r * radius / rings
            for q in range(sectors):
                cosd.append(np.cos(th) * np.cos(tr) + np.sin(th) * np.sin(tr) * np.cos(ph - 2 * np.pi * q / sectors))
        cosd = np.array(cosd)
        order = np.argsort(-cosd, kind="stable")
        idx.append(j)
        bins.append(int(order[0]))
        margin = min(margin, cosd[order[0]] - cosd[order[1]])
    return idx, bins, margin


def _table(m=(30, 30, 30), order=4, lam=0.006, seed=40):
    dirs, bvals = synth.multishell_table(list(m), [1000, 2000, 3000][:len(m)], seed=seed)
    return osh.SHBasisOracle(dirs, bvals, order, lam)


@pytest.mark.parametrize("radius,R,Sec", [(np.deg2rad(25), 4, 12), (np.deg2rad(30), 3, 8), (np.pi / 5, 1, 5)])
def test_bins_are_nearest_kernel_points(radius, R, Sec):
    ob = _table(m=(40, 40, 40))
    lsc = olsc.LSCNeighbourOracle(ob, 4, 3, radius, R, Sec, "all")
    n_checked = 0
    for (s, p), (indptr, indices, bins) in lsc.nb.items():
        for i, g in enumerate(lsc.dirs[s]):
            ix, bx, margin = _polar_bins(g, lsc.dirs[p], radius, R, Sec)
            assert margin > 1e-9
            assert list(indices[indptr[i]:indptr[i + 1]]) == ix
            assert list(bins[indptr[i]:indptr[i + 1]]) == bx
            n_checked += len(ix)
    assert n_checked > 1000


def test_identity_below_the_smallest_angle():
    ob = osh.SHBasisOracle(synth.hemisphere_directions(60, seed=31), np.full(60, 1000.0), 6, 0.0)
    g = ob.dirs
    cosines = np.abs(g @ g.T)
    np.fill_diagonal(cosines, 0.0)
    radius = 0.5 * float(np.arccos(cosines.max()))
    lsc = olsc.LSCNeighbourOracle(ob, 6, 1, radius, 2, 6)
    indptr, indices, bins = lsc.nb[0, 0]
    assert np.all(np.diff(indptr) == 1) and np.all(indices == np.arange(60)) and np.all(bins == 0)
    c = synth.gaussian((4, 2, 1, 28), 1.0, seed=1, tag="coeffs")
    w = np.zeros((2, 1, 2, 1, lsc.K))
    w[0, 0, 0, 0, 0] = 1.0
    w[1, 0, 1, 0, 0] = 1.0
    np.testing.assert_allclose(lsc.forward(c, w, np.zeros((2, 1))), c, atol=1e-11)


@pytest.mark.parametrize("window", ["same", "adjacent", "all"])
def test_constant_signal_counts_occupied_kernel_points(window):
    ob = _table(m=(30, 35, 40))
    radius, R, Sec = np.deg2rad(30), 2, 6
    lsc = olsc.LSCNeighbourOracle(ob, 4, 3, radius, R, Sec, window)
    c = np.zeros((1, 1, 3, 15))
    c[..., 0] = np.sqrt(4 * np.pi)  # the constant signal 1 on every shell
    w = np.ones((1, 3, 1, 3, lsc.K))
    ys = lsc.direction_space(c, w, np.zeros((1, 3)))
    win = olsc.shell_window(3, 3, window)
    for s in range(3):
        for i, g in enumerate(lsc.dirs[s]):
            expect = sum(len(set(_polar_bins(g, lsc.dirs[p], radius, R, Sec)[1])) for p in range(3) if win[s, p])
            assert abs(ys[s][0, 0, i] - expect) < 1e-11


def test_brute_force_means_on_tiny_table():
    g = synth.hemisphere_directions(12, seed=34)
    ob = osh.SHBasisOracle(g, np.full(12, 1000.0), 2, 0.0)
    radius, R, Sec = np.deg2rad(50), 2, 3
    lsc = olsc.LSCNeighbourOracle(ob, 2, 1, radius, R, Sec)
    funcs = [lambda p: p[..., 0] ** 2, lambda p: p[..., 0] * p[..., 1],
             lambda p: 1 + p[..., 2] ** 2 - p[..., 1] * p[..., 2]]
    # exact SH coefficients of each quadratic by product quadrature (no pseudo-inverse)
    from tests.test_oracle_sh import product_quadrature
    qd, qw = product_quadrature(2)
    Bq = osh.real_sh(2, qd)
    c = np.stack([Bq.T @ (qw * f(qd)) for f in funcs])[:, None, None, :]
    w = synth.gaussian((1, 1, 1, 1, lsc.K), 0.5, seed=4)
    y = lsc.direction_space(c, w, np.array([[0.25]]))[0]
    for v, f in enumerate(funcs):
        for i in range(12):
            ix, bx, _ = _polar_bins(g[i], g, radius, R, Sec)
            manual = 0.25
            for k in set(bx):
                vals = [f(g[j]) for j, kb in zip(ix, bx) if kb == k]
                manual += w[0, 0, 0, 0, k] * sum(vals) / len(vals)
            assert abs(y[v, 0, i] - manual) < 1e-12


@pytest.mark.parametrize("window,order_in,order_out", [("adjacent", 4, 4), ("all", 2, 6), ("same", 6, 4)])
def test_collapsed_route_equals_literal(window, order_in, order_out):
    ob = _table(order=order_out)
    lsc = olsc.LSCNeighbourOracle(ob, order_in, 3, np.deg2rad(25), 2, 8, window)
    c = synth.gaussian((3, 2, 3, osh.n_coef(order_in)), 1.0, seed=20, tag="coeffs")
    w = synth.gaussian((3, 3, 2, 3, lsc.K), 0.1, seed=21)
    b = synth.gaussian((3, 3), 0.1, seed=22)
    ref = lsc.forward(c, w, b)
    np.testing.assert_allclose(lsc.forward_collapsed(c, w, b), ref, atol=1e-12 * np.abs(ref).max())


def test_backward_matches_finite_differences_and_adjoint():
    ob = _table(order=6)
    lsc = olsc.LSCNeighbourOracle(ob, 4, 3, np.deg2rad(25), 2, 8, "adjacent")
    V, Ci, Co = 4, 2, 3
    c = synth.gaussian((V, Ci, 3, 15), 1.0, seed=10, tag="coeffs")
    w = synth.gaussian((Co, 3, Ci, 3, lsc.K), 0.1, seed=11)
    b = synth.gaussian((Co, 3), 0.1, seed=12)
    d = synth.gaussian((V, Co, 3, 28), 1.0, seed=13, tag="grads")
    dc, dw, db = lsc.backward(c, w, d)

    def loss(c_, w_, b_):
        return float(np.sum(lsc.forward(c_, w_, b_) * d))

    rng = np.random.default_rng(0)
    for name, x, gr in (("c", c, dc), ("w", w, dw), ("b", b, db)):
        dx = rng.standard_normal(x.shape)
        if name == "w":
            dx *= lsc.win[None, :, None, :, None]
        h = 1e-6 * np.linalg.norm(x) / np.linalg.norm(dx)
        args_p = {"c": c, "w": w, "b": b}
        args_m = dict(args_p)
        args_p[name] = x + h * dx
        args_m[name] = x - h * dx
        fd = (loss(args_p["c"], args_p["w"], args_p["b"]) - loss(args_m["c"], args_m["w"], args_m["b"])) / (2 * h)
        an = float(np.sum(gr * dx))
        assert abs(fd - an) <= 1e-4 * max(abs(an), 1e-12), (name, fd, an)
    lin = float(np.sum(lsc.forward(c, w, np.zeros_like(b)) * d))
    assert abs(lin - float(np.sum(c * dc))) < 1e-10 * max(1.0, abs(lin))
    assert np.all(dw[:, 0, :, 2] == 0) and np.all(dw[:, 2, :, 0] == 0)


def test_needs_matching_shell_counts():
    ob = _table()
    with pytest.raises(ValueError):
        olsc.LSCNeighbourOracle(ob, 4, 2, np.deg2rad(25), 2, 8, "all")
