"""The oracle's pins catch plausible mistakes: each case plants one mistake in the
oracle (a dropped term or factor, a wrong sign, index or axis, a transposed operand)
and runs the pins that guard that part; at least one of them must fail.

Mistakes are planted on the CPU, in the oracle only, through pytest's monkeypatch
(undone after each case).  The pins are the functions of tests/test_oracle_*.py,
called directly.
"""
import numpy as np
import pytest

from oracle import lsc as olsc
from oracle import sh as osh
from tests import test_oracle_lsc as pl
from tests import test_oracle_lsc_neighbours as pn
from tests import test_oracle_sh as ps


def _patch_real_sh(mp, fn):
    # oracle.lsc binds real_sh by name: plant the mistake in both namespaces
    mp.setattr(osh, "real_sh", fn)
    mp.setattr(olsc, "real_sh", fn)


def no_condon_shortley(mp):
    orig = osh.assoc_legendre
    mp.setattr(osh, "assoc_legendre", lambda l, m, x: (-1.0) ** m * orig(l, m, x))


def cos_sin_swapped(mp):
    orig = osh.real_sh

    def swapped(order, dirs):
        B = orig(order, dirs)
        out = B.copy()
        for l in range(0, order + 1, 2):
            for m in range(1, l + 1):
                out[:, osh.sh_index(l, m)] = B[:, osh.sh_index(l, -m)]
                out[:, osh.sh_index(l, -m)] = B[:, osh.sh_index(l, m)]
        return out
    _patch_real_sh(mp, swapped)


def norm_without_4pi(mp):
    from math import factorial, sqrt
    mp.setattr(osh, "_norm", lambda l, m: sqrt((2 * l + 1) * factorial(l - m) / factorial(l + m)))


def penalty_not_squared(mp):
    mp.setattr(osh, "lb_penalty", lambda order: osh.sh_lm(order)[0] * (osh.sh_lm(order)[0] + 1.0))


def ridge_penalty(mp):
    mp.setattr(osh, "lb_penalty", lambda order: np.ones(osh.n_coef(order)))


def lambda_dropped(mp):
    orig = osh.pinv_normal
    mp.setattr(osh, "pinv_normal", lambda B, order, lam: orig(B, order, 0.0))


def signal2sh_adjoint_transposed(mp):
    def wrong(self, d_sh):
        out = np.empty(d_sh.shape[:-2] + (self.dirs.shape[0],))
        for s, (r, B) in enumerate(zip(self.rows, self.B)):
            out[..., r] = d_sh[..., s, :] @ B.T  # B in place of P
        return out
    mp.setattr(osh.SHBasisOracle, "signal2sh_backward", wrong)


def frame_largest_axis(mp):
    def wrong(g):
        g = np.asarray(g, np.float64)
        a = np.zeros(3)
        a[int(np.argmax(np.abs(g)))] = 1.0
        e1 = a - np.dot(a, g) * g
        e1 /= np.linalg.norm(e1)
        return e1, np.cross(g, e1)
    mp.setattr(olsc, "tangent_frame", wrong)


def ring_angle_off_by_one(mp):
    orig = olsc.kernel_points
    mp.setattr(olsc, "kernel_points",
               lambda dirs, radius, rings, sectors: orig(dirs, radius * rings / (rings + 1), rings, sectors))


def sector_azimuth_off_by_one(mp):
    def wrong(dirs, radius, rings, sectors):
        dirs = np.asarray(dirs, np.float64)
        out = np.empty((dirs.shape[0], 1 + rings * sectors, 3))
        for i, g in enumerate(dirs):
            e1, e2 = olsc.tangent_frame(g)
            out[i, 0] = g
            for r in range(1, rings + 1):
                th = r * radius / rings
                for q in range(sectors):
                    ph = 2.0 * np.pi * q / (sectors + 1)
                    out[i, 1 + (r - 1) * sectors + q] = np.cos(th) * g + np.sin(th) * (np.cos(ph) * e1 + np.sin(ph) * e2)
        return out
    mp.setattr(olsc, "kernel_points", wrong)


def window_two_wide(mp):
    orig = olsc.shell_window

    def wrong(s_out, s_in, mode):
        if mode == "adjacent":
            s = np.arange(s_out)
            return np.abs(s[:, None] - s[None, :]) <= 2
        return orig(s_out, s_in, mode)
    mp.setattr(olsc, "shell_window", wrong)


def neighbours_not_antipodal(mp):
    def wrong(dirs, radius):
        g = np.asarray(dirs, np.float64)
        c = np.cos(radius)
        indptr, idx = [0], []
        for i in range(g.shape[0]):
            idx.extend(j for j in range(g.shape[0]) if float(np.dot(g[i], g[j])) >= c)
            indptr.append(len(idx))
        return np.array(indptr, np.int64), np.array(idx, np.int64)
    mp.setattr(olsc, "neighbour_csr", wrong)


def bias_dropped(mp):
    orig = olsc.LSCOracle.direction_space
    mp.setattr(olsc.LSCOracle, "direction_space", lambda self, c, w, b: orig(self, c, w, np.zeros_like(b)))


def bias_projection_wrong_axis(mp):
    orig = olsc.LSCOracle.collapse_mats

    def wrong(self):
        M, _ = orig(self)
        return M, [P[:, :1].sum(axis=1) * np.ones(P.shape[0]) for P in self.Pout]  # first column only
    mp.setattr(olsc.LSCOracle, "collapse_mats", wrong)


def weight_gradient_unmasked(mp):
    orig = olsc.LSCOracle.backward

    def wrong(self, c_in, w, d_out):
        dc, dw, db = orig(self, c_in, w, d_out)
        for s in range(self.s_out):  # the window mask left off dw: fill the masked entries
            U = self.resample(c_in, s)
            dy = d_out[:, :, s, :] @ self.Pout[s]
            dw[:, s] = np.einsum("vai,vcpik->acpk", dy, U, optimize=True)
        return dc, dw, db
    mp.setattr(olsc.LSCOracle, "backward", wrong)


def resample_adjoint_wrong_shell(mp):
    def wrong(self, dU, s):
        return np.einsum("ikj,vcpik->vcpj", self.BK[(s + 1) % len(self.BK)], dU, optimize=True)
    mp.setattr(olsc.LSCOracle, "resample_adjoint", wrong)


def ring_reduce_mean(mp):
    orig = olsc.ring_reduce
    mp.setattr(olsc, "ring_reduce", lambda dw, rings, sectors: np.concatenate(
        [orig(dw, rings, sectors)[..., :1], orig(dw, rings, sectors)[..., 1:] / sectors], axis=-1))


def band_multiplier_without_sector_factor(mp):
    orig = olsc.ring_band_multipliers

    def wrong(w_ring, order, radius, rings, sectors):
        w = np.asarray(w_ring, np.float64).copy()
        w[..., 1:] /= sectors
        return orig(w, order, radius, rings, sectors)
    mp.setattr(olsc, "ring_band_multipliers", wrong)


def neighbour_not_oriented(mp):
    def wrong(g_i, kpts_i, dirs_in, radius):
        c = np.cos(radius)
        idx, bins = [], []
        for j in range(dirs_in.shape[0]):
            if abs(float(np.dot(g_i, dirs_in[j]))) >= c:
                idx.append(j)
                bins.append(int(np.argmax(kpts_i @ dirs_in[j])))  # -g_j not flipped
        return np.array(idx, np.int64), np.array(bins, np.int64)
    mp.setattr(olsc, "neighbour_bins", wrong)


def neighbour_sum_not_mean(mp):
    orig = olsc.LSCNeighbourOracle.__init__

    def wrong(self, *a, **k):
        orig(self, *a, **k)
        for key in self.A:
            self.A[key] = (self.A[key] > 0).astype(np.float64)
    mp.setattr(olsc.LSCNeighbourOracle, "__init__", wrong)


SH_PINS = [ps.test_basis_matches_scipy_complex_harmonics, lambda: ps.test_basis_orthonormal_under_exact_quadrature(8),
           ps.test_addition_theorem_and_y0, ps.test_pinv_routes_agree, ps.test_constant_signal_recovered_for_any_lambda,
           ps.test_projector_properties, ps.test_penalty_closed_form_on_equal_weight_design,
           ps.test_transform_adjoints]
GEOM_PINS = [pl.test_kernel_geometry, lambda: pl.test_funk_hecke_ring_uniform_kernel(3, 9, np.deg2rad(30), 8),
             pl.test_paper_moving_average_example, pl.test_brute_force_kernel_sums_on_tiny_sphere]
LSC_PINS = [pl.test_identity_for_centre_only_kernel, pl.test_order_zero_is_a_kernel_sum_for_any_lambda,
            lambda: pl.test_collapsed_route_equals_literal("adjacent", 4), pl.test_shell_window_masks_weights,
            pl.test_backward_matches_finite_differences_and_adjoint]
RING_PINS = [lambda: pl.test_ring_tied_kernel_is_band_scaling(2, 9, np.deg2rad(30), 8),
             pl.test_ring_expand_reduce_adjoint]
NB_PINS = [lambda: pn.test_bins_are_nearest_kernel_points(np.deg2rad(25), 4, 12),
           pn.test_identity_below_the_smallest_angle, lambda: pn.test_constant_signal_counts_occupied_kernel_points("same"),
           pn.test_brute_force_means_on_tiny_table, pn.test_backward_matches_finite_differences_and_adjoint]

MUTANTS = {
    "basis: Condon-Shortley phase dropped": (no_condon_shortley, SH_PINS),
    "basis: cos and sin halves swapped": (cos_sin_swapped, SH_PINS),
    "basis: 4 pi dropped from the normalisation": (norm_without_4pi, SH_PINS),
    "pseudo-inverse: penalty l(l+1) not squared": (penalty_not_squared, SH_PINS),
    "pseudo-inverse: ridge penalty in place of Laplace-Beltrami": (ridge_penalty, SH_PINS),
    "pseudo-inverse: lambda dropped": (lambda_dropped, SH_PINS),
    "Signal2SH adjoint: B in place of P": (signal2sh_adjoint_transposed, SH_PINS),
    "kernel: frame from the largest axis": (frame_largest_axis, GEOM_PINS),
    "kernel: ring angles r alpha / (R + 1)": (ring_angle_off_by_one, GEOM_PINS),
    "kernel: azimuths 2 pi q / (Sec + 1)": (sector_azimuth_off_by_one, GEOM_PINS),
    "T2: adjacent window two shells wide": (window_two_wide, [pl.test_tables_t2_t3_t4] + LSC_PINS),
    "T3: neighbours not antipodal": (neighbours_not_antipodal, [pl.test_tables_t2_t3_t4]),
    "LSC: bias dropped": (bias_dropped, LSC_PINS),
    "LSC collapse: bias projection from one column": (bias_projection_wrong_axis, LSC_PINS),
    "LSC backward: window mask left off dw": (weight_gradient_unmasked, LSC_PINS),
    "LSC backward: adjoint resampling of another shell": (resample_adjoint_wrong_shell, LSC_PINS),
    "ring-tied: reduce by mean not sum": (ring_reduce_mean, RING_PINS),
    "ring-tied: band multipliers without the sector factor": (band_multiplier_without_sector_factor, RING_PINS),
    "resampling-free: antipodal neighbour not oriented": (neighbour_not_oriented, NB_PINS),
    "resampling-free: sum in place of the bin mean": (neighbour_sum_not_mean, NB_PINS),
}


def _outcomes(pins):
    """Per pin: None (passed), or the type of what it raised."""
    out = []
    for pin in pins:
        try:
            pin()
            out.append(None)
        except Exception as e:
            out.append(type(e))
    return out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    plant, pins = MUTANTS[name]
    plant(monkeypatch)
    # caught by a pin's assertion, not only by an error the planted code happens to raise
    assert AssertionError in _outcomes(pins), f"no pin caught: {name}"


def test_pins_pass_on_the_oracle_as_written():
    """The same pin lists with nothing planted: every pin passes."""
    for pins in (SH_PINS, GEOM_PINS, LSC_PINS, RING_PINS, NB_PINS, [pl.test_tables_t2_t3_t4]):
        assert _outcomes(pins) == [None] * len(pins)
