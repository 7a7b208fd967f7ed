"""The Python layers' interface against the paper's usage examples (Sec. 2.2 and 2.3), on
the CPU: the parameter names the examples use, the kernel-vector length n + 1 their
values give, and the 5-D activation layout of Sec. 2.1 (subjects x features x H x W x D)
mapped to the library's feature-rows x voxel-columns layout and back."""
import inspect
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_1808_01517_gb300 import _lib as L
from paper_1808_01517_gb300 import layers, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")


def _params(cls):
    return set(inspect.signature(cls.__init__).parameters)


def test_layers_take_the_papers_parameter_names():
    assert {"sh_order", "gradients", "lb_lambda"} <= _params(layers.Signal2SH)
    assert {"sh_order", "gradients"} <= _params(layers.SH2Signal)
    assert {"shells_in", "shells_out", "sampled_gradients", "sh_order_in", "sh_order_out", "kernel_sizes",
            "lb_lambda", "angular_distance"} <= _params(layers.LocalSphericalConvolution)


def test_example_values_give_the_papers_kernel_vector():
    """kernel_sizes [5] and angular_distance pi/5: one ring of five points around the
    origin, a kernel vector of n + 1 = 6 weights (the example's [1, 1, 1, n + 1] conv
    weight), on the example's order and lambda."""
    with open(GOLDEN) as f:
        ex = json.load(f)
    s2sh, lsc = ex["signal2sh_example"], ex["lsc_moving_average"]
    dirs, bvals = synth.multishell_table([60], [1000], seed=5)
    basis = L.SHBasis(dirs, bvals, s2sh["sh_order"], s2sh["lb_lambda"], host_only=True)
    assert basis.n_coef == 15
    out = L.SHBasis(dirs, bvals, lsc["sh_order"], lsc["lb_lambda"], host_only=True)
    ks = lsc["kernel_sizes"]
    geom = L.LSCGeometry(out, lsc["sh_order"], lsc["shells_in"], math.pi * lsc["angular_distance_over_pi"], len(ks),
                         ks[0], "same", host_only=True)
    assert geom.K == len(lsc["weights"]) == ks[0] + 1
    kp = geom.tables(0)["kpts"]
    g = dirs[0]
    # origin first, then the ring at angular distance alpha (one ring: theta_1 = alpha)
    np.testing.assert_allclose(kp[0, 0], g, atol=1e-15)
    np.testing.assert_allclose(kp[0, 1:] @ g, math.cos(math.pi / 5), atol=1e-14)


def test_five_dimensional_layout_round_trip():
    B, F, H, W, D = 2, 3, 4, 5, 6
    x = torch.arange(B * F * H * W * D, dtype=torch.float32).reshape(B, F, H, W, D)
    flat, restore = layers._to_rows(x)
    assert flat.shape == (F, B * H * W * D)
    b, f, h, w, d = 1, 2, 3, 1, 4
    assert flat[f, ((b * H + h) * W + w) * D + d] == x[b, f, h, w, d]
    assert torch.equal(restore(flat), x)
    y = torch.zeros(7, B * H * W * D)  # another feature count on the way back
    assert restore(y).shape == (B, 7, H, W, D)
    two_d = torch.zeros(F, 10)
    assert layers._to_rows(two_d)[0] is two_d
    with pytest.raises(ValueError):
        layers._to_rows(torch.zeros(2, 3, 4))
