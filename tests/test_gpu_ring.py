"""Ring-tied (isotropic) LSC kernels through the layer (delimit_lsc_ring_expand /
_reduce around the general LSC) against the FP64 oracle: forward, input gradient,
ring-weight gradient and bias gradient; and the band-scaling identity on the GPU
(sectors above the order, lambda 0: each SH band scaled by w0 + Sec sum_r w_r P_l)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2, rows_to_sh, sh_to_rows  # noqa: E402

pytestmark = pytest.mark.gpu
DT = {"f32": torch.float32, "bf16": torch.bfloat16}
TOL = {"f32": TOL_F32, "bf16": TOL_BF16}


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("R,Sec", [(4, 12), (2, 3)])  # 3 sectors < order 8: exact only through the expansion
def test_ring_tied_layer_vs_oracle(prec, R, Sec):
    dirs, bvals = synth.multishell_table([40, 40, 40], [1000, 2000, 3000], seed=17)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    rad = np.deg2rad(25)
    og = olsc.LSCOracle(ob, 8, 3, rad, R, Sec, "adjacent")
    ci, co, V = 4, 6, 777
    lay = layers.LocalSphericalConvolution(3, 3, dirs, 8, 8, [Sec] * R, 0.006, rad, bvals, ci, co, "adjacent",
                                           ring_tied=True).cuda()
    w_ring = synth.gaussian((co, 3, ci, 3, R + 1), 0.1, seed=18) * og.win[None, :, None, :, None]
    b = synth.gaussian((co, 3), 0.1, seed=19)
    with torch.no_grad():
        lay.weight.copy_(torch.from_numpy(w_ring))
        lay.bias.copy_(torch.from_numpy(b))
    c = synth.gaussian((V, ci, 3, 45), 1.0, seed=20, tag="coeffs")
    d = synth.gaussian((V, co, 3, 45), 1.0, seed=21, tag="grads")
    x = layers.empty_act(3 * ci * 45, V, DT[prec])
    x.copy_(torch.from_numpy(sh_to_rows(c)).to(DT[prec]))
    x.requires_grad_(True)
    y = lay(x)
    y.backward(torch.from_numpy(sh_to_rows(d)).to(y.dtype).cuda())
    torch.cuda.synchronize()
    w = olsc.ring_expand(w_ring, R, Sec)
    ref_y = og.forward(c, w, b)
    ref_din, ref_dw, ref_db = og.backward(c, w, d)
    got_y = rows_to_sh(y.detach().float().cpu().numpy(), 3, co, 45)
    got_din = rows_to_sh(x.grad.float().cpu().numpy(), 3, ci, 45)
    assert rel_l2(got_y, ref_y) <= TOL[prec]
    assert rel_l2(got_din, ref_din) <= TOL[prec]
    ref_dring = olsc.ring_reduce(ref_dw, R, Sec)
    assert lay.weight.grad.shape == (co, 3, ci, 3, R + 1)
    assert rel_l2(lay.weight.grad.cpu().numpy(), ref_dring) <= TOL[prec]
    assert rel_l2(lay.bias.grad.cpu().numpy(), ref_db) <= TOL[prec]


def test_ring_band_scaling_on_gpu():
    dirs, bvals = synth.multishell_table([90], [1000], seed=23)
    R, Sec, L4, rad = 2, 7, 4, np.deg2rad(30)
    ci, co, V = 3, 2, 1000
    lay = layers.LocalSphericalConvolution(1, 1, dirs, L4, L4, [Sec] * R, 0.0, rad, bvals, ci, co,
                                           ring_tied=True, bias=False).cuda()
    w_ring = synth.gaussian((co, 1, ci, 1, R + 1), 0.3, seed=24)
    with torch.no_grad():
        lay.weight.copy_(torch.from_numpy(w_ring))
    c = synth.gaussian((V, ci, 1, 15), 1.0, seed=25, tag="coeffs")
    x = layers.empty_act(ci * 15, V, torch.float32)
    x.copy_(torch.from_numpy(sh_to_rows(c)).float())
    with torch.no_grad():
        y = lay(x)
    mu = olsc.ring_band_multipliers(w_ring, L4, rad, R, Sec)  # [co, 1, ci, 1, 15]
    ref = np.einsum("oscpj,vcpj->vosj", mu, c)
    assert rel_l2(rows_to_sh(y.cpu().numpy(), 1, co, 15), ref) <= TOL_F32
    st, code = L.device_error(0)
    assert st == L.OK and code == 0
