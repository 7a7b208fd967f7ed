"""GPU parity of the resampling-free LSC (acquired neighbours binned to kernel points,
DELIMIT_LSC_NEIGHBOURS) against the FP64 oracle: forward, input gradient, weight and
bias gradients through the C ABI, in FP32 (tensor cores through split operands, CUDA
cores) and BF16 (tensor cores with and without two-CTA clusters, CUDA cores); the 65,536-voxel
configuration on sampled voxels; and the layer with ``resample=False``."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2, rows_to_sh, sh_to_rows  # noqa: E402
from tests.test_gpu_lsc import _gpu_lsc  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = {"f32": TOL_F32, "bf16": TOL_BF16}

CASES = {
    # three 40-direction shells, adjacent-shell mixing, 25 deg, 4 x 12 kernel, ragged voxel count
    "adjacent": dict(m=[40, 40, 40], order_in=8, order_out=8, V=777, ci=4, co=8, rad=25, R=4, Sec=12,
                     win="adjacent"),
    # one 60-direction shell, 30 deg, 3 x 8 kernel, 1 -> 8 channels
    "single": dict(m=[60], order_in=8, order_out=8, V=1000, ci=1, co=8, rad=30, R=3, Sec=8, win="same"),
    # every shell into every shell, orders 4 -> 8, unequal shells
    "all_mixed": dict(m=[30, 36, 42], order_in=4, order_out=8, V=300, ci=2, co=5, rad=25, R=2, Sec=6, win="all"),
}


def _setup(cfg, seed=11):
    dirs, bvals = synth.multishell_table(cfg["m"], [1000, 2000, 3000][:len(cfg["m"])], seed=seed)
    ob = osh.SHBasisOracle(dirs, bvals, cfg["order_out"], 0.006)
    lb = L.SHBasis(dirs, bvals, cfg["order_out"], 0.006)
    S, rad = len(cfg["m"]), np.deg2rad(cfg["rad"])
    og = olsc.LSCNeighbourOracle(ob, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"])
    lg = L.LSCGeometry(lb, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"], neighbours=True)
    return og, lg, dirs, bvals


@pytest.mark.parametrize("prec,tc,cluster", [("f32", False, 2), ("f32", True, 2), ("bf16", True, 2),
                                             ("bf16", True, 1), ("bf16", False, 2)])
@pytest.mark.parametrize("case", list(CASES))
def test_resampling_free_lsc_vs_oracle(case, prec, tc, cluster, gemm_cluster):
    gemm_cluster(cluster)
    cfg = CASES[case]
    og, lg, _, _ = _setup(cfg)
    V, ci, co = cfg["V"], cfg["ci"], cfg["co"]
    c = synth.gaussian((V, ci, og.s_in, og.n_in), 1.0, seed=1, tag="coeffs")
    w = synth.gaussian((co, og.s_out, ci, og.s_in, og.K), 0.1, seed=2)
    b = synth.gaussian((co, og.s_out), 0.1, seed=3)
    d = synth.gaussian((V, co, og.s_out, og.n_out), 1.0, seed=4, tag="grads")
    L.set_tensor_cores(tc)
    try:
        y, din, dw, db = _gpu_lsc(lg, c, w, b, d, ci, co, prec)
    finally:
        L.set_tensor_cores(True)
    ref_y = og.forward(c, w, b)
    ref_din, ref_dw, ref_db = og.backward(c, w, d)
    errs = {"c_out": rel_l2(y, ref_y), "dc_in": rel_l2(din, ref_din), "dw": rel_l2(dw, ref_dw),
            "db": rel_l2(db, ref_db)}
    assert all(v <= TOL[prec] for v in errs.values()), errs
    assert np.all(dw.transpose(1, 3, 0, 2, 4)[~og.win] == 0)


def test_resampling_free_full_size_sampled():
    """65,536 voxels, 3 x 90 directions, 16 -> 64 channels, 25 deg, 4 x 12 kernel,
    adjacent shells, BF16 on tensor cores: forward and input gradient on 64 sampled
    voxels against the oracle, weight gradient by linearity on a 512-voxel launch."""
    cfg = dict(m=[90, 90, 90], order_in=8, order_out=8, rad=25, R=4, Sec=12, win="adjacent")
    og, lg, _, _ = _setup(cfg, seed=1808)
    V = 65536
    c = synth.gaussian((V, 16, 3, 45), 1.0, seed=5, tag="coeffs").astype(np.float32)
    w = synth.gaussian((64, 3, 16, 3, 49), 0.1, seed=6)
    b = synth.gaussian((64, 3), 0.1, seed=7)
    d = synth.gaussian((V, 64, 3, 45), 1.0, seed=8, tag="grads").astype(np.float32)
    y, din, dw, db = _gpu_lsc(lg, c, w, b, d, 16, 64, "bf16")
    idx = synth.voxel_subset(V, 64)
    ref_y = og.forward(c[idx].astype(np.float64), w, b)
    ref_din, _, _ = og.backward(c[idx].astype(np.float64), w, d[idx].astype(np.float64))
    assert rel_l2(y[idx], ref_y) <= TOL_BF16
    assert rel_l2(din[idx], ref_din) <= TOL_BF16
    sub = synth.voxel_subset(V, 512)
    w2 = synth.gaussian(w.shape, 0.1, seed=9) * og.win[None, :, None, :, None]
    _, _, dw_sub, _ = _gpu_lsc(lg, c[sub], w, b, d[sub], 16, 64, "bf16")
    lhs = float(np.sum(dw_sub * w2))
    rhs = float(np.sum(d[sub].astype(np.float64) * og.forward(c[sub].astype(np.float64), w2, np.zeros_like(b))))
    assert abs(lhs - rhs) <= TOL_BF16 * np.linalg.norm(dw_sub) * np.linalg.norm(w2) * 4
    assert np.isfinite(dw).all() and np.isfinite(db).all()


def test_resampling_free_layer_autograd():
    cfg = CASES["adjacent"]
    og, _, dirs, bvals = _setup(cfg, seed=12)
    ci, co, V = 4, 6, 500
    lay = layers.LocalSphericalConvolution(3, 3, dirs, 8, 8, [12] * 4, 0.006, np.deg2rad(25), bvals, ci, co,
                                           "adjacent", resample=False).cuda()
    w = synth.gaussian((co, 3, ci, 3, 49), 0.1, seed=13) * og.win[None, :, None, :, None]
    b = synth.gaussian((co, 3), 0.1, seed=14)
    with torch.no_grad():
        lay.weight.copy_(torch.from_numpy(w))
        lay.bias.copy_(torch.from_numpy(b))
    c = synth.gaussian((V, ci, 3, 45), 1.0, seed=15, tag="coeffs")
    d = synth.gaussian((V, co, 3, 45), 1.0, seed=16, tag="grads")
    x = layers.empty_act(3 * ci * 45, V, torch.bfloat16)
    x.copy_(torch.from_numpy(sh_to_rows(c)).to(torch.bfloat16))
    x.requires_grad_(True)
    y = lay(x)
    y.backward(torch.from_numpy(sh_to_rows(d)).to(y.dtype).cuda())
    torch.cuda.synchronize()
    ref_y = og.forward(c, w, b)
    ref_din, ref_dw, ref_db = og.backward(c, w, d)
    assert rel_l2(rows_to_sh(y.detach().float().cpu().numpy(), 3, co, 45), ref_y) <= TOL_BF16
    assert rel_l2(rows_to_sh(x.grad.float().cpu().numpy(), 3, ci, 45), ref_din) <= TOL_BF16
    assert rel_l2(lay.weight.grad.cpu().numpy(), ref_dw) <= TOL_BF16
    assert rel_l2(lay.bias.grad.cpu().numpy(), ref_db) <= TOL_BF16
