"""The method's degenerate cases through the tensor-core kernels, against the FP64 oracle.

Order 0 (one coefficient per shell), order 2, an order-0 input beside an order-8
output, a one-point ring (K = 2), the largest radius (pi/2: every direction a
neighbour) and a shell of one direction.  The transforms (all four) and the LSC
(forward, input, weight and bias gradients) run with tensor cores required, in both
precisions, so none of these shapes may fall back to the CUDA cores.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2, rows_to_sh, rows_to_sig, sh_to_rows, sig_to_rows  # noqa: E402

pytestmark = pytest.mark.gpu
DT = {"f32": torch.float32, "bf16": torch.bfloat16}
TOL = {"f32": TOL_F32, "bf16": TOL_BF16}

CASES = {
    # order 0 in and out: one coefficient per shell, lambda 0
    "order0": dict(m=[30, 30], order_out=0, lam=0.0, order_in=0, R=2, Sec=6, rad=np.deg2rad(20), win="adjacent"),
    # order-0 input into order-8 output shells, one-point ring (K = 2), every shell mixed
    "order0_in_one_point_ring": dict(m=[30, 30], order_out=8, lam=0.006, order_in=0, R=1, Sec=1,
                                     rad=np.deg2rad(20), win="all"),
    # the largest radius: every direction of the shell is a neighbour
    "radius_pi2": dict(m=[30, 30], order_out=4, lam=0.0, order_in=4, R=1, Sec=1, rad=np.pi / 2, win="same"),
    # order 2, radius pi/2, 3 rings x 7 sectors
    "order2_pi2": dict(m=[30, 30], order_out=2, lam=0.006, order_in=2, R=3, Sec=7, rad=np.pi / 2, win="adjacent"),
    # a shell of a single direction beside two of 20 (regularised fit of order 2)
    "one_direction_shell": dict(m=[1, 20, 20], order_out=2, lam=0.006, order_in=2, R=2, Sec=6,
                                rad=np.deg2rad(25), win="adjacent"),
}


def _dev(a, dt):
    t = layers.empty_act(a.shape[0], a.shape[1], dt)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dt))
    return t


def _tables(cfg):
    bv = [1000, 2000, 3000][:len(cfg["m"])]
    dirs, bvals = synth.multishell_table(cfg["m"], bv, seed=21)
    return dirs, bvals


@pytest.mark.parametrize("prec", ["bf16", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_transforms_edge_cases(case, prec):
    cfg = CASES[case]
    dirs, bvals = _tables(cfg)
    ob = osh.SHBasisOracle(dirs, bvals, cfg["order_out"], cfg["lam"])
    lb = L.SHBasis(dirs, bvals, cfg["order_out"], cfg["lam"])
    V, C = 1000, 2
    sig = synth.fibre_signal(dirs, bvals, V * C, seed=3).astype(np.float64).reshape(C, V, -1).transpose(1, 0, 2)
    sh = ob.signal2sh(sig)
    dsh = synth.gaussian(sh.shape, 1.0, seed=4, tag="grads")
    dsig = synth.gaussian(sig.shape, 1.0, seed=5, tag="grads")
    S, N, m = ob.n_shells, ob.n_coef, ob.m
    out_dt = torch.float32
    L.set_tensor_cores(L.TC_REQUIRE)
    try:
        def run(kind, x_rows):
            y = layers.transform(kind, lb, _dev(x_rows, DT[prec]), C, out_dtype=out_dt)
            torch.cuda.synchronize()
            return y.double().cpu().numpy()
        got = {"signal2sh": rows_to_sh(run("signal2sh", sig_to_rows(sig, m)), S, C, N),
               "sh2signal": rows_to_sig(run("sh2signal", sh_to_rows(sh)), m, C),
               "signal2sh_backward": rows_to_sig(run("signal2sh_backward", sh_to_rows(dsh)), m, C),
               "sh2signal_backward": rows_to_sh(run("sh2signal_backward", sig_to_rows(dsig, m)), S, C, N)}
    finally:
        L.set_tensor_cores(True)
    ref = {"signal2sh": sh, "sh2signal": ob.sh2signal(sh), "signal2sh_backward": ob.signal2sh_backward(dsh),
           "sh2signal_backward": ob.sh2signal_backward(dsig)}
    errs = {k: rel_l2(got[k], ref[k]) for k in got}
    assert all(v <= TOL[prec] for v in errs.values()), errs


@pytest.mark.parametrize("prec", ["bf16", "f32"])
@pytest.mark.parametrize("case", list(CASES))
def test_lsc_edge_cases(case, prec):
    cfg = CASES[case]
    dirs, bvals = _tables(cfg)
    S = len(cfg["m"])
    ob = osh.SHBasisOracle(dirs, bvals, cfg["order_out"], cfg["lam"])
    lb = L.SHBasis(dirs, bvals, cfg["order_out"], cfg["lam"])
    og = olsc.LSCOracle(ob, cfg["order_in"], S, cfg["rad"], cfg["R"], cfg["Sec"], cfg["win"])
    lg = L.LSCGeometry(lb, cfg["order_in"], S, cfg["rad"], cfg["R"], cfg["Sec"], cfg["win"])
    assert lg.K == 1 + cfg["R"] * cfg["Sec"]
    V, ci, co = 777, 3, 5
    c = synth.gaussian((V, ci, S, og.n_in), 1.0, seed=1, tag="coeffs")
    w = synth.gaussian((co, S, ci, S, og.K), 0.1, seed=2)
    b = synth.gaussian((co, S), 0.1, seed=3)
    d = synth.gaussian((V, co, S, og.n_out), 1.0, seed=4, tag="grads")
    L.set_tensor_cores(L.TC_REQUIRE)
    try:
        x = _dev(sh_to_rows(c), DT[prec])
        wt, bt = torch.from_numpy(w).float().cuda(), torch.from_numpy(b).float().cuda()
        y = layers.lsc_forward(lg, x, wt, bt, ci, co)
        din, dw, db = layers.lsc_backward(lg, x, wt, _dev(sh_to_rows(d), DT[prec]), ci, co)
        torch.cuda.synchronize()
    finally:
        L.set_tensor_cores(True)
    ref_y = og.forward(c, w, b)
    ref_din, ref_dw, ref_db = og.backward(c, w, d)
    errs = {"c_out": rel_l2(rows_to_sh(y.double().cpu().numpy(), S, co, og.n_out), ref_y),
            "dc_in": rel_l2(rows_to_sh(din.double().cpu().numpy(), S, ci, og.n_in), ref_din),
            "dw": rel_l2(dw.cpu().numpy(), ref_dw), "db": rel_l2(db.cpu().numpy(), ref_db)}
    assert all(v <= TOL[prec] for v in errs.values()), errs
    st, code = L.device_error(torch.cuda.current_stream().cuda_stream)
    assert st == L.OK and code == 0
