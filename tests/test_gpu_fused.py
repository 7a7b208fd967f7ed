"""The LSC forward with SH2Signal fused into one kernel (delimit_lsc_forward_sh2signal).

Against the unfused pair (delimit_lsc_forward, then delimit_sh2signal on the same
output basis), which rounds c_out to BF16 at the same point and multiplies by the same
BF16 operator, and against the FP64 oracle (LSC forward then SH2Signal, BF16 bar 1e-2).
Shapes: the benchmark's (65,536 voxels, 3 x 90 directions, 16 -> 64 channels, adjacent
shells, 4 x 12 kernel), ragged voxel counts, one shell (60 directions, 8 -> 8 channels),
mixed SH orders with every shell mixed, the resampling-free form, no bias.  Requests the
kernel does not take are refused with DELIMIT_ERR_UNSUPPORTED and a reason.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, rel_l2, rows_to_sig, sh_to_rows  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "bench": dict(m=[90, 90, 90], order_in=8, V=65536, ci=16, co=64, R=4, Sec=12, rad=25, win="adjacent"),
    "ragged": dict(m=[40, 40, 40], order_in=8, V=777, ci=8, co=8, R=4, Sec=12, rad=25, win="adjacent"),
    "ragged_large": dict(m=[90, 90, 90], order_in=8, V=65376, ci=16, co=64, R=4, Sec=12, rad=25, win="adjacent"),
    "one_shell": dict(m=[60], order_in=8, V=1000, ci=8, co=8, R=3, Sec=8, rad=30, win="same"),
    "mixed_all": dict(m=[30, 30, 30], order_in=4, V=3001, ci=8, co=4, R=2, Sec=6, rad=25, win="all"),
    "resampling_free": dict(m=[40, 40, 40], order_in=8, V=1999, ci=8, co=8, R=4, Sec=12, rad=25, win="adjacent",
                            neighbours=True),
    "no_bias": dict(m=[40, 40, 40], order_in=8, V=515, ci=8, co=12, R=2, Sec=6, rad=25, win="adjacent", bias=False),
}


def _setup(cfg, seed=1808):
    dirs, bvals = synth.multishell_table(cfg["m"], [1000, 2000, 3000][:len(cfg["m"])], seed=seed)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    lb = L.SHBasis(dirs, bvals, 8, 0.006)
    S = len(cfg["m"])
    rad = np.deg2rad(cfg["rad"])
    nb = cfg.get("neighbours", False)
    cls = olsc.LSCNeighbourOracle if nb else olsc.LSCOracle
    og = cls(ob, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"])
    lg = L.LSCGeometry(lb, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"], neighbours=nb)
    return ob, og, lb, lg


@pytest.mark.parametrize("case", list(CASES))
def test_fused_matches_unfused_and_oracle(case):
    cfg = CASES[case]
    ob, og, lb, lg = _setup(cfg)
    V, ci, co, S = cfg["V"], cfg["ci"], cfg["co"], len(cfg["m"])
    c = synth.gaussian((V, ci, S, og.n_in), 1.0, seed=5, tag="coeffs").astype(np.float32)
    w = synth.gaussian((co, S, ci, S, og.K), 0.1, seed=6)
    b = synth.gaussian((co, S), 0.1, seed=7) if cfg.get("bias", True) else None
    x = layers.empty_act(S * ci * og.n_in, V, torch.bfloat16)
    x.copy_(torch.from_numpy(np.ascontiguousarray(sh_to_rows(c))).to(torch.bfloat16))
    wt = torch.from_numpy(w).float().cuda()
    bt = torch.from_numpy(b).float().cuda() if b is not None else None
    assert layers.lsc_forward_sh2signal_supported(lg, V, ci, co, torch.bfloat16)
    L.set_tensor_cores(L.TC_REQUIRE)
    try:
        fused = layers.lsc_forward_sh2signal(lg, x, wt, bt, ci, co)
        c_out = layers.lsc_forward(lg, x, wt, bt, ci, co)
        unfused = layers.transform("sh2signal", lb, c_out, co)
        torch.cuda.synchronize()
    finally:
        L.set_tensor_cores(True)
    f, u = fused.float(), unfused.float()
    # same rounding points, same BF16 operands: equal up to rare one-ulp flips of the FP32 sums
    same = float((f == u).float().mean())
    assert same >= 0.999, same
    assert rel_l2(f.cpu().numpy(), u.cpu().numpy()) <= 1e-3
    # the FP64 oracle on sampled voxels (all of them when few)
    idx = synth.voxel_subset(V, min(V, 96), seed=3)
    xin = x[:, torch.from_numpy(idx).cuda()].double().cpu().numpy()
    c_in = np.transpose(xin.reshape(S, ci, og.n_in, -1), (3, 1, 0, 2))
    ref = ob.sh2signal(og.forward(c_in, w, b if b is not None else np.zeros((co, S))))
    got = rows_to_sig(f[:, torch.from_numpy(idx).cuda()].double().cpu().numpy(), cfg["m"], co)
    assert rel_l2(got, ref) <= TOL_BF16
    st, code = L.device_error(torch.cuda.current_stream().cuda_stream)
    assert st == L.OK and code == 0


def test_fused_refuses_what_it_does_not_take():
    lib = L.get()
    cfg = CASES["ragged"]
    _, _, _, lg = _setup(cfg)
    assert lib.delimit_lsc_forward_sh2signal_supported(lg.handle, 100, 4, 8, L.F32) == L.ERR_UNSUPPORTED
    assert b"BF16" in lib.delimit_last_error()
    assert lib.delimit_lsc_forward_sh2signal_supported(lg.handle, 100, 8, 6, L.BF16) == L.ERR_UNSUPPORTED
    assert b"multiple of 4" in lib.delimit_last_error()
    # 4 x 45 input rows per shell: the operator's input blocks carry padding
    assert lib.delimit_lsc_forward_sh2signal_supported(lg.handle, 100, 4, 8, L.BF16) == L.ERR_UNSUPPORTED
    assert b"padding" in lib.delimit_last_error()
    # order 10 output: 66 coefficients, more than a 48-row channel slot
    dirs, bvals = synth.multishell_table([90], [1000], seed=2)
    lb10 = L.SHBasis(dirs, bvals, 10, 0.006)
    lg10 = L.LSCGeometry(lb10, 8, 1, np.deg2rad(25), 2, 6, "same")
    assert lib.delimit_lsc_forward_sh2signal_supported(lg10.handle, 100, 8, 8, L.BF16) == L.ERR_UNSUPPORTED
    assert len(lib.delimit_last_error()) > 0
    # tensor cores switched off: no fused kernel on the CUDA cores
    L.set_tensor_cores(L.TC_OFF)
    try:
        assert lib.delimit_lsc_forward_sh2signal_supported(lg.handle, 100, 8, 8, L.BF16) == L.ERR_UNSUPPORTED
    finally:
        L.set_tensor_cores(True)
    assert lib.delimit_lsc_forward_sh2signal_supported(lg.handle, 100, 8, 8, L.BF16) == L.OK
