"""The collapsed LSC operator W as built for a BF16 forward, against the FP64 oracle.

W[(s,co,a)][(s',ci,b)] = sum_k w[co,s,ci,s',k] M_{s,s'}[k][a][b] (Sec. 2.3, the exact
collapse), read back from the workspace after delimit_lsc_forward.  Shapes with K <= 64,
c_in dividing 128 and c_in N_in a multiple of 8 (no padding between shell blocks, so the
forward reads W) take the tensor-core build (trace name lsc_build_w_tc: FP32-level
part products, then BF16), the others the CUDA-core build (lsc_build_w).  Blocks outside
the window and the padding columns between shell blocks are zero.

Both builds multiply the library's FP32 copy of M (each entry rounded by 2^-24 of
itself) and sum K products in FP32 (a recursive sum: within K 2^-24 of the sum of
magnitudes), so W before its BF16 rounding is within e = (K + 1) 2^-24 sum_k |w_k| |M_k|
of the FP64 operator.  Against the FP64 operator rounded to BF16, each entry is within
one BF16 ulp plus e (about 2 % of the entries at the benchmark's shape round the other
way); against each other, the tensor-core and CUDA-core builds share M and differ by
their summation order only: equal in at least 99.9 % of the entries, and each entry
within one ulp plus 2e.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lsc as olsc  # noqa: E402
from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    # the benchmark's shape: three shells, adjacent windows, K = 49, 16 -> 8 channels
    "bench_adjacent": dict(m=[40, 40, 40], order_in=8, ci=16, co=8, R=4, Sec=12, win="adjacent", tc=True),
    # two input channels, mixed orders 6 -> 8 (N_in = 28), every shell mixed
    "ci2_all_mixed": dict(m=[30, 30, 30], order_in=6, ci=2, co=5, R=2, Sec=6, win="all", tc=True),
    # one shell, 32 input channels (four channels per 128-pair tile), K = 22
    "ci32_one_shell": dict(m=[40], order_in=8, ci=32, co=4, R=3, Sec=7, win="same", tc=True),
    # 128 input channels (one channel per tile), K = 64 exactly, order 2 input (N_in = 6)
    "ci128_k64": dict(m=[30, 30], order_in=2, ci=128, co=2, R=7, Sec=9, win="adjacent", tc=True),
    # the resampling-free form: one collapse matrix per shell pair
    "resampling_free": dict(m=[40, 40, 40], order_in=8, ci=8, co=4, R=4, Sec=12, win="adjacent", tc=True,
                            neighbours=True),
    # c_in N_in = 4 x 15 = 60: padded shell blocks, so the forward reads Wt, which the
    # CUDA-core build writes
    "ci4_padded_blocks": dict(m=[30, 30], order_in=4, ci=4, co=5, R=2, Sec=6, win="adjacent", tc=False),
    # c_in = 3 does not divide 128: the CUDA-core build (with padded shell blocks)
    "ci3_cuda_cores": dict(m=[30, 30], order_in=4, ci=3, co=5, R=2, Sec=6, win="adjacent", tc=False),
    # K = 73 > 64: the CUDA-core build
    "k73_cuda_cores": dict(m=[40, 40], order_in=6, ci=8, co=4, R=6, Sec=12, win="adjacent", tc=False),
}


@pytest.mark.parametrize("case", list(CASES))
def test_operator_build_matches_oracle(case):
    cfg = CASES[case]
    dirs, bvals = synth.multishell_table(cfg["m"], [1000, 2000, 3000][:len(cfg["m"])], seed=31)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    lb = L.SHBasis(dirs, bvals, 8, 0.006)
    S = len(cfg["m"])
    rad = np.deg2rad(25)
    nb = cfg.get("neighbours", False)
    cls = olsc.LSCNeighbourOracle if nb else olsc.LSCOracle
    og = cls(ob, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"])
    lg = L.LSCGeometry(lb, cfg["order_in"], S, rad, cfg["R"], cfg["Sec"], cfg["win"], neighbours=nb)
    ci, co, K, n_in, n_out = cfg["ci"], cfg["co"], og.K, og.n_in, og.n_out
    w = synth.gaussian((co, S, ci, S, K), 0.1, seed=8).astype(np.float32)
    V = 64
    x = layers.empty_act(S * ci * n_in, V, torch.bfloat16)
    x.copy_(torch.from_numpy(synth.gaussian((S * ci * n_in, V), 1.0, seed=9, tag="coeffs")).to(torch.bfloat16))
    ws = layers.lsc_workspace(lg, V, ci, co, torch.bfloat16, False)
    in_blk = (ci * n_in + 7) // 8 * 8
    rows, ldw = S * co * n_out, S * in_blk
    wt = torch.from_numpy(w).cuda()

    def build(mode):
        """W as a BF16 forward under tensor-core policy `mode` builds it, and the trace."""
        t, ptr, _ = ws
        t.fill_(0xFF)  # every entry of W is written (padding included) or the check below fails
        L.set_tensor_cores(mode)
        L.trace_enable(True)
        try:
            layers.lsc_forward(lg, x, wt, None, ci, co, workspace=ws)
            torch.cuda.synchronize()
            trace = L.trace_summary()
        finally:
            L.trace_enable(False)
            L.set_tensor_cores(True)
        off = ptr - t.data_ptr()
        return t[off:off + rows * ldw * 2].view(torch.bfloat16).float().reshape(rows, ldw).cpu().numpy(), trace

    W, trace = build(L.TC_PREFER)
    assert ("lsc_build_w_tc" in trace) == cfg["tc"] and ("lsc_build_w" in trace) == (not cfg["tc"]), trace
    assert np.isfinite(W).all()
    # the FP64 operator block by block, and the bound of the FP32 copy of M
    ref = np.zeros((rows, ldw))
    err = np.zeros((rows, ldw))
    for s in range(S):
        for p in range(S):
            if not og.win[s, p]:
                continue
            Mp = og.pair_mats(s, p)
            wsp = w[:, s, :, p, :].astype(np.float64)
            rs, cs = slice(s * co * n_out, (s + 1) * co * n_out), slice(p * in_blk, p * in_blk + ci * n_in)
            ref[rs, cs] = np.einsum("ack,kxy->axcy", wsp, Mp).reshape(co * n_out, ci * n_in)
            err[rs, cs] = (K + 1) * 2.0 ** -24 * np.einsum("ack,kxy->axcy", np.abs(wsp), np.abs(Mp)).reshape(
                co * n_out, ci * n_in)
    ref16 = torch.from_numpy(ref).to(torch.bfloat16).float().numpy()
    mag = np.maximum(np.abs(ref16), np.abs(W))
    ulp = np.exp2(np.floor(np.log2(np.maximum(mag, 1e-30)))) * 2.0 ** -7
    over = np.abs(W - ref16) - (ulp + err)
    assert (over <= 1e-12).all(), float(over.max())
    assert (W[ref == 0] == 0).all()  # outside the window and the padding
    if cfg["tc"]:
        Wc, trace_c = build(L.TC_OFF)
        assert "lsc_build_w" in trace_c and "lsc_build_w_tc" not in trace_c, trace_c
        same = float((W == Wc).mean())
        assert same >= 0.999, same
        magc = np.maximum(mag, np.abs(Wc))
        ulpc = np.exp2(np.floor(np.log2(np.maximum(magc, 1e-30)))) * 2.0 ** -7
        over_c = np.abs(W - Wc) - (ulpc + 2 * err)
        assert (over_c <= 1e-12).all(), float(over_c.max())
    st, code = L.device_error(torch.cuda.current_stream().cuda_stream)
    assert st == L.OK and code == 0
