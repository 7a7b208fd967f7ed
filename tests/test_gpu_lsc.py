"""GPU parity of the LSC forward and backward against the FP64 oracle (literal form).

All calls go through the C ABI.  FP32 path: relative L2 <= 1e-5 per output;
BF16 path (bf16 activations, fp32 accumulation, fp32 master weights): <= 1e-2.
Both precisions run on the tensor cores (FP32 as three-part BF16 splits with six
part products) and on the CUDA cores; the tensor-core GEMMs with and without
two-CTA clusters (odd voxel-tile and row-tile counts included).
"""
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

CASES = {
    # the 1,000-voxel configuration: one 60-direction shell, order 8, lambda 0.006,
    # 1 -> 8 channels, radius 30 deg, 3 rings x 8 sectors, weights N(0, 0.1)
    "c1": dict(m=[60], b=[1000], order_in=8, order_out=8, lam=0.006, V=1000, ci=1, co=8, rad=30, R=3, Sec=8,
               win="same"),
    # three shells, adjacent-shell mixing, radius 25 deg, 4 x 12 (K = 49), ragged voxel count
    "adjacent": dict(m=[40, 40, 40], b=[1000, 2000, 3000], order_in=8, order_out=8, lam=0.006, V=777, ci=4, co=8,
                     rad=25, R=4, Sec=12, win="adjacent"),
    # shells-as-channels (all input shells), mixed orders, 1 input shell -> 3 output shells
    "all_mixed": dict(m=[30, 30, 30], b=[1000, 2000, 3000], order_in=4, order_out=8, lam=0.006, V=300, ci=1, co=5,
                      rad=25, R=2, Sec=6, win="all", s_in=1),
    # many kernel points (6 rings x 12 sectors, K = 73: the operator build and the weight-
    # gradient reduction each take a second chunk of kernel points) and 5 x 7 = 35 channel
    # pairs (a ragged pair block), two shells, mixed orders 6 -> 8
    "many_points": dict(m=[40, 40], b=[1000, 2000], order_in=6, order_out=8, lam=0.006, V=600, ci=5, co=7,
                        rad=30, R=6, Sec=12, win="adjacent"),
    # the paper's moving-average example (order 4, [5], pi/5)
    "paper_ma": dict(m=[60], b=[1000], order_in=4, order_out=4, lam=0.006, V=257, ci=1, co=1, rad=36, R=1, Sec=5,
                     win="same"),
}


def _setup(cfg, seed=11):
    dirs, bvals = synth.multishell_table(cfg["m"], cfg["b"], seed=seed)
    ob = osh.SHBasisOracle(dirs, bvals, cfg["order_out"], cfg["lam"])
    lb = L.SHBasis(dirs, bvals, cfg["order_out"], cfg["lam"])
    s_in = cfg.get("s_in", len(cfg["m"]))
    rad = np.deg2rad(cfg["rad"])
    og = olsc.LSCOracle(ob, cfg["order_in"], s_in, rad, cfg["R"], cfg["Sec"], cfg["win"])
    lg = L.LSCGeometry(lb, cfg["order_in"], s_in, rad, cfg["R"], cfg["Sec"], cfg["win"])
    return og, lg


def _dev(a, dt):
    t = layers.empty_act(a.shape[0], a.shape[1], dt)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dt))
    return t


def _inputs(og, cfg, seed=1):
    V, ci, co = cfg["V"], cfg["ci"], cfg["co"]
    c = synth.gaussian((V, ci, og.s_in, og.n_in), 1.0, seed=seed, tag="coeffs")
    w = synth.gaussian((co, og.s_out, ci, og.s_in, og.K), 0.1, seed=seed + 1)
    b = synth.gaussian((co, og.s_out), 0.1, seed=seed + 2)
    d = synth.gaussian((V, co, og.s_out, og.n_out), 1.0, seed=seed + 3, tag="grads")
    return c, w, b, d


def _gpu_lsc(lg, c, w, b, d, ci, co, prec):
    x = _dev(sh_to_rows(c), DT[prec])
    wt = torch.from_numpy(w).float().cuda()
    bt = torch.from_numpy(b).float().cuda()
    y = layers.lsc_forward(lg, x, wt, bt, ci, co)
    din, dw, db = layers.lsc_backward(lg, x, wt, _dev(sh_to_rows(d), DT[prec]), ci, co)
    torch.cuda.synchronize()
    return (rows_to_sh(y.float().cpu().numpy(), lg.s_out, co, lg.n_out),
            rows_to_sh(din.float().cpu().numpy(), lg.s_in, ci, lg.n_in), dw.cpu().numpy(), db.cpu().numpy())


@pytest.mark.parametrize("prec,tc,cluster", [("f32", False, 2), ("f32", True, 2), ("f32", True, 1),
                                             ("bf16", True, 2), ("bf16", True, 1), ("bf16", False, 2)])
@pytest.mark.parametrize("case", list(CASES))
def test_lsc_vs_oracle(case, prec, tc, cluster, gemm_cluster):
    # cluster: CTAs per cluster of the tensor-core GEMMs (2 = CTA pairs with 2-SM MMAs);
    # f32 with tc: FP32 activations through three-part BF16 splits on the tensor cores
    gemm_cluster(cluster)
    cfg = CASES[case]
    og, lg = _setup(cfg)
    c, w, b, d = _inputs(og, cfg)
    if case == "paper_ma":
        w = np.full_like(w, 1.0 / 6.0)
        b = np.zeros_like(b)
    L.set_tensor_cores(tc)
    try:
        y, din, dw, db = _gpu_lsc(lg, c, w, b, d, cfg["ci"], cfg["co"], prec)
    finally:
        L.set_tensor_cores(True)
    ref_y = og.forward(c, w, b)
    ref_din, ref_dw, ref_db = og.backward(c, w, d)
    errs = {"c_out": rel_l2(y, ref_y), "dc_in": rel_l2(din, ref_din), "dw": rel_l2(dw, ref_dw),
            "db": rel_l2(db, ref_db)}
    assert all(v <= TOL[prec] for v in errs.values()), errs
    # weights outside the shell window get exactly zero gradient
    assert np.all(dw.transpose(1, 3, 0, 2, 4)[~og.win] == 0)


FULL = {
    # the bench's launch configuration
    "adjacent": dict(order_in=8, win="adjacent"),
    # SH order 4 in, 8 out, every input shell into every output shell (shells as channels)
    "mixed_all": dict(order_in=4, win="all"),
}


def _bf16(x):
    """Round to the nearest BF16 value (ties to even), as float64: the values a BF16 upload holds."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _dw_collapse(og, c, d, rnd=None, chunk=8192):
    """Every weight-gradient entry over all voxels by the oracle's collapse route:
    G[(co,s,a),(ci,s',b)] = sum_v d[v,co,s,a] c[v,ci,s',b] in FP64 (voxel chunks), then
    dw[co,s,ci,s',k] = sum_ab M_{s,s'}[k,a,b] G (zero outside the window).  rnd: the rounding
    applied to the operands first (the values a BF16 upload holds), or None."""
    V, co, S, n_out = d.shape
    ci, n_in = c.shape[1], c.shape[3]
    G = np.zeros((co * S * n_out, ci * c.shape[2] * n_in))
    for v0 in range(0, V, chunk):
        dd = d[v0:v0 + chunk].reshape(-1, G.shape[0]).astype(np.float64)
        cc = c[v0:v0 + chunk].reshape(-1, G.shape[1]).astype(np.float64)
        if rnd is not None:
            dd, cc = rnd(dd), rnd(cc)
        G += dd.T @ cc
    G = G.reshape(co, S, n_out, ci, c.shape[2], n_in)
    dw = np.zeros((co, S, ci, c.shape[2], og.K))
    for s in range(S):
        for sp in range(c.shape[2]):
            if og.win[s, sp]:
                dw[:, s, :, sp, :] = np.einsum("kab,oaib->oik", og.pair_mats(s, sp), G[:, s, :, :, sp, :],
                                               optimize=True)
    return dw


def _worst_slice(got, ref, win):
    """Largest relative L2 error over the (co, s, ci, s') kernel vectors inside the window."""
    e = np.linalg.norm(got - ref, axis=-1)
    r = np.linalg.norm(ref, axis=-1)
    m = win[None, :, None, :] & (r > 0)
    return float((e[m] / r[m]).max())


@pytest.mark.parametrize("variant,prec", [("adjacent", "bf16"), ("mixed_all", "bf16"), ("adjacent", "f32"),
                                          ("mixed_all", "f32")])
def test_lsc_full_size_sampled(variant, prec):
    """65,536 voxels, 3 x 90 directions, 16 -> 64 channels, radius 25 deg, 4 x 12 kernel, on
    the tensor cores (BF16, or FP32 through split operands), in the launch configuration
    the benchmark times.  Forward and input gradient on 64 sampled voxels against the oracle;
    every weight-gradient entry against the oracle's collapse route over all voxels (and,
    for BF16, against the exact gradient of the BF16 values the GEMMs read, which only FP32
    accumulation separates from the kernels' result); the bias gradient in full."""
    tol = TOL[prec]
    cfg = dict(m=[90, 90, 90], b=[1000, 2000, 3000], order_out=8, lam=0.006, V=65536, ci=16, co=64,
               rad=25, R=4, Sec=12, **FULL[variant])
    og, lg = _setup(cfg, seed=1808)
    V, n_in, n_out = cfg["V"], og.n_in, og.n_out
    c = synth.gaussian((V, 16, 3, n_in), 1.0, seed=5, tag="coeffs").astype(np.float32)
    w = synth.gaussian((64, 3, 16, 3, 49), 0.1, seed=6)
    b = synth.gaussian((64, 3), 0.1, seed=7)
    d = synth.gaussian((V, 64, 3, n_out), 1.0, seed=8, tag="grads").astype(np.float32)
    L.set_tensor_cores(L.TC_REQUIRE)  # the LSC GEMMs must not fall back to the CUDA cores
    try:
        y, din, dw, db = _gpu_lsc(lg, c, w, b, d, 16, 64, prec)
    finally:
        L.set_tensor_cores(True)
    idx = synth.voxel_subset(V, 64)
    ref_y = og.forward(c[idx].astype(np.float64), w, b)
    ref_din, _, _ = og.backward(c[idx].astype(np.float64), w, d[idx].astype(np.float64))
    assert rel_l2(y[idx], ref_y) <= tol
    assert rel_l2(din[idx], ref_din) <= tol
    # every dw entry (351,232 inside the window at adjacent shells) over all 65,536 voxels
    ref_dw = _dw_collapse(og, c, d)
    assert rel_l2(dw, ref_dw) <= tol
    # kernel vectors one by one: the input rounding alone spreads them about the global
    # figure, so this bound only has to catch a wrong tile or split, not the rounding
    assert _worst_slice(dw, ref_dw, og.win) <= 3 * tol
    assert np.all(dw.transpose(1, 3, 0, 2, 4)[~og.win] == 0)
    if prec == "bf16":
        # the BF16 GEMMs read bf16(c) and bf16(d) exactly; what separates their dw from the
        # FP64 gradient of those values is FP32 accumulation and the FP32 collapse matrices
        ex_dw = _dw_collapse(og, c, d, rnd=_bf16)
        e_ex, e_ws = rel_l2(dw, ex_dw), _worst_slice(dw, ex_dw, og.win)
        print(f"dw vs exact gradient of the BF16 operands: {e_ex:.3e} (worst slice {e_ws:.3e})")
        assert e_ex <= 2e-4 and e_ws <= 1e-3
    # db = sum over voxels of P_out-weighted upstream gradient, a plain reduction
    q = og.collapse_mats()[1]
    ref_db = np.stack([np.einsum("vcx,x->c", d[:, :, s, :].astype(np.float64), q[s]) for s in range(3)], 1)
    assert rel_l2(db, ref_db) <= tol
    assert np.isfinite(dw).all() and np.linalg.norm(dw) > 0


def test_lsc_zero_voxels_and_workspace_errors():
    og, lg = _setup(CASES["c1"])
    lib = L.get()
    w = torch.zeros((8, 1, 1, 1, 25), device="cuda")
    dw = torch.full_like(w, 7.0)
    db = torch.full((8, 1), 7.0, device="cuda")
    ws_n = lg.workspace_size(0, 1, 8, L.BF16, True)
    ws = torch.empty(ws_n + 256, dtype=torch.uint8, device="cuda")
    wsp = (ws.data_ptr() + 255) // 256 * 256
    st = lib.delimit_lsc_backward(lg.handle, None, w.data_ptr(), None, None, dw.data_ptr(), db.data_ptr(), 0, 1, 8,
                                  8, 8, L.BF16, 0, wsp, ws_n, None)
    torch.cuda.synchronize()
    assert st == L.OK and float(dw.abs().sum()) == 0 and float(db.abs().sum()) == 0
    x = layers.empty_act(45, 100, torch.bfloat16)
    y = layers.empty_act(8 * 45, 100, torch.bfloat16)
    need = lg.workspace_size(100, 1, 8, L.BF16, False)
    st = lib.delimit_lsc_forward(lg.handle, x.data_ptr(), w.data_ptr(), None, y.data_ptr(), 100, 1, 8, x.stride(0),
                                 y.stride(0), L.BF16, 0, wsp, need - 1, None)
    assert st == L.ERR_WORKSPACE
    st = lib.delimit_lsc_forward(lg.handle, x.data_ptr(), w.data_ptr(), None, y.data_ptr(), 100, 1, 8, x.stride(0),
                                 y.stride(0), L.BF16, 0, wsp + 16, need, None)
    assert st == L.ERR_ALIGNMENT


@pytest.mark.parametrize("prec,tc,case", [("bf16", True, "adjacent"), ("bf16", False, "adjacent"),
                                          ("f32", True, "adjacent"), ("f32", True, "all_mixed")])
def test_backward_reuses_forward_operator(prec, tc, case):
    """A backward flagged OPERATOR_READY on the forward's workspace gives the same
    bits as a backward that rebuilds the collapsed operator itself (for FP32 on the
    tensor cores including its split parts; all_mixed reads Wt in the forward)."""
    cfg = CASES[case]
    og, lg = _setup(cfg)
    c, w, b, d = _inputs(og, cfg, seed=5)
    ci, co = cfg["ci"], cfg["co"]
    x = _dev(sh_to_rows(c), DT[prec])
    g = _dev(sh_to_rows(d), DT[prec])
    wt, bt = torch.from_numpy(w).float().cuda(), torch.from_numpy(b).float().cuda()
    L.set_tensor_cores(tc)
    try:
        ws = layers.lsc_workspace(lg, x.shape[1], ci, co, DT[prec], True)
        layers.lsc_forward(lg, x, wt, bt, ci, co, workspace=ws)
        got = layers.lsc_backward(lg, x, wt, g, ci, co, workspace=ws, operator_ready=True)
        ref = layers.lsc_backward(lg, x, wt, g, ci, co)
        torch.cuda.synchronize()
    finally:
        L.set_tensor_cores(True)
    for a, r in zip(got, ref):
        assert torch.equal(a, r)
