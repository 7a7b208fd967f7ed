"""GPU parity of Signal2SH / SH2Signal and their adjoints against the FP64 oracle.

Every call goes through the C ABI (via the ctypes binding).  FP32 path:
relative L2 <= 1e-5; BF16 path (bf16 in, fp32 accumulate): <= 1e-2.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2, rows_to_sh, rows_to_sig, sh_to_rows, sig_to_rows  # noqa: E402

pytestmark = pytest.mark.gpu
DT = {"f32": torch.float32, "bf16": torch.bfloat16}
TOL = {"f32": TOL_F32, "bf16": TOL_BF16}


def _dev(a, dt):
    t = layers.empty_act(a.shape[0], a.shape[1], dt)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dt))
    return t


def _run(kind, lb, x_rows, C, in_dt, out_dt):
    x = _dev(x_rows, in_dt)
    y = layers.transform(kind, lb, x, C, out_dtype=out_dt)
    torch.cuda.synchronize()
    return y.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("case", ["c1", "multishell_ragged", "channels", "wide_shell"])
def test_transforms_vs_oracle(prec, tc, case):
    L.set_tensor_cores(tc)
    try:
        if case == "c1":  # 1,000 voxels, 60 directions, order 8, lambda 0.006
            dirs, bvals = synth.multishell_table([60], [1000], seed=1808)
            order, lam, V, C = 8, 0.006, 1000, 1
        elif case == "multishell_ragged":  # 3 x 90 directions, ragged voxel count
            dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=1808)
            order, lam, V, C = 8, 0.006, 3001, 1
        elif case == "channels":  # channels and unequal shells
            dirs, bvals = synth.multishell_table([30, 45], [1000, 2000], seed=7)
            order, lam, V, C = 4, 0.06, 515, 16
        else:  # 150 directions, order 10: beyond the staged CUDA-core kernel's 128 inputs / 120 outputs
            dirs, bvals = synth.multishell_table([150], [2000], seed=9)
            order, lam, V, C = 10, 0.006, 300, 2
        ob = osh.SHBasisOracle(dirs, bvals, order, lam)
        lb = L.SHBasis(dirs, bvals, order, lam)
        m = ob.m
        sig = synth.fibre_signal(dirs, bvals, V * C, seed=3).astype(np.float64).reshape(C, V, -1).transpose(1, 0, 2)
        sh = ob.signal2sh(sig)  # [V, C, S, N]
        in_dt = DT[prec]
        out_dt = torch.float32 if prec == "bf16" else DT[prec]
        # forward
        got = rows_to_sh(_run("signal2sh", lb, sig_to_rows(sig, m), C, in_dt, out_dt), ob.n_shells, C, ob.n_coef)
        assert rel_l2(got, sh) <= TOL[prec]
        got = rows_to_sig(_run("sh2signal", lb, sh_to_rows(sh), C, in_dt, out_dt), m, C)
        assert rel_l2(got, ob.sh2signal(sh)) <= TOL[prec]
        # adjoints
        dsh = synth.gaussian(sh.shape, 1.0, seed=4, tag="grads")
        got = rows_to_sig(_run("signal2sh_backward", lb, sh_to_rows(dsh), C, in_dt, out_dt), m, C)
        assert rel_l2(got, ob.signal2sh_backward(dsh)) <= TOL[prec]
        dsig = synth.gaussian(sig.shape, 1.0, seed=5, tag="grads")
        got = rows_to_sh(_run("sh2signal_backward", lb, sig_to_rows(dsig, m), C, in_dt, out_dt), ob.n_shells, C,
                         ob.n_coef)
        assert rel_l2(got, ob.sh2signal_backward(dsig)) <= TOL[prec]
    finally:
        L.set_tensor_cores(True)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_transforms_full_size_sampled(prec):
    """The 1,048,576-voxel, 3 x 90-direction, order-8 workload in the bench's launch
    configuration; 4,096 sampled voxels are checked against the oracle."""
    dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=1808)
    V = 1 << 20
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    lb = L.SHBasis(dirs, bvals, 8, 0.006)
    sig = synth.fibre_signal(dirs, bvals, V, seed=1808)  # [V, 270] float32
    x = layers.empty_act(270, V, DT[prec])
    x.copy_(torch.from_numpy(np.ascontiguousarray(sig.T)).to(DT[prec]))
    c = layers.transform("signal2sh", lb, x, 1, out_dtype=torch.float32)
    s_back = layers.transform("sh2signal", lb, c, 1, out_dtype=torch.float32)
    torch.cuda.synchronize()
    idx = synth.voxel_subset(V, 4096)
    ref_c = ob.signal2sh(sig[idx].astype(np.float64)[:, None, :])  # [k, 1, S, N]
    got_c = rows_to_sh(c[:, idx].cpu().numpy(), 3, 1, 45)
    assert rel_l2(got_c, ref_c) <= TOL[prec]
    got_s = s_back[:, idx].cpu().numpy().T
    ref_s = ob.sh2signal(got_c)[:, 0, :]  # oracle SH2Signal of the GPU's own coefficients
    assert rel_l2(got_s, ref_s) <= TOL[prec]


def test_transform_edge_cases():
    dirs, bvals = synth.multishell_table([30], [1000], seed=2)
    lb = L.SHBasis(dirs, bvals, 4, 0.006)
    lib = L.get()
    x = layers.empty_act(30, 64, torch.float32)
    y = layers.empty_act(15, 64, torch.float32)
    # zero voxels is a no-op
    assert lib.delimit_signal2sh(lb.handle, x.data_ptr(), y.data_ptr(), 0, 1, 64, 64, L.F32, L.F32, None) == L.OK
    # misaligned pointer and unaligned row stride
    assert lib.delimit_signal2sh(lb.handle, x.data_ptr() + 4, y.data_ptr(), 8, 1, 64, 64, L.F32, L.F32,
                                 None) == L.ERR_ALIGNMENT
    assert lib.delimit_signal2sh(lb.handle, x.data_ptr(), y.data_ptr(), 8, 1, 63, 64, L.F32, L.F32,
                                 None) == L.ERR_ALIGNMENT
    # ld < n_vox
    assert lib.delimit_signal2sh(lb.handle, x.data_ptr(), y.data_ptr(), 80, 1, 64, 64, L.F32, L.F32,
                                 None) == L.ERR_INVALID_ARG
    # single voxel, and voxel count 7 with ld 64, both paths
    ob = osh.SHBasisOracle(dirs, bvals, 4, 0.006)
    for V in (1, 7, 129):
        sig = synth.fibre_signal(dirs, bvals, V, seed=V).astype(np.float64)
        for prec in ("f32", "bf16"):
            got = _run("signal2sh", lb, sig.T.copy(), 1, DT[prec], torch.float32)
            assert rel_l2(got.T, sig @ ob.P[0].T) <= TOL[prec]
    st, code = L.device_error(0)
    assert st == L.OK and code == 0
