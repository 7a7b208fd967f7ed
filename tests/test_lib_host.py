"""The C-ABI library without a GPU: exports, host FP64 tables vs the oracle, argument errors.

The library builds its tables with its own code (normalised Legendre
recurrence, Chebyshev azimuth recurrence, its own Cholesky); here they are
compared with the oracle's independent numpy computation.  Integer tables are
compared bit-exactly.
"""
import ctypes as C
import glob
import os
import re
import threading

import numpy as np
import pytest

from oracle import lsc as olsc
from oracle import sh as osh
from paper_1808_01517_gb300 import _lib as L
from paper_1808_01517_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(delimit_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = L.get()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares argtypes for every one of them
    assert names <= set(L.SIGNATURES), names - set(L.SIGNATURES)
    assert lib.delimit_version() >= 100
    assert lib.delimit_status_string(L.ERR_RANK_DEFICIENT) == b"rank deficient"


@pytest.fixture(scope="module")
def table3():
    dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=1808)
    return dirs, bvals


def test_basis_tables_match_oracle(table3):
    dirs, bvals = table3
    for order, lam in ((8, 0.006), (4, 0.06), (8, 0.0), (12, 0.006)):
        lb = L.SHBasis(dirs, bvals, order, lam, host_only=True)
        ob = osh.SHBasisOracle(dirs, bvals, order, lam)
        assert lb.n_shells == 3 and lb.m == [90, 90, 90] and lb.dir_off == [0, 90, 180]
        for s in range(3):
            B, P, idx = lb.tables(s)
            np.testing.assert_array_equal(idx, ob.rows[s])
            np.testing.assert_allclose(B, ob.B[s], rtol=0, atol=1e-12)
            scale = np.abs(ob.P[s]).max()
            np.testing.assert_allclose(P, ob.P[s], rtol=0, atol=1e-12 * max(1.0, scale))


def test_shell_grouping_order_and_dir_index():
    dirs, bvals = synth.multishell_table([20, 30], [3000, 1000], seed=3)
    lb = L.SHBasis(dirs, bvals, 4, 0.006, host_only=True)
    assert lb.bval == [1000.0, 3000.0] and lb.m == [30, 20] and lb.dir_off == [0, 30]
    _, _, idx0 = lb.tables(0)
    np.testing.assert_array_equal(idx0, np.arange(20, 50))


def test_basis_argument_errors():
    g = synth.hemisphere_directions(30, seed=4)
    b = np.full(30, 1000.0)
    for args, status in (((g, b, 3, 0.0), L.ERR_INVALID_ARG),                      # odd order
                         ((g * 1.01, b, 4, 0.0), L.ERR_INVALID_ARG),               # not unit
                         ((g, np.where(np.arange(30) == 3, 0.0, b), 4, 0.0), L.ERR_INVALID_ARG),  # b = 0
                         ((g, b, 4, -1.0), L.ERR_INVALID_ARG),                     # negative lambda
                         ((g[:10], b[:10], 4, 0.0), L.ERR_RANK_DEFICIENT),         # 10 dirs < 15 coefs
                         ((g, b, 18, 0.0), L.ERR_INVALID_ARG)):                    # order too high
        with pytest.raises(L.DelimitError) as ei:
            L.SHBasis(*args, host_only=True)
        assert ei.value.status == status, args[2:]
    # lambda > 0 regularises the under-determined case
    L.SHBasis(g[:10], b[:10], 4, 0.006, host_only=True)


def test_lsc_tables_match_oracle(table3):
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 8, 0.006, host_only=True)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    for order_in, window, R, Sec, rad in ((8, "adjacent", 4, 12, np.deg2rad(25)), (4, "same", 1, 5, np.pi / 5),
                                          (6, "all", 3, 8, np.deg2rad(30))):
        s_in = 3 if window != "all" else 2
        lg = L.LSCGeometry(lb, order_in, s_in, rad, R, Sec, window, host_only=True)
        og = olsc.LSCOracle(ob, order_in, s_in, rad, R, Sec, window)
        M, q = og.collapse_mats()
        assert lg.K == og.K == 1 + R * Sec
        for s in range(3):
            t = lg.tables(s)
            np.testing.assert_allclose(t["kpts"], og.kpts[s], rtol=0, atol=1e-14)
            np.testing.assert_allclose(t["M"], M[s], rtol=0, atol=1e-12)
            np.testing.assert_allclose(t["q"], q[s], rtol=0, atol=1e-12)
            ip, ix = olsc.neighbour_csr(og.dirs[s], rad)
            np.testing.assert_array_equal(t["nb_indptr"], ip)
            np.testing.assert_array_equal(t["nb_indices"], ix)
            np.testing.assert_array_equal(t["window"], og.win[s])
            T4 = olsc.kernel_row_index(lb.m, lg.K)
            np.testing.assert_array_equal(t["row_index"], T4[lb.dir_off[s]:lb.dir_off[s] + lb.m[s]])


@pytest.mark.parametrize("order_out,lam,order_in,R,Sec,rad,win", [
    (0, 0.0, 0, 2, 6, np.deg2rad(20), "adjacent"),   # one coefficient per shell
    (8, 0.006, 0, 1, 1, np.deg2rad(20), "all"),      # order-0 input, one-point ring (K = 2)
    (4, 0.0, 4, 1, 1, np.pi / 2, "same"),            # largest radius: every direction a neighbour
    (2, 0.006, 2, 3, 7, np.pi / 2, "adjacent")])
def test_degenerate_lsc_tables_match_oracle(order_out, lam, order_in, R, Sec, rad, win):
    dirs, bvals = synth.multishell_table([30, 30], [1000, 2000], seed=5)
    lb = L.SHBasis(dirs, bvals, order_out, lam, host_only=True)
    ob = osh.SHBasisOracle(dirs, bvals, order_out, lam)
    lg = L.LSCGeometry(lb, order_in, 2, rad, R, Sec, win, host_only=True)
    og = olsc.LSCOracle(ob, order_in, 2, rad, R, Sec, win)
    M, q = og.collapse_mats()
    assert lg.K == 1 + R * Sec
    for s in range(2):
        t = lg.tables(s)
        np.testing.assert_allclose(t["kpts"], og.kpts[s], rtol=0, atol=1e-14)
        np.testing.assert_allclose(t["M"], M[s], rtol=0, atol=1e-12)
        np.testing.assert_allclose(t["q"], q[s], rtol=0, atol=1e-12)
        ip, ix = olsc.neighbour_csr(og.dirs[s], rad)
        np.testing.assert_array_equal(t["nb_indptr"], ip)
        np.testing.assert_array_equal(t["nb_indices"], ix)
    if rad == np.pi / 2:
        assert (np.diff(ip) == 30).all()


def test_resampling_free_tables_match_oracle(table3):
    """Neighbour tables and bins of the resampling-free form are bit-exact against the
    oracle; the per-shell-pair collapse matrices agree to 1e-12."""
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 8, 0.006, host_only=True)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    for order_in, window, R, Sec, rad in ((8, "adjacent", 4, 12, np.deg2rad(25)), (4, "all", 1, 5, np.pi / 5),
                                          (6, "same", 3, 8, np.deg2rad(30))):
        lg = L.LSCGeometry(lb, order_in, 3, rad, R, Sec, window, host_only=True, neighbours=True)
        og = olsc.LSCNeighbourOracle(ob, order_in, 3, rad, R, Sec, window)
        M, q = og.collapse_mats()
        n_entries = 0
        for s in range(3):
            t = lg.tables(s)
            np.testing.assert_allclose(t["M"], np.stack(M[s]), rtol=0, atol=1e-12)
            np.testing.assert_allclose(t["q"], q[s], rtol=0, atol=1e-12)
            for p in range(3):
                ip, ix, bx = lg.neighbour_table(s, p)
                oip, oix, obx = og.nb[s, p]
                np.testing.assert_array_equal(ip, oip)
                np.testing.assert_array_equal(ix, oix)
                np.testing.assert_array_equal(bx, obx)
                n_entries += len(ix)
        assert n_entries > 0
    # the resampled geometry has no neighbour-bin table; shell counts must match
    lg = L.LSCGeometry(lb, 4, 3, 0.4, 2, 6, "same", host_only=True)
    assert L.get().delimit_lsc_neighbour_table(lg.handle, 0, 0, None, None, None) == L.ERR_INVALID_ARG
    with pytest.raises(L.DelimitError):
        L.LSCGeometry(lb, 4, 2, 0.4, 2, 6, "all", host_only=True, neighbours=True)


def test_lsc_argument_errors(table3):
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 4, 0.006, host_only=True)
    for args in ((4, 2, 0.4, 2, 6, "adjacent"),   # adjacent needs shells_in == shells_out
                 (4, 3, 0.0, 2, 6, "same"),       # radius 0
                 (4, 3, 2.0, 2, 6, "same"),       # radius > pi/2
                 (4, 3, 0.4, 0, 6, "same"),       # no rings
                 (5, 3, 0.4, 2, 6, "same")):      # odd order
        with pytest.raises(L.DelimitError) as ei:
            L.LSCGeometry(lb, *args, host_only=True)
        assert ei.value.status == L.ERR_INVALID_ARG


def test_host_only_handles_refuse_compute(table3):
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 4, 0.006, host_only=True)
    st = L.get().delimit_signal2sh(lb.handle, 16, 16, 10, 1, 16, 16, L.F32, L.F32, None)
    assert st == L.ERR_INVALID_ARG
    assert b"HOST_ONLY" in L.get().delimit_last_error()


def test_workspace_size_is_monotone(table3):
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 8, 0.006, host_only=True)
    lg = L.LSCGeometry(lb, 8, 3, np.deg2rad(25), 4, 12, "adjacent", host_only=True)
    a = lg.workspace_size(65536, 16, 64, L.BF16, False)
    b = lg.workspace_size(65536, 16, 64, L.BF16, True)
    assert 0 < a < b
    assert lg.workspace_size(65536, 0, 64, L.BF16, False) == 0


def test_fp32_workspace_holds_the_split_operands(table3):
    """FP32 activations on the tensor cores keep three BF16 parts of the LSC input (and,
    backward, of dY) per voxel: the workspace grows with the voxel count by at least
    3 x 2 bytes per input row (forward) and per input and output row (backward) more
    than the BF16 workspace does."""
    dirs, bvals = table3
    lb = L.SHBasis(dirs, bvals, 8, 0.006, host_only=True)
    lg = L.LSCGeometry(lb, 8, 3, np.deg2rad(25), 4, 12, "adjacent", host_only=True)
    rows_in, rows_out = 3 * 16 * 45, 3 * 64 * 45
    for backward, rows in ((False, rows_in), (True, rows_in + rows_out)):
        grow = {}
        for t in (L.BF16, L.F32):
            grow[t] = lg.workspace_size(2 * 65536, 16, 64, t, backward) - lg.workspace_size(65536, 16, 64, t, backward)
        assert grow[L.F32] - grow[L.BF16] >= 65536 * rows * 3 * 2


def test_eval_only_basis():
    g = synth.hemisphere_directions(30, seed=8)
    b = np.full(30, 1000.0)
    lb = L.SHBasis(g, b, 8, 0.0, host_only=True, eval_only=True)  # 30 directions < 45 coefficients
    B, P, _ = lb.tables(0)
    np.testing.assert_allclose(B, osh.real_sh(8, g), atol=1e-12)
    assert np.all(P == 0)
    with pytest.raises(L.DelimitError):
        L.LSCGeometry(lb, 8, 1, 0.4, 2, 6, "same", host_only=True)


def test_binding_constants_match_header():
    txt = open(os.path.join(ROOT, "include", "delimit.h")).read()
    vals = {m[0]: int(m[1]) for m in re.findall(r"\b(DELIMIT_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    vals |= {m[0]: int(m[1]) for m in re.findall(r"#define\s+(DELIMIT_[A-Z0-9_]+)\s+\(?(-?\d+)u?\)?", txt)}
    for name in ["OK", "ERR_INVALID_ARG", "ERR_RANK_DEFICIENT", "ERR_UNSUPPORTED", "ERR_ALIGNMENT", "ERR_CUDA",
                 "ERR_DEVICE_TIMEOUT", "ERR_OOM", "ERR_WORKSPACE", "F32", "BF16", "HOST_ONLY", "EVAL_ONLY",
                 "WINDOW_SAME", "WINDOW_ADJACENT", "WINDOW_ALL"]:
        assert vals["DELIMIT_" + name] == getattr(L, name), name
    assert vals["DELIMIT_LSC_OPERATOR_READY"] == L.OPERATOR_READY


def test_every_entry_point_refuses_null_pointers_with_a_reason():
    """Each compute or table entry point, given NULL pointers (and non-zero sizes), returns
    INVALID_ARG and leaves a message in delimit_last_error, without touching a device."""
    lib = L.get()
    device_calls = {"delimit_device_error", "delimit_selftest_wait_timeout"}
    no_status = {"delimit_version", "delimit_kernel_launches", "delimit_cuda_core_fallbacks",
                 "delimit_status_string", "delimit_last_error",
                 "delimit_trace_enable", "delimit_trace_summary", "delimit_set_tensor_cores",
                 "delimit_lsc_workspace_size", "delimit_mask_compact_workspace_size",
                 "delimit_sh_basis_destroy", "delimit_lsc_geometry_destroy"}
    ints = (C.c_int, C.c_int64, C.c_size_t, C.c_uint32, C.c_uint64, C.c_long, C.c_uint)
    checked = 0
    for name, (_, args) in sorted(L.SIGNATURES.items()):
        if name in device_calls or name in no_status:
            continue
        vals = [0.0 if a in (C.c_double, C.c_float) else (64 if a in ints else None) for a in args]
        out = {}

        def run():  # the message is thread-local: a fresh thread starts without one
            out["st"] = getattr(lib, name)(*vals)
            out["msg"] = lib.delimit_last_error()
        t = threading.Thread(target=run)
        t.start()
        t.join()
        assert out["st"] == L.ERR_INVALID_ARG, (name, out["st"])
        assert out["msg"], name
        checked += 1
    assert checked >= 20
    # NULL handles are accepted by destroy (no-op) and give a zero workspace size
    assert lib.delimit_sh_basis_destroy(None) == L.OK and lib.delimit_lsc_geometry_destroy(None) == L.OK
    assert lib.delimit_lsc_workspace_size(None, 64, 1, 1, L.BF16, 0) == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: with the shared library absent and its build failing, loading raises,
    and a layer call on host tensors raises instead of computing anything on the CPU."""
    from paper_1808_01517_gb300 import build as _build
    from paper_1808_01517_gb300 import layers
    import torch

    def no_build(*args, **kwargs):
        raise RuntimeError("nvcc unavailable")
    monkeypatch.delenv("DELIMIT_LIB", raising=False)
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "libdelimit.so"))
    monkeypatch.setattr(_build, "build", no_build)
    with pytest.raises(RuntimeError, match="nvcc unavailable"):
        L.get()
    monkeypatch.undo()
    dirs, bvals = synth.multishell_table([30], [1000], seed=1)
    basis = L.SHBasis(dirs, bvals, 4, 0.006, host_only=True)
    if not torch.cuda.is_available():
        with pytest.raises(Exception):
            layers.transform("signal2sh", basis, torch.zeros((30, 64)), 1)


def test_tensor_core_policy_modes():
    """delimit_set_tensor_cores takes 0 (CUDA cores), 1 (tensor cores where a kernel takes
    the call) and 2 (tensor cores required) and refuses anything else."""
    lib = L.get()
    try:
        for m in (0, 1, 2):
            assert lib.delimit_set_tensor_cores(m) == L.OK
        for m in (-1, 3):
            assert lib.delimit_set_tensor_cores(m) == L.ERR_INVALID_ARG
        assert isinstance(L.cuda_core_fallbacks(), int)
    finally:
        L.set_tensor_cores(True)


def test_gemm_cluster_setting():
    """delimit_set_gemm_cluster takes 0 (each GEMM's default), 1 (single CTAs) and 2 (CTA
    pairs) and refuses anything else with a message."""
    lib = L.get()
    try:
        for n in (0, 1, 2):
            assert lib.delimit_set_gemm_cluster(n) == L.OK
        for n in (-1, 3, 4):
            assert lib.delimit_set_gemm_cluster(n) == L.ERR_INVALID_ARG
            assert b"cluster" in lib.delimit_last_error()
    finally:
        L.set_gemm_cluster(0)
