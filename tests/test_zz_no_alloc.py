"""The allocation-free LSC forward (delimit_lsc_forward_noalloc) against the regular one.

Callers that cannot allocate device memory where they run the layer (for
example inside a region where the CUDA allocator must not be called, or under
a fixed memory budget) use this entry point: its scratch is a fixed 16 MiB
array inside the library instead of a caller-supplied workspace.  These tests
call it through the C ABI twice in a row, with different weights and inputs,
and compare each result with delimit_lsc_forward's on the same inputs; they
also check that sizes beyond the fixed scratch are refused.  Collected last
(file name) so that a failure here does not hide the other GPU tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2  # noqa: E402

pytestmark = pytest.mark.gpu


def _regular_forward(geom, x, w, b, ci, co, out):
    ws_n = geom.workspace_size(x.shape[1], ci, co, layers._code(x), False)
    ws = torch.empty(ws_n + 256, dtype=torch.uint8, device="cuda")
    wsp = (ws.data_ptr() + 255) // 256 * 256
    L.check(L.get().delimit_lsc_forward(geom.handle, x.data_ptr(), w.data_ptr(), b.data_ptr(), out.data_ptr(),
                                        x.shape[1], ci, co, x.stride(0), out.stride(0), layers._code(x), 0, wsp, ws_n,
                                        torch.cuda.current_stream().cuda_stream), "delimit_lsc_forward")


def _noalloc_forward(geom, x, w, b, ci, co, out):
    return L.get().delimit_lsc_forward_noalloc(geom.handle, x.data_ptr(), w.data_ptr(), b.data_ptr(), out.data_ptr(),
                                               x.shape[1], ci, co, x.stride(0), out.stride(0), layers._code(x),
                                               torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("dtype,tol", [(torch.bfloat16, TOL_BF16), (torch.float32, TOL_F32)])
def test_noalloc_forward_matches_regular_forward_twice(dtype, tol):
    # three shells of 40 directions, order 8, adjacent-shell mixing, 2 -> 4 channels, 4 x 12 kernel
    dirs, bvals = synth.multishell_table([40, 40, 40], [1000, 2000, 3000], seed=21)
    basis = L.SHBasis(dirs, bvals, 8, 0.006)
    geom = L.LSCGeometry(basis, 8, 3, np.deg2rad(25), 4, 12, "adjacent")
    ci, co, V = 2, 4, 1000
    assert geom.workspace_size(V, ci, co, layers._code(torch.empty(0, dtype=dtype)), False) <= 16 << 20
    for call in range(2):
        x = layers.empty_act(3 * ci * 45, V, dtype)
        x.copy_(torch.from_numpy(synth.gaussian((3 * ci * 45, V), 1.0, seed=30 + call, tag="coeffs")).to(dtype))
        w = torch.from_numpy(synth.gaussian((co, 3, ci, 3, geom.K), 0.1, seed=40 + call)).float().cuda()
        b = torch.from_numpy(synth.gaussian((co, 3), 0.1, seed=50 + call)).float().cuda()
        ref = layers.empty_act(3 * co * 45, V, dtype)
        got = layers.empty_act(3 * co * 45, V, dtype)
        _regular_forward(geom, x, w, b, ci, co, ref)
        st = _noalloc_forward(geom, x, w, b, ci, co, got)
        assert st == L.OK, L.get().delimit_last_error()
        torch.cuda.synchronize()
        err = rel_l2(got.float().cpu().numpy(), ref.float().cpu().numpy())
        assert err <= tol, (call, err)
    st, code = L.device_error(0)
    assert st == L.OK and code == 0


def test_noalloc_forward_refuses_sizes_beyond_its_scratch():
    dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=22)
    basis = L.SHBasis(dirs, bvals, 8, 0.006)
    geom = L.LSCGeometry(basis, 8, 3, np.deg2rad(25), 4, 12, "adjacent")
    ci, co, V = 16, 64, 256  # collapsed operator of about 75 MB
    assert geom.workspace_size(V, ci, co, L.BF16, False) > 16 << 20
    x = layers.empty_act(3 * ci * 45, V, torch.bfloat16)
    y = layers.empty_act(3 * co * 45, V, torch.bfloat16)
    w = torch.zeros((co, 3, ci, 3, geom.K), device="cuda")
    b = torch.zeros((co, 3), device="cuda")
    st = _noalloc_forward(geom, x, w, b, ci, co, y)
    assert st == L.ERR_WORKSPACE
    assert b"16 MiB" in L.get().delimit_last_error()
