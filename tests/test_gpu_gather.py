"""Signal2SH of masked voxels with the b = 0 normalisation fused into the load
(delimit_signal2sh_gather) against the FP64 oracle: sh[:, k] = P (dwi[:, idx[k]] / b0[idx[k]]).
Voxels with b0 <= 0 give zero coefficients; an index outside the volume gives zeros
and an INVALID_ARG report from delimit_device_error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sh as osh  # noqa: E402
from paper_1808_01517_gb300 import _lib as L  # noqa: E402
from paper_1808_01517_gb300 import layers, synth  # noqa: E402
from tests._layout import TOL_BF16, TOL_F32, rel_l2, rows_to_sh, sig_to_rows  # noqa: E402

pytestmark = pytest.mark.gpu


def _volume(n_src, C, seed):
    dirs, bvals = synth.multishell_table([45, 60], [1000, 2000], seed=seed)
    rng = np.random.default_rng(seed)
    sig = synth.fibre_signal(dirs, bvals, n_src * C, seed=seed).astype(np.float64)  # [n_src*C, dirs]
    sig = sig.reshape(C, n_src, -1).transpose(1, 0, 2)  # [n_src, C, dirs], normalised
    s0 = rng.uniform(400.0, 1600.0, n_src)
    s0[rng.random(n_src) < 0.05] = 0.0  # some voxels without signal
    dwi = sig * np.maximum(s0, 1.0)[:, None, None]  # raw signal
    mask = rng.random(n_src) < 0.4
    return dirs, bvals, sig, dwi, s0, mask


@pytest.mark.parametrize("prec,tol", [("f32", TOL_F32), ("bf16", TOL_BF16)])
@pytest.mark.parametrize("with_b0", [True, False])
def test_gather_matches_oracle(prec, tol, with_b0):
    n_src, C = 5003, 2
    dirs, bvals, sig, dwi, s0, mask = _volume(n_src, C, seed=41)
    ob = osh.SHBasisOracle(dirs, bvals, 6, 0.006)
    lb = L.SHBasis(dirs, bvals, 6, 0.006)
    src = dwi if with_b0 else sig
    dt = torch.float32 if prec == "f32" else torch.bfloat16
    vol = layers.empty_act(C * dirs.shape[0], n_src, dt)
    vol.copy_(torch.from_numpy(sig_to_rows(src, ob.m)).to(dt))
    idx = np.flatnonzero(mask)
    index = torch.from_numpy(idx).cuda()
    b0 = torch.from_numpy(s0.astype(np.float32)).cuda() if with_b0 else None
    got = layers.signal2sh_gather(lb, vol, index, b0=b0, channels=C, out_dtype=torch.float32)
    torch.cuda.synchronize()
    # the oracle sees the same (rounded) inputs, divided in FP64
    x = torch.from_numpy(sig_to_rows(src, ob.m)).to(dt).double().numpy()  # rows x n_src
    cols = x[:, idx]
    if with_b0:
        b = s0[idx].astype(np.float32).astype(np.float64)
        cols = np.where(b > 0, cols / np.where(b > 0, b, 1.0), 0.0)
    # library signal rows (s, c, i) -> oracle [V, C, dirs]
    sig_sel = np.empty((len(idx), C, dirs.shape[0]))
    r0 = off = 0
    for m in ob.m:
        sig_sel[:, :, off:off + m] = cols[r0:r0 + C * m].reshape(C, m, -1).transpose(2, 0, 1)
        r0 += C * m
        off += m
    ref = ob.signal2sh(sig_sel)  # [n, C, S, N]
    got_sh = rows_to_sh(got.cpu().numpy(), ob.n_shells, C, ob.n_coef)
    assert rel_l2(got_sh, ref) <= tol
    if with_b0:
        zero = s0[idx] <= 0
        assert zero.any() and np.all(got_sh[zero] == 0)
    st, code = L.device_error(0)
    assert st == L.OK and code == 0


def test_gather_index_out_of_range_reports_and_zeroes():
    n_src, C = 300, 1
    dirs, bvals, sig, dwi, s0, mask = _volume(n_src, C, seed=43)
    lb = L.SHBasis(dirs, bvals, 4, 0.006)
    vol = layers.empty_act(dirs.shape[0], n_src, torch.float32)
    vol.copy_(torch.from_numpy(sig[:, 0, :].T.copy()).float())
    index = torch.tensor([0, 5, n_src + 7, 9, -3], dtype=torch.int64, device="cuda")
    got = layers.signal2sh_gather(lb, vol, index, channels=1, out_dtype=torch.float32)
    st, code = L.device_error(0)
    assert st == L.ERR_INVALID_ARG and code == 0x2100
    g = got.cpu().numpy()
    assert np.all(g[:, 2] == 0) and np.all(g[:, 4] == 0) and np.any(g[:, 1] != 0)
    st, code = L.device_error(0)  # cleared by the read
    assert st == L.OK and code == 0
