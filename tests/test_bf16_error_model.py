"""Error budget of the BF16 path, on the CPU: the chain (Signal2SH -> LSC -> SH2Signal,
forward and backward) written in the collapsed form with every tensor the BF16 path
stores rounded to BF16 (round to nearest even): the transform operators P_s and B_s,
the collapsed LSC operator W, and the activations c_in, c_out, s_out, dc_out, dc_in,
ds_in.  Products are exact (FP64) in the model; the library accumulates in FP32.

At the benchmark workload (3 x 90 directions, order 8, 16 -> 64 channels, adjacent
shells, 4 x 12 kernel) on 64 voxels the model gives relative L2 errors of about 4.4e-3
(s_out) and 4.2e-3 (ds_in) against the unrounded chain; the library's BF16 chain
measures the same against the FP64 oracle.  So the BF16 path's error is its storage
rounding, below the 1e-2 tolerance with room to spare, and the FP32 accumulation adds
nothing visible.  With rounding switched off the model is the oracle's chain (a check
of the model's structure against the literal route).
"""
import numpy as np

from oracle import lsc as olsc
from oracle import sh as osh
from paper_1808_01517_gb300 import synth


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def exact(x):
    return np.asarray(x, np.float64)


def chain(ob, og, sig, w, b, ds, r):
    """sig [V, Ci, dirs], ds [V, Co, dirs] -> (s_out [V, Co, dirs], ds_in [V, Ci, dirs]),
    every stored tensor passed through r."""
    S = ob.n_shells
    M, q = og.collapse_mats()
    P = [r(p) for p in ob.P]
    B = [r(x) for x in ob.B]
    V, Ci, Co = sig.shape[0], sig.shape[1], w.shape[0]
    c_in = np.stack([r(sig[:, :, rows] @ P[s].T) for s, rows in enumerate(ob.rows)], axis=2)
    W = {(s, p): r(np.einsum("ack,kxy->axcy", w[:, s, :, p, :], M[s]))
         for s in range(S) for p in range(S) if og.win[s, p]}
    c_out = np.zeros((V, Co, S, ob.n_coef))
    for s in range(S):
        acc = sum(np.einsum("axcy,vcy->vax", W[s, p], c_in[:, :, p, :]) for p in range(S) if og.win[s, p])
        c_out[:, :, s, :] = r(acc + b[None, :, s, None] * q[s][None, None, :])
    s_out = np.empty((V, Co, sig.shape[2]))
    for s, rows in enumerate(ob.rows):
        s_out[:, :, rows] = r(c_out[:, :, s, :] @ B[s].T)
    dc_out = np.stack([r(ds[:, :, rows] @ B[s]) for s, rows in enumerate(ob.rows)], axis=2)
    dc_in = np.zeros((V, Ci, S, ob.n_coef))
    for p in range(S):
        acc = sum(np.einsum("axcy,vax->vcy", W[s, p], dc_out[:, :, s, :]) for s in range(S) if og.win[s, p])
        dc_in[:, :, p, :] = r(acc)
    ds_in = np.empty_like(sig)
    for s, rows in enumerate(ob.rows):
        ds_in[:, :, rows] = r(dc_in[:, :, s, :] @ P[s])
    return s_out, ds_in


def _rel(a, ref):
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def test_bf16_rounding_is_to_nearest_even():
    one = 1.0
    ulp = 2.0 ** -7  # BF16 spacing just above 1
    assert bf16(one + ulp * 0.49) == one and bf16(one + ulp * 0.51) == one + ulp
    assert bf16(one + ulp * 0.5) == one                  # tie to the even neighbour
    assert bf16(one + ulp * 1.5) == one + 2 * ulp        # tie to the even neighbour
    assert bf16(-3.0) == -3.0


def test_bf16_storage_model_of_the_benchmark_chain():
    dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=1808)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    og = olsc.LSCOracle(ob, 8, 3, np.deg2rad(25), 4, 12, "adjacent")
    V, Ci, Co = 64, 16, 64
    # inputs as the BF16 chain holds them (its error is measured from these same values)
    sig = bf16(synth.fibre_signal(dirs, bvals, V * Ci, seed=1808).reshape(Ci, V, -1).transpose(1, 0, 2))
    ds = bf16(synth.gaussian((V, Co, 270), 0.1, seed=1808, tag="grads"))
    w = synth.gaussian((Co, 3, Ci, 3, og.K), 0.1, seed=1808).astype(np.float32).astype(np.float64)
    b = synth.gaussian((Co, 3), 0.1, seed=1809).astype(np.float32).astype(np.float64)

    ref_s, ref_d = chain(ob, og, sig, w, b, ds, exact)
    # without rounding the model is the oracle's chain (literal route)
    c_in = ob.signal2sh(sig)
    np.testing.assert_allclose(ref_s, ob.sh2signal(og.forward(c_in, w, b)), rtol=0, atol=1e-12 * np.abs(ref_s).max())
    dc_in, _, _ = og.backward(c_in, w, ob.sh2signal_backward(ds))
    lit_d = ob.signal2sh_backward(dc_in)
    np.testing.assert_allclose(ref_d, lit_d, rtol=0, atol=1e-12 * np.abs(ref_d).max())

    got_s, got_d = chain(ob, og, sig, w, b, ds, bf16)
    e_s, e_d = _rel(got_s, ref_s), _rel(got_d, ref_d)
    # a handful of BF16 roundings (unit roundoff 2^-8) in series: a few 1e-3, well below 1e-2
    assert 2e-3 < e_s < 7e-3 and 2e-3 < e_d < 7e-3, (e_s, e_d)


def chain_fp32_forward(ob, og, sig, w, b):
    """The forward chain with every operand and every operation in float32 (numpy's float32
    BLAS accumulates in float32): the error level of FP32 arithmetic itself."""
    f = np.float32
    S = ob.n_shells
    M, q = og.collapse_mats()
    P, B = [p.astype(f) for p in ob.P], [x.astype(f) for x in ob.B]
    M, q = [m.astype(f) for m in M], [x.astype(f) for x in q]
    sig, w, b = sig.astype(f), w.astype(f), b.astype(f)
    V, Co = sig.shape[0], w.shape[0]
    c_in = np.stack([sig[:, :, rows] @ P[s].T for s, rows in enumerate(ob.rows)], axis=2)
    c_out = np.zeros((V, Co, S, ob.n_coef), f)
    for s in range(S):
        acc = np.zeros((V, Co * ob.n_coef), f)
        for p in range(S):
            if og.win[s, p]:
                W = np.einsum("ack,kxy->axcy", w[:, s, :, p, :], M[s]).astype(f)
                acc += c_in[:, :, p, :].reshape(V, -1) @ W.reshape(Co * ob.n_coef, -1).T
        c_out[:, :, s, :] = acc.reshape(V, Co, -1) + b[None, :, s, None] * q[s][None, None, :]
    s_out = np.empty((V, Co, sig.shape[2]), f)
    for s, rows in enumerate(ob.rows):
        s_out[:, :, rows] = c_out[:, :, s, :] @ B[s].T
    return s_out.astype(np.float64)


def test_fp32_arithmetic_error_level():
    """FP32 storage alone costs ~1e-7 here; FP32 accumulation of the long sums (K up to
    2,160 per LSC output) brings FP32 arithmetic to a few 1e-7, the level of the
    library's FP32 paths (about 1e-6), an order of magnitude below the 1e-5 tolerance."""
    dirs, bvals = synth.multishell_table([90, 90, 90], [1000, 2000, 3000], seed=1808)
    ob = osh.SHBasisOracle(dirs, bvals, 8, 0.006)
    og = olsc.LSCOracle(ob, 8, 3, np.deg2rad(25), 4, 12, "adjacent")
    V, Ci, Co = 64, 16, 64
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)  # noqa: E731
    sig = f32(synth.fibre_signal(dirs, bvals, V * Ci, seed=1808).reshape(Ci, V, -1).transpose(1, 0, 2))
    w = f32(synth.gaussian((Co, 3, Ci, 3, og.K), 0.1, seed=1808))
    b = f32(synth.gaussian((Co, 3), 0.1, seed=1809))
    ds = f32(synth.gaussian((V, Co, 270), 0.1, seed=1808, tag="grads"))
    ref_s, _ = chain(ob, og, sig, w, b, ds, exact)
    st_s, _ = chain(ob, og, sig, w, b, ds, f32)
    assert _rel(st_s, ref_s) < 3e-7
    e = _rel(chain_fp32_forward(ob, og, sig, w, b), ref_s)
    assert 5e-8 < e < 3e-6, e
