"""FP32 arithmetic on the BF16 tensor cores, modelled on the CPU.

The FP32 paths (the split-operand LSC GEMMs, the FP32 transforms, the tensor-core
operator build) split every FP32 operand into three BF16 parts by rounding to nearest
and subtracting: x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); and they keep
the six part products a_i b_j with i + j <= 2 (the other three are below 2^-24 of the
leading one).  For FP32 inputs the split is exact (24 significant bits in three pieces
of 8), and the six products give the product sum to within a few units of 2^-24 of the
sum of magnitudes: FP32-level accuracy before the FP32 accumulation in TMEM.
"""
import numpy as np

from tests.test_bf16_error_model import bf16

# the six part products kept, as (part of a, part of b)
TERMS = [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (2, 0)]


def split3(x):
    x = np.asarray(x, np.float32).astype(np.float64)
    x0 = bf16(x)
    x1 = bf16(x - x0)
    x2 = bf16(x - x0 - x1)
    return x0, x1, x2


def _fp32_samples(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))
    return x.astype(np.float32)


def test_three_part_split_of_fp32_is_exact():
    x = _fp32_samples(200_000, 1)
    x0, x1, x2 = split3(x)
    xd = x.astype(np.float64)
    assert np.array_equal(x0 + x1 + x2, xd)
    # each part is a BF16 value, and each is at most 2^-8 of the one before
    for p in (x0, x1, x2):
        assert np.array_equal(bf16(p), p)
    nz = x0 != 0
    assert (np.abs(x1[nz]) <= np.abs(x0[nz]) * 2.0 ** -8).all()
    nz = x1 != 0
    assert (np.abs(x2[nz]) <= np.abs(x1[nz]) * 2.0 ** -8).all()


def test_six_part_products_reach_fp32_accuracy():
    rng = np.random.default_rng(2)
    for K in (1, 49, 64, 2025):
        a = rng.standard_normal((64, K)).astype(np.float32)
        b = rng.standard_normal((K, 16)).astype(np.float32)
        pa, pb = split3(a), split3(b)
        approx = sum(pa[i] @ pb[j] for i, j in TERMS)
        exact = a.astype(np.float64) @ b.astype(np.float64)
        mag = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
        assert (np.abs(approx - exact) <= 3 * 2.0 ** -24 * mag).all()
        # the leading product alone (plain BF16 operands) is far from FP32 level
        lead = pa[0] @ pb[0]
        assert np.abs(lead - exact).max() > 100 * 2.0 ** -24 * mag.max()


def test_dropped_products_are_below_fp32_resolution():
    x = _fp32_samples(100_000, 3)
    y = _fp32_samples(100_000, 4)
    px, py = split3(x)[:3], split3(y)[:3]
    xy = np.abs(x.astype(np.float64) * y.astype(np.float64))
    for i, j in [(1, 2), (2, 1), (2, 2)]:
        assert (np.abs(px[i] * py[j]) <= 2.0 ** -24 * xy * 1.0001).all()
