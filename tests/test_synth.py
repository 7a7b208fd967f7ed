"""The seeded input generators: determinism, shapes and value ranges."""
import numpy as np

from paper_1808_01517_gb300 import synth


def test_directions_are_unit_upper_hemisphere_and_seeded():
    g = synth.hemisphere_directions(90, seed=1)
    np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-15)
    assert np.all(g[:, 2] >= 0)
    np.testing.assert_array_equal(g, synth.hemisphere_directions(90, seed=1))
    assert not np.allclose(g, synth.hemisphere_directions(90, seed=2))


def test_multishell_table_groups_shells():
    d, b = synth.multishell_table([90, 90, 90], [1000, 2000, 3000])
    assert d.shape == (270, 3) and list(np.unique(b)) == [1000, 2000, 3000]
    assert np.all(b[:90] == 1000) and np.all(b[180:] == 3000)


def test_fibre_signal_range_and_determinism():
    d, b = synth.multishell_table([30, 30], [1000, 3000])
    s = synth.fibre_signal(d, b, 500, seed=3, snr=1e9)  # noise-free limit
    assert s.shape == (500, 60) and s.dtype == np.float32
    assert np.all(s > 0) and np.all(s <= 1.0 + 1e-6)
    # higher b attenuates more on average
    assert s[:, 30:].mean() < s[:, :30].mean()
    s2 = synth.fibre_signal(d, b, 500, seed=3, snr=1e9, chunk=77)
    np.testing.assert_allclose(s, s2, atol=1e-6)
    noisy = synth.fibre_signal(d, b, 500, seed=3, snr=20)
    assert 0.02 < np.std(noisy - s) < 0.08


def test_perturbed_tables_stay_close():
    d, _ = synth.multishell_table([90], [1000])
    p = synth.perturbed_table(d, np.deg2rad(5), np.deg2rad(2), seed=1, sub=3)
    ang = np.degrees(np.arccos(np.clip(np.sum(p * d, 1), -1, 1)))
    assert ang.max() <= 7.0 + 1e-9 and ang.mean() > 0.1
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-14)


def test_mask_size():
    m = synth.ellipsoid_mask((40, 50, 40), 20000, seed=1)
    assert m.sum() == 20000
