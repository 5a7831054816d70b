"""Seeded synthetic inputs: determinism, shapes, value ranges."""
import numpy as np

import synth


def test_generate_is_deterministic_and_in_range():
    w = synth.Workload("t", 4, 24, 20, mask_p=0.3, peak=50.0, sigma_g=0.02, seed=5, n_blobs=12,
                       drift=True)
    a, b = synth.generate(w), synth.generate(w)
    for k in ("x", "masks", "b"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["x"].shape == (4, 24, 20) and a["masks"].shape == (4, 24, 20)
    assert a["b"].shape == (1, 24, 20) and a["b"].dtype == np.float32
    assert a["x"].max() == 1.0 and a["x"].min() > 0.0
    assert set(np.unique(a["masks"])) <= {0, 1}
    assert 0.2 < a["masks"].mean() < 0.4
    np.testing.assert_array_equal(a["b64"], a["b"].astype(np.float64))


def test_noise_free_acquisition_sums_masked_planes():
    w = synth.Workload("t", 6, 10, 9, n_shots=2, per_slice_masks=False, peak=None, seed=3,
                       n_blobs=5)
    g = synth.generate(w)
    x, m = g["x"], g["masks"]
    assert m.shape == (3, 10, 9)
    for j in range(2):
        exp = sum(m[r] * x[j * 3 + r] for r in range(3))
        np.testing.assert_allclose(g["b64"][j], exp.astype(np.float32), rtol=0, atol=0)


def test_blob_count_scales_with_volume():
    assert synth.blob_count(8, 128, 128) == 200
    assert synth.blob_count(16, 512, 512) == 6400
    assert synth.blob_count(32, 1024, 1024) == 20000
