"""Pins of the oracle's BM3D u-step against independent restatements: exhaustive
block matching, scipy's orthonormal DCT, an explicit Haar matrix, numpy's Kaiser
window, a dense-matrix BM3D stage, and the limits (zero threshold, vanishing
noise level, constant images)."""
import numpy as np
import pytest

from tests.dense import (bm3d_brute_force_match, bm3d_refs, bm3d_stage_dense, dct_matrix,
                         haar_matrix)


def _blobs(seed, H, W, noise=0.05):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.full((H, W), 0.1)
    for _ in range(max(2, H * W // 120)):
        cy, cx, s = rng.uniform(0, H), rng.uniform(0, W), rng.uniform(1.5, 4)
        img += rng.uniform(0.2, 1) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * s * s))
    img /= img.max()
    return img, (img + noise * rng.standard_normal((H, W))).astype(np.float32).astype(np.float64)


def test_reference_grid(oracle):
    for n in (8, 9, 11, 20, 23, 64):
        assert oracle.bm3d_ref_positions(n) == bm3d_refs(n)
    assert oracle.bm3d_ref_positions(20) == [0, 3, 6, 9, 12]
    assert oracle.bm3d_ref_positions(11) == [0, 3]


def test_dct_is_scipy_orthonormal_dct(oracle):
    C = oracle.bm3d_dct8()
    np.testing.assert_allclose(C, dct_matrix(), atol=1e-15)
    np.testing.assert_allclose(C @ C.T, np.eye(8), atol=1e-14)


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16])
def test_group_transform_equals_dense_matrices(oracle, L):
    import scipy.fft

    g = np.random.default_rng(L).standard_normal((L, 8, 8))
    t = oracle.bm3d_transform(g)
    d2 = np.stack([scipy.fft.dctn(p, norm="ortho") for p in g])
    exp = np.einsum("kl,lab->kab", haar_matrix(L), d2)
    np.testing.assert_allclose(t, exp, atol=1e-13)
    np.testing.assert_allclose(oracle.bm3d_transform(t, inverse=True), g, atol=1e-13)
    Hm = haar_matrix(L)
    np.testing.assert_allclose(Hm @ Hm.T, np.eye(L), atol=1e-14)


def test_kaiser_window_is_numpy_kaiser(oracle):
    k = np.kaiser(8, 2.0)
    np.testing.assert_allclose(oracle.bm3d_kaiser(), np.outer(k, k), atol=1e-14)


@pytest.mark.parametrize("H,W,seed", [(16, 16, 0), (24, 30, 1), (20, 9, 2)])
@pytest.mark.parametrize("stage", [1, 2])
def test_match_lists_equal_exhaustive_search(oracle, H, W, seed, stage):
    _, noisy = _blobs(seed, H, W, noise=0.02)
    idx, cnt = oracle.bm3d_match(noisy, stage)
    groups = bm3d_brute_force_match(noisy, 2500 if stage == 1 else 400)
    assert len(groups) == len(cnt)
    for r, grp in enumerate(groups):
        assert cnt[r] == len(grp)
        assert idx[r, :cnt[r]].tolist() == grp
        assert np.all(idx[r, cnt[r]:] == -1)
    assert cnt.max() > 1  # some real groups formed


def test_ties_break_on_linear_index(oracle):
    """A constant image makes every candidate tie at SSD 0: the lowest indices win."""
    img = np.full((20, 20), 0.3)
    idx, cnt = oracle.bm3d_match(img, 1)
    W = 20
    # reference (0, 0): the next 15 positions in row-major order of the window
    exp = [0] + [ci * W + cj for ci in range(0, 13) for cj in range(0, 13) if (ci, cj) != (0, 0)][:15]
    assert idx[0].tolist() == exp and cnt[0] == 16


@pytest.mark.parametrize("H,W,seed", [(16, 20, 3), (21, 18, 4)])
def test_stages_equal_dense_restatement(oracle, H, W, seed):
    _, noisy = _blobs(seed, H, W, noise=0.04)
    sigma = 0.04
    basic = oracle.bm3d_stage(noisy, sigma)
    np.testing.assert_allclose(basic, bm3d_stage_dense(noisy, sigma), atol=1e-12)
    basic32 = basic.astype(np.float32).astype(np.float64)
    final = oracle.bm3d_stage(noisy, sigma, guide=basic32)
    np.testing.assert_allclose(final, bm3d_stage_dense(noisy, sigma, guide=basic32), atol=1e-12)
    np.testing.assert_allclose(oracle.bm3d(noisy, sigma),
                               oracle.bm3d_stage(noisy, sigma, guide=basic), atol=0)


def test_zero_threshold_and_vanishing_noise_are_identity(oracle):
    _, noisy = _blobs(5, 24, 26)
    np.testing.assert_allclose(oracle.bm3d_stage(noisy, 0.05, lambda3d=0.0), noisy, atol=1e-13)
    np.testing.assert_allclose(oracle.bm3d_stage(noisy, 1e-7, guide=noisy), noisy, atol=1e-9)


def test_constant_image_preserved(oracle):
    c = np.full((19, 23), 0.42)
    np.testing.assert_allclose(oracle.bm3d_stage(c, 0.05), c, atol=1e-13)
    np.testing.assert_allclose(oracle.bm3d(c, 0.05), c, atol=1e-4)


def test_small_images_unchanged(oracle):
    x = np.random.default_rng(0).random((7, 30))
    np.testing.assert_array_equal(oracle.bm3d(x, 0.05), x)


def test_denoises(oracle):
    clean, noisy = _blobs(6, 48, 48, noise=0.05)
    out = oracle.bm3d(noisy, 0.05)
    err = lambda a: np.sqrt(np.mean((a - clean) ** 2))  # noqa: E731
    assert err(out) < 0.6 * err(noisy)
