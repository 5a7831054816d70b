"""Pins of the WNNM oracle against constructions it does not compute itself: a
group built from known singular vectors and values (the expected estimate follows
from the stated shrinkage formula without any SVD), the sigma -> 0 identity, the
large-sigma collapse to the group mean, constant images, and the reduction of the
WNNM ADMM to Algorithm 1 with an identity u-step (Tikhonov at lambda = 0)."""
import numpy as np
import pytest

import oracle
from oracle import wnnm as wn


def _orth(rng, n, k):
    q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return q


@pytest.mark.parametrize("m,r,sigma", [(16, 3, 0.05), (9, 5, 0.02), (4, 2, 0.1)])
def test_group_from_known_singular_values(m, r, sigma):
    rng = np.random.default_rng(m + r)
    U = _orth(rng, 64, r)
    # right singular vectors orthogonal to the all-ones vector: the group mean is mu
    P = np.eye(m) - np.ones((m, m)) / m
    V = np.linalg.qr(P @ rng.standard_normal((m, r)))[0]
    s = np.sort(rng.uniform(0.05, 2.0, r))[::-1]
    mu = rng.uniform(0, 1, (64, 1))
    Y = (U * s) @ V.T + mu
    sh = np.sqrt(np.maximum(s * s - 64 * sigma * sigma, 0.0))
    x = np.maximum(s - sigma * sigma * 2 * np.sqrt(2) * np.sqrt(m) / (sh + 1e-8), 0.0)
    expected = (U * x) @ V.T + mu
    np.testing.assert_allclose(wn.wnnm_group(Y, sigma), expected, rtol=0, atol=1e-12)


def test_large_sigma_collapses_to_group_mean():
    rng = np.random.default_rng(2)
    Y = rng.random((64, 12))
    np.testing.assert_allclose(wn.wnnm_group(Y, 50.0), np.repeat(Y.mean(1, keepdims=True), 12, 1),
                               rtol=0, atol=1e-12)


def test_vanishing_sigma_is_identity():
    rng = np.random.default_rng(3)
    img = rng.random((30, 27))
    np.testing.assert_allclose(wn.wnnm_slice(img, 1e-9), img, rtol=0, atol=1e-9)


def test_constant_and_small_images():
    np.testing.assert_allclose(wn.wnnm_slice(np.full((20, 17), 0.3), 0.05),
                               np.full((20, 17), 0.3), rtol=0, atol=1e-14)
    small = np.random.default_rng(4).random((7, 30))
    np.testing.assert_array_equal(wn.wnnm_slice(small, 0.05), small)


def test_denoises():
    rng = np.random.default_rng(5)
    yy, xx = np.mgrid[0:40, 0:40]
    clean = 0.5 + 0.3 * np.sin(xx / 4.0) * np.cos(yy / 5.0)
    noisy = clean + 0.05 * rng.standard_normal(clean.shape)
    out = wn.wnnm_slice(noisy, 0.05)
    assert np.linalg.norm(out - clean) < 0.6 * np.linalg.norm(noisy - clean)


def test_admm_with_identity_u_step_is_tikhonov_at_zero_lambda():
    rng = np.random.default_rng(6)
    Z, H, W = 4, 12, 10
    masks = (rng.random((Z, H, W)) < 0.5).astype(np.uint8)
    b = rng.random((1, H, W))
    v, *_ = wn.admm_wnnm(b, masks, Z, rho=1.0, gamma=0.0, sigma=1e-12, iters=5)
    v_r, *_ = oracle.admm(b, masks, Z, rho=1.0, lam=0.0, gamma=0.0, iters=5,
                          denoiser="tikhonov")
    np.testing.assert_allclose(v, v_r, rtol=0, atol=1e-9)
