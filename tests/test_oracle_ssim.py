"""Pins of the oracle's 3-D SSIM (Sec. IV, evaluation metrics) against things
other than its own separable passes: the definition written out voxel by voxel
with an explicit clipped 11^3 window, scipy's Gaussian filter with the clipped
window's renormalisation, the closed form for constant volumes, identity and
symmetry."""
import itertools

import numpy as np
import pytest

import oracle

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _brute(x, y):
    """The local ssim at every voxel from the explicit clipped Gaussian window."""
    Z, H, W = x.shape
    k = np.arange(-5, 6)
    g1 = np.exp(-(k ** 2) / (2 * 1.5 ** 2))
    total = 0.0
    out = np.empty_like(x)
    for z, i, j in itertools.product(range(Z), range(H), range(W)):
        z0, z1 = max(0, z - 5), min(Z, z + 6)
        i0, i1 = max(0, i - 5), min(H, i + 6)
        j0, j1 = max(0, j - 5), min(W, j + 6)
        w = (g1[z0 - z + 5:z1 - z + 5, None, None] * g1[None, i0 - i + 5:i1 - i + 5, None] *
             g1[None, None, j0 - j + 5:j1 - j + 5])
        w = w / w.sum()
        px, py = x[z0:z1, i0:i1, j0:j1], y[z0:z1, i0:i1, j0:j1]
        mx, my = (w * px).sum(), (w * py).sum()
        vx = (w * (px - mx) ** 2).sum()
        vy = (w * (py - my) ** 2).sum()
        cxy = (w * (px - mx) * (py - my)).sum()
        s = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        out[z, i, j] = s
        total += s
    return total / x.size, out


@pytest.mark.parametrize("shape", [(3, 7, 9), (1, 12, 5), (13, 4, 6)])
def test_equals_definition_written_out(shape):
    rng = np.random.default_rng(sum(shape))
    x = rng.random(shape)
    y = np.clip(x + 0.2 * rng.standard_normal(shape), 0, 1)
    ref, ref_map = _brute(x, y)
    got, got_map = oracle.ssim3d(x, y, return_map=True)
    assert abs(got - ref) <= 1e-12
    np.testing.assert_allclose(got_map, ref_map, rtol=0, atol=1e-12)


def test_equals_scipy_gaussian_filter_restatement():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    x = rng.random((9, 40, 31))
    y = np.clip(0.8 * x + 0.1 + 0.1 * rng.standard_normal(x.shape), 0, 1)

    def mean(f):
        kw = dict(sigma=1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
        return ndi.gaussian_filter(f, **kw) / ndi.gaussian_filter(np.ones_like(f), **kw)

    mx, my = mean(x), mean(y)
    vx, vy, cxy = mean(x * x) - mx * mx, mean(y * y) - my * my, mean(x * y) - mx * my
    smap = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    assert abs(oracle.ssim3d(x, y) - smap.mean()) <= 1e-12


def test_constant_volumes_closed_form():
    for a, b in [(0.3, 0.7), (1.0, 0.0), (0.5, 0.5)]:
        x = np.full((4, 6, 5), a)
        y = np.full((4, 6, 5), b)
        # exact in real arithmetic; the window means of x^2 - mean^2 leave ~1e-17 of
        # rounding in the variances, amplified by 1/c2
        assert abs(oracle.ssim3d(x, y) - (2 * a * b + C1) / (a * a + b * b + C1)) <= 1e-12


def test_identity_and_symmetry():
    rng = np.random.default_rng(9)
    x = rng.random((5, 20, 18))
    y = rng.random((5, 20, 18))
    assert abs(oracle.ssim3d(x, x) - 1.0) <= 1e-14
    assert abs(oracle.ssim3d(x, y) - oracle.ssim3d(y, x)) <= 1e-15
    assert oracle.ssim3d(x, y) < 0.5  # independent noise volumes are far from similar
