"""Pins of the oracle's forward model, adjoint, diag(Phi Phi^T) and v-update.

Each check compares the oracle with an independent statement: a dense matrix
built pixel by pixel from Sec. III-A, or a dense linear solve of the
v-subproblem (Eq. v-sub-1 / v-update), never with the oracle's own formula.
"""
import numpy as np
import pytest

from tests.dense import phi_matrix

CASES = [
    # (n_shots, R, H, W, per_slice, binary)
    (1, 4, 3, 5, True, True),
    (2, 3, 4, 3, True, True),
    (3, 2, 2, 4, False, True),
    (2, 4, 3, 3, True, False),
]


def _masks(rng, n, H, W, binary):
    if binary:
        return (rng.random((n, H, W)) < 0.5).astype(np.float64)
    return rng.random((n, H, W))


@pytest.mark.parametrize("N,R,H,W,per_slice,binary", CASES)
def test_forward_adjoint_match_dense(oracle, N, R, H, W, per_slice, binary):
    rng = np.random.default_rng(7)
    Z = N * R
    m = _masks(rng, Z if per_slice else R, H, W, binary)
    P = phi_matrix(m, Z, N)
    v = rng.standard_normal((Z, H, W))
    b = rng.standard_normal((N, H, W))
    np.testing.assert_allclose(oracle.forward(v, m, N).ravel(), P @ v.ravel(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.adjoint(b, m, Z).ravel(), P.T @ b.ravel(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,R,H,W,per_slice,binary", CASES)
def test_adjoint_identity(oracle, N, R, H, W, per_slice, binary):
    rng = np.random.default_rng(11)
    Z = N * R
    m = _masks(rng, Z if per_slice else R, H, W, binary)
    x = rng.standard_normal((Z, H, W))
    y = rng.standard_normal((N, H, W))
    lhs = float(np.sum(oracle.forward(x, m, N) * y))
    rhs = float(np.sum(x * oracle.adjoint(y, m, Z)))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


@pytest.mark.parametrize("N,R,H,W,per_slice,binary", CASES)
def test_phiphit_is_diagonal_of_dense(oracle, N, R, H, W, per_slice, binary):
    """Phi Phi^T is diagonal (Sec. III-B); its diagonal is the oracle's D."""
    rng = np.random.default_rng(3)
    Z = N * R
    m = _masks(rng, Z if per_slice else R, H, W, binary)
    P = phi_matrix(m, Z, N)
    PPt = P @ P.T
    assert np.count_nonzero(PPt - np.diag(np.diag(PPt))) == 0
    np.testing.assert_allclose(oracle.phiphit(m, Z, N).ravel(), np.diag(PPt), atol=1e-14)
    if binary:
        # for {0,1} masks D counts the open mirrors: an integer in [0, R]
        D = oracle.phiphit(m, Z, N)
        assert np.all(D == np.round(D)) and D.min() >= 0 and D.max() <= R


@pytest.mark.parametrize("N,R,H,W,per_slice,binary", CASES)
@pytest.mark.parametrize("rho", [0.05, 1.0, 7.5])
def test_vupdate_equals_dense_solve(oracle, N, R, H, W, per_slice, binary, rho):
    """Woodbury form == (Phi^T Phi + rho I)^{-1} (Phi^T b + rho g) (Eq. v-update)."""
    rng = np.random.default_rng(5)
    Z = N * R
    m = _masks(rng, Z if per_slice else R, H, W, binary)
    P = phi_matrix(m, Z, N)
    b = rng.standard_normal((N, H, W))
    u = rng.standard_normal((Z, H, W))
    d = rng.standard_normal((Z, H, W))
    g = (u - d).ravel()
    A = P.T @ P + rho * np.eye(Z * H * W)
    v_dense = np.linalg.solve(A, P.T @ b.ravel() + rho * g)
    v = oracle.vupdate(b, u, d, m, rho).ravel()
    np.testing.assert_allclose(v, v_dense, rtol=0, atol=1e-11)
    # the normal equations of Eq. (v-sub-1) with the 1/2 data term
    res = A @ v - (P.T @ b.ravel() + rho * g)
    assert np.max(np.abs(res)) <= 1e-11


def test_vupdate_dark_pixel_keeps_g(oracle):
    """Where every mask is closed (D = 0) the data term is absent: v = g."""
    rng = np.random.default_rng(9)
    Z, H, W = 4, 3, 3
    m = (rng.random((Z, H, W)) < 0.5).astype(np.float64)
    m[:, 1, 2] = 0.0
    b = rng.standard_normal((1, H, W))
    u, d = rng.standard_normal((2, Z, H, W))
    v = oracle.vupdate(b, u, d, m, 0.7)
    np.testing.assert_array_equal(v[:, 1, 2], (u - d)[:, 1, 2])


def test_vupdate_single_open_mirror_closed_form(oracle):
    """One open mirror at a pixel: v_r = (b + rho g_r)/(1 + rho), the others keep g."""
    Z, H, W = 3, 1, 1
    m = np.zeros((Z, H, W))
    m[1] = 1.0
    b = np.array([[[2.0]]])
    u = np.array([[[0.5]], [[1.5]], [[-1.0]]])
    d = np.array([[[0.25]], [[-0.5]], [[0.0]]])
    rho = 3.0
    v = oracle.vupdate(b, u, d, m, rho)
    g = u - d
    assert v[0, 0, 0] == pytest.approx(g[0, 0, 0], abs=1e-15)
    assert v[2, 0, 0] == pytest.approx(g[2, 0, 0], abs=1e-15)
    assert v[1, 0, 0] == pytest.approx((2.0 + rho * g[1, 0, 0]) / (1 + rho), abs=1e-15)
