"""Pins of the oracle's denoising steps (Eq. u-sub / u-update).

TV prox: two-pixel closed form, an independent primal-dual solver, mean
preservation, constant fixed point, the large-weight limit and a T-step
dense-matrix restatement of the dual iteration.
Tikhonov / Gauss-Seidel sweep: first-order optimality of every slice's
subproblem, checked on one ADMM iteration.
"""
import numpy as np
import pytest

from tests.dense import chambolle_pock_tv, cyclic_laplacian, grad_matrix, tv_value


@pytest.mark.parametrize("shape", [(1, 2), (2, 1)])
@pytest.mark.parametrize("a,b,theta", [(0.0, 1.0, 0.2), (0.0, 1.0, 0.6), (3.0, -1.0, 0.5),
                                       (1.0, 1.4, 0.1)])
def test_tv_two_pixels_closed_form(oracle, shape, a, b, theta):
    """min theta|u2-u1| + 1/2((u1-a)^2+(u2-b)^2): shrink the gap by 2 theta, or merge."""
    g = np.array([a, b]).reshape(shape)
    u = oracle.tv_prox(g, theta, T=4000).ravel()
    if abs(b - a) <= 2 * theta:
        exp = np.array([(a + b) / 2, (a + b) / 2])
    else:
        s = np.sign(b - a)
        exp = np.array([a + theta * s, b - theta * s])
    np.testing.assert_allclose(u, exp, atol=1e-6)


@pytest.mark.parametrize("H,W,theta", [(4, 4, 0.1), (5, 6, 0.3), (6, 3, 0.05)])
def test_tv_matches_independent_primal_dual(oracle, H, W, theta):
    rng = np.random.default_rng(H * 31 + W)
    g = rng.random((H, W))
    u_cp = chambolle_pock_tv(g, theta, iters=30000)
    u = oracle.tv_prox(g, theta, T=60000)
    np.testing.assert_allclose(u, u_cp, atol=2e-5)
    # both are minimisers: objective values agree to high precision
    f = lambda x: theta * tv_value(x) + 0.5 * np.sum((x - g) ** 2)  # noqa: E731
    assert abs(f(u) - f(u_cp)) < 1e-8


@pytest.mark.parametrize("T", [1, 3, 20])
def test_tv_preserves_mean_and_constants(oracle, T):
    rng = np.random.default_rng(T)
    g = rng.random((7, 9))
    u = oracle.tv_prox(g, 0.2, T=T)
    assert abs(u.sum() - g.sum()) < 1e-12
    c = np.full((5, 8), 0.37)
    np.testing.assert_array_equal(oracle.tv_prox(c, 0.5, T=T), c)


def test_tv_zero_weight_is_identity(oracle):
    g = np.random.default_rng(1).random((4, 5))
    np.testing.assert_array_equal(oracle.tv_prox(g, 0.0, T=20), g)


def test_tv_large_weight_gives_mean(oracle):
    g = np.random.default_rng(2).random((3, 4))
    u = oracle.tv_prox(g, 50.0, T=20000)
    np.testing.assert_allclose(u, np.full_like(g, g.mean()), atol=1e-6)


@pytest.mark.parametrize("H,W,T,theta,tau", [(5, 7, 20, 0.15, 0.125), (8, 3, 7, 0.4, 0.1),
                                             (1, 6, 12, 0.2, 0.125)])
def test_tv_T_steps_match_dense_dual_iteration(oracle, H, W, T, theta, tau):
    """The inexact T-step prox equals Chambolle's dual iteration written with the
    dense gradient K and div = -K^T (pins discretisation, boundary and step)."""
    rng = np.random.default_rng(H + 100 * W + T)
    g = rng.random((H, W))
    K = grad_matrix(H, W)
    HW = H * W
    p = np.zeros(2 * HW)
    for _ in range(T):
        s = K @ (-(K.T @ p) - g.ravel() / theta)
        nrm = np.hypot(s[:HW], s[HW:])
        den = np.concatenate([1 + tau * nrm, 1 + tau * nrm])
        p = (p + tau * s) / den
    u_dense = g.ravel() + theta * (K.T @ p)
    u = oracle.tv_prox(g, theta, T=T, tau=tau).ravel()
    np.testing.assert_allclose(u, u_dense, rtol=0, atol=1e-13)


def _one_iteration_inputs(rng, Z, H, W):
    m = (rng.random((Z, H, W)) < 0.5).astype(np.float64)
    b = rng.random((1, H, W)) * 3
    u0 = rng.standard_normal((Z, H, W))
    d0 = rng.standard_normal((Z, H, W)) * 0.3
    return m, b, u0, d0


@pytest.mark.parametrize("Z,gamma", [(1, 0.0), (2, 0.4), (5, 0.0), (5, 0.7)])
def test_tikhonov_gauss_seidel_sweep_optimality(oracle, Z, gamma):
    """After one Algorithm-1 iteration with Tikhonov, each u_n zeroes the gradient of
    its subproblem (Eq. temporal_u_sub, psi=||u||^2) at the neighbours the sweep used:
    u_{n-1} already updated, u_{n+1} still old, cyclic; and d1 = d0 + v1 - u1."""
    rng = np.random.default_rng(Z * 10 + int(gamma * 10))
    H, W = 3, 4
    rho, lam = 0.9, 0.3
    m, b, u0, d0 = _one_iteration_inputs(rng, Z, H, W)
    v1, u1, d1, k = oracle.admm(b, m, Z, rho=rho, lam=lam, gamma=gamma, iters=1,
                                denoiser="tikhonov", u0=u0, d0=d0)
    assert k == 1
    np.testing.assert_allclose(v1, oracle.vupdate(b, u0, d0, m, rho), atol=1e-14)
    gam = gamma if Z > 1 else 0.0
    for n in range(Z):
        prev = u1[(n - 1) % Z] if n >= 1 else u0[Z - 1]
        nxt = u0[(n + 1) % Z] if n < Z - 1 else u1[0]
        grad = (2 * lam * u1[n] + rho * (u1[n] - v1[n] - d0[n])
                + gam * (u1[n] - prev) + gam * (u1[n] - nxt))
        assert np.max(np.abs(grad)) < 1e-13
    np.testing.assert_allclose(d1, d0 + v1 - u1, atol=1e-15)


def test_cyclic_laplacian_matches_objective():
    """The z term (gamma/2) sum_n ||v_n - v_{n-1}||^2, one cyclic edge per slice, is
    (gamma/2) v^T L v with the Laplacian the fixed-point tests use."""
    rng = np.random.default_rng(0)
    for Z in (2, 3, 6):
        v = rng.standard_normal(Z)
        direct = sum((v[n] - v[(n - 1) % Z]) ** 2 for n in range(Z))
        assert abs(v @ cyclic_laplacian(Z) @ v - direct) < 1e-12
