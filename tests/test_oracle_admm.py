"""Pins of the oracle's full Algorithm-1 runs against closed-form minimisers.

Tikhonov (slice-based and temporal): ADMM's fixed point must be the unique
minimiser of 1/2||b - Phi v||^2 + lambda||v||^2 + gamma/2 sum_n||v_n - v_{n-1}||^2,
obtained here by a dense linear solve.  TV: the fixed point (with an accurate
inner prox) must minimise the TV objective, checked against an independent
primal-dual solve of the whole problem.  PSNR and the stopping rule are pinned
by closed forms.
"""
import numpy as np
import pytest

from tests.dense import cyclic_laplacian, grad_matrix, phi_matrix


def _problem(seed, N, R, H, W, per_slice=True, p=0.5):
    rng = np.random.default_rng(seed)
    Z = N * R
    m = (rng.random((Z if per_slice else R, H, W)) < p).astype(np.float64)
    x = rng.random((Z, H, W))
    P = phi_matrix(m, Z, N)
    b = (P @ x.ravel()).reshape(N, H, W) + 0.01 * rng.standard_normal((N, H, W))
    return m, b, P, Z


@pytest.mark.parametrize("N,R,H,W", [(1, 4, 3, 3), (2, 3, 2, 4)])
def test_tikhonov_slice_fixed_point(oracle, N, R, H, W):
    lam, rho = 0.05, 0.5
    m, b, P, Z = _problem(1, N, R, H, W)
    A = P.T @ P + 2 * lam * np.eye(P.shape[1])
    v_star = np.linalg.solve(A, P.T @ b.ravel())
    v, u, d, k = oracle.admm(b, m, Z, rho=rho, lam=lam, iters=3000, denoiser="tikhonov")
    np.testing.assert_allclose(v.ravel(), v_star, atol=1e-9)
    np.testing.assert_allclose(u, v, atol=1e-9)
    # the closed form Phi^T [ b / (2 lambda + D) ] of the slice-based model
    D = np.diag(P @ P.T)
    np.testing.assert_allclose(v_star, P.T @ (b.ravel() / (2 * lam + D)), atol=1e-12)


@pytest.mark.parametrize("N,R,H,W,gamma", [(1, 5, 2, 3, 0.3), (2, 2, 3, 2, 0.8), (1, 2, 2, 2, 0.5)])
def test_tikhonov_temporal_fixed_point(oracle, N, R, H, W, gamma):
    lam, rho = 0.05, 1.0
    m, b, P, Z = _problem(2, N, R, H, W)
    HW = H * W
    Lz = np.kron(cyclic_laplacian(Z), np.eye(HW))
    A = P.T @ P + 2 * lam * np.eye(Z * HW) + gamma * Lz
    v_star = np.linalg.solve(A, P.T @ b.ravel())
    v, u, d, k = oracle.admm(b, m, Z, rho=rho, lam=lam, gamma=gamma, iters=4000,
                             denoiser="tikhonov")
    np.testing.assert_allclose(v.ravel(), v_star, atol=1e-8)


def _tv_full_problem_cp(P, b, Z, H, W, lam, gamma, iters=60000):
    """Independent solver for min 1/2||Pv-b||^2 + lam sum_n TV(v_n) + gamma/2 v^T L v:
    Chambolle-Pock with F = lam||.||_{2,1} o K (block K per slice) and a quadratic G."""
    HW = H * W
    Ks = grad_matrix(H, W)
    K = np.kron(np.eye(Z), Ks)  # rows: slice n -> [2HW] block
    Lz = np.kron(cyclic_laplacian(Z), np.eye(HW))
    Q = P.T @ P + gamma * Lz
    c = P.T @ b.ravel()
    L = np.linalg.norm(K, 2)
    sig = tau = 0.99 / L
    Minv = np.linalg.inv(np.eye(Z * HW) + tau * Q)
    v = np.zeros(Z * HW)
    vb = v.copy()
    y = np.zeros(K.shape[0])
    for _ in range(iters):
        y = y + sig * (K @ vb)
        yy = y.reshape(Z, 2, HW)
        nrm = np.maximum(1.0, np.hypot(yy[:, 0], yy[:, 1]) / lam)
        y = (yy / nrm[:, None, :]).ravel()
        vn = Minv @ (v - tau * (K.T @ y) + tau * c)
        vb = 2 * vn - v
        v = vn
    return v


@pytest.mark.parametrize("gamma", [0.0, 0.4])
def test_tv_admm_fixed_point_minimises_objective(oracle, gamma):
    """With an accurate inner prox, Algorithm 1 with TV reaches the minimum of the
    TV (+ z) objective.  At gamma = 0 the objective has flat directions where no
    mask is open, so there the objective values are compared; at gamma > 0 the
    minimiser is unique and the volumes are compared."""
    H, W, N, R = 4, 4, 1, 3
    lam, rho = 0.02, 0.5
    m, b, P, Z = _problem(3, N, R, H, W)
    HW = H * W
    Lz = np.kron(cyclic_laplacian(Z), np.eye(HW))
    Ks = grad_matrix(H, W)

    def objective(v):
        v = v.ravel()
        tv = 0.0
        for n in range(Z):
            gv = Ks @ v[n * HW:(n + 1) * HW]
            tv += np.sum(np.hypot(gv[:HW], gv[HW:]))
        return 0.5 * np.sum((P @ v - b.ravel()) ** 2) + lam * tv + 0.5 * gamma * v @ Lz @ v

    v_cp = _tv_full_problem_cp(P, b, Z, H, W, lam, gamma, iters=20000)
    v, u, d, k = oracle.admm(b, m, Z, rho=rho, lam=lam, gamma=gamma, iters=1500,
                             denoiser="tv", tv_inner=1500)
    assert objective(v) - objective(v_cp) < 1e-6
    np.testing.assert_allclose(u, v, atol=1e-6)
    if gamma > 0:
        np.testing.assert_allclose(v.ravel(), v_cp, atol=1e-6)


def test_gamma_zero_equals_slice_based(oracle):
    """gamma = 0 reduces Algorithm 1 to the slice-based method (Sec. III-C note)."""
    m, b, P, Z = _problem(4, 1, 4, 5, 5)
    a = oracle.admm(b, m, Z, rho=1.0, lam=0.05, gamma=0.0, iters=5, denoiser="tv")
    # slice-based: every slice denoised independently from v + d, never from neighbours
    v = np.zeros((Z, 5, 5))
    u = np.zeros_like(v)
    d = np.zeros_like(v)
    for _ in range(5):
        v = oracle.vupdate(b, u, d, m, 1.0)
        u = oracle.tv_prox(v + d, 0.05 / 1.0, T=20)
        d = d + v - u
    np.testing.assert_allclose(a[0], v, atol=1e-13)
    np.testing.assert_allclose(a[1], u, atol=1e-13)


def test_psnr_closed_form(oracle):
    """A uniform error eps on a volume of max V gives PSNR = 20 log10(V / eps)."""
    ref = np.random.default_rng(0).random((3, 4, 5))
    ref[1, 2, 3] = 2.0
    eps = 1e-3
    assert oracle.psnr(ref + eps, ref) == pytest.approx(20 * np.log10(2.0 / eps), abs=1e-9)


def test_tolerance_stops_early(oracle):
    m, b, P, Z = _problem(5, 1, 4, 6, 6)
    v, u, d, k = oracle.admm(b, m, Z, rho=1.0, lam=0.05, iters=500, tol=1e-3,
                             denoiser="tikhonov")
    assert 2 <= k < 500
    v2, *_ = oracle.admm(b, m, Z, rho=1.0, lam=0.05, iters=k, denoiser="tikhonov")
    np.testing.assert_array_equal(v, v2)
    vp, *_ = oracle.admm(b, m, Z, rho=1.0, lam=0.05, iters=k - 1, denoiser="tikhonov")
    assert np.linalg.norm(v - vp) / np.linalg.norm(vp) < 1e-3
    if k > 2:
        vpp, *_ = oracle.admm(b, m, Z, rho=1.0, lam=0.05, iters=k - 2, denoiser="tikhonov")
        assert np.linalg.norm(vp - vpp) / np.linalg.norm(vpp) >= 1e-3
