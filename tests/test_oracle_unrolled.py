"""Pins of the FP64 oracle of the differentiable unrolled PnP-ADMM: it reduces to
the C oracle's Algorithm 1 when the masks are binary and the prior vanishes;
its Huber-TV prox converges to the C oracle's TV prox as eps -> 0 and meets the
Huber prox optimality condition for eps > 0; its autograd gradient matches
central finite differences."""
import numpy as np
import pytest
import torch

from oracle import unrolled as un


def _problem(seed, B, Z, H, W):
    g = torch.Generator().manual_seed(seed)
    logits = torch.randn(B, Z, H, W, generator=g, dtype=torch.float64)
    x = torch.rand(B, Z, H, W, generator=g, dtype=torch.float64)
    b = (torch.sigmoid(logits) * x).sum(1)
    return logits, b


@pytest.mark.parametrize("Z,gamma", [(4, 0.0), (4, 0.3), (2, 0.5)])
def test_reduces_to_algorithm_1(oracle, Z, gamma):
    rng = np.random.default_rng(Z)
    H, W = 6, 5
    masks = (rng.random((Z, H, W)) < 0.5).astype(np.float64)
    b = rng.random((1, H, W))
    logits = torch.tensor(np.where(masks > 0, 40.0, -40.0))[None]
    v = un.unrolled_admm(logits, torch.tensor(b), 0.8, 1e-12, gamma, iters=4, T=3, tau=0.125,
                         eps=1e-3)
    v_ref, *_ = oracle.admm(b, masks, Z, rho=0.8, lam=0.0, gamma=gamma, iters=4,
                            denoiser="tikhonov")
    np.testing.assert_allclose(v[0].numpy(), v_ref, atol=1e-10)


def test_huber_prox_tends_to_tv_prox(oracle):
    g = np.random.default_rng(1).random((6, 7))
    u = un.huber_tv_prox(torch.tensor(g), 0.2, 30000, 0.125, 0.0).numpy()
    np.testing.assert_allclose(u, oracle.tv_prox(g, 0.2, 30000), atol=2e-5)


def test_huber_prox_optimality():
    g = torch.tensor(np.random.default_rng(2).random((6, 6)))
    theta, eps = 0.15, 0.05
    u = un.huber_tv_prox(g, theta, 40000, 0.125, eps)
    gx, gy = un.grad2(u)
    nrm = torch.clamp(torch.sqrt(gx * gx + gy * gy), min=eps)
    # Huber TV gradient: grad^T (grad u / max(eps, |grad u|)) = -div(...)
    res = (u - g) - theta * un.div2(gx / nrm, gy / nrm)
    assert float(res.abs().max()) < 1e-6


def test_autograd_matches_finite_differences():
    logits, b = _problem(3, 1, 3, 5, 4)
    x = torch.rand(1, 3, 5, 4, generator=torch.Generator().manual_seed(9), dtype=torch.float64)
    kw = dict(iters=2, T=4, tau=0.125, eps=1e-2)

    def loss(lg, r, l_, gm):
        v = un.unrolled_admm(lg, b, r, l_, gm, **kw)
        return 0.5 * ((v - x) ** 2).sum()

    lg = logits.clone().requires_grad_(True)
    r = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    l_ = torch.tensor(0.07, dtype=torch.float64, requires_grad=True)
    gm = torch.tensor(0.2, dtype=torch.float64, requires_grad=True)
    L = loss(lg, r, l_, gm)
    grads = torch.autograd.grad(L, [lg, r, l_, gm])
    h = 1e-6
    base = [logits, torch.tensor(0.9, dtype=torch.float64), torch.tensor(0.07, dtype=torch.float64),
            torch.tensor(0.2, dtype=torch.float64)]
    for k in (1, 2, 3):
        plus = [t.clone() for t in base]
        minus = [t.clone() for t in base]
        plus[k] = plus[k] + h
        minus[k] = minus[k] - h
        fd = (loss(*plus) - loss(*minus)) / (2 * h)
        assert abs(float(fd) - float(grads[k])) <= 1e-6 * max(1.0, abs(float(fd)))
    for idx in [(0, 0, 0, 0), (0, 1, 2, 3), (0, 2, 4, 1)]:
        plus = logits.clone()
        minus = logits.clone()
        plus[idx] += h
        minus[idx] -= h
        fd = (loss(plus, *base[1:]) - loss(minus, *base[1:])) / (2 * h)
        assert abs(float(fd) - float(grads[0][idx])) <= 1e-6 * max(1.0, abs(float(fd)))
