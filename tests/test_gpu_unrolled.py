"""Differentiable unrolled PnP-ADMM on the GPU (hand-written adjoint behind a
torch.autograd.Function) against the FP64 oracle map and its autograd gradient,
finite differences, and checkpoint-period invariance; one run at the full
batch-8, 512 x 512 x 16, 30-iteration size."""
import numpy as np
import pytest
import torch

from oracle import unrolled as un
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return m


def _problem(seed, B, Z, H, W):
    g = torch.Generator().manual_seed(seed)
    logits = torch.randn(B, Z, H, W, generator=g)
    x = torch.rand(B, Z, H, W, generator=g)
    b = (torch.sigmoid(logits.double()) * x.double()).sum(1).float()
    return logits, b, x


CFG = dict(iters=4, tv_steps=8, tv_tau=0.125, huber_eps=1e-3, ckpt_every=2)


def _scalars(rho=0.9, lam=0.05, gamma=0.2, dev="cuda", dtype=torch.float32):
    return [torch.tensor(v, dtype=dtype, device=dev, requires_grad=True) for v in (rho, lam, gamma)]


@pytest.mark.parametrize("B,Z,H,W", [(2, 4, 24, 20), (1, 3, 17, 33), (1, 2, 40, 9), (1, 3, 70, 45)])
def test_forward_and_gradient_match_fp64_oracle(cs, B, Z, H, W):
    logits, b, x = _problem(B + Z + H, B, Z, H, W)
    vbar = torch.randn(B, Z, H, W, generator=torch.Generator().manual_seed(4))
    # GPU
    lg = logits.cuda().requires_grad_(True)
    r, l_, gm = _scalars()
    v = cs.unrolled_admm(lg, b.cuda(), r, l_, gm, **CFG)
    (v * vbar.cuda()).sum().backward()
    # FP64 oracle on the same float32 inputs
    lg64 = logits.double().requires_grad_(True)
    r64, l64, g64 = _scalars(dev="cpu", dtype=torch.float64)
    v64 = un.unrolled_admm(lg64, b.double(), r64, l64, g64, iters=CFG["iters"],
                           T=CFG["tv_steps"], tau=CFG["tv_tau"], eps=CFG["huber_eps"])
    (v64 * vbar.double()).sum().backward()
    assert rel_l2(v.detach().cpu().numpy(), v64.detach().numpy()) <= 1e-5
    assert rel_l2(lg.grad.cpu().numpy(), lg64.grad.numpy()) <= 1e-3
    for a, e in ((r, r64), (l_, l64), (gm, g64)):
        ga, ge = float(a.grad), float(e.grad)
        assert abs(ga - ge) <= 1e-3 * max(abs(ge), 1e-3), (ga, ge)


def test_checkpoint_period_does_not_change_gradients(cs):
    logits, b, _ = _problem(5, 1, 4, 20, 18)
    vbar = torch.randn(1, 4, 20, 18, generator=torch.Generator().manual_seed(6)).cuda()
    out = []
    for every in (1, 3, 4):
        lg = logits.cuda().requires_grad_(True)
        r, l_, gm = _scalars()
        v = cs.unrolled_admm(lg, b.cuda(), r, l_, gm, **dict(CFG, ckpt_every=every))
        (v * vbar).sum().backward()
        out.append((lg.grad.cpu().numpy(), float(r.grad), float(l_.grad), float(gm.grad)))
    for o in out[1:]:
        np.testing.assert_array_equal(o[0], out[0][0])
        assert o[1:] == out[0][1:]


@pytest.mark.parametrize("B,Z,H,W,every", [(1, 4, 20, 18, 3), (2, 3, 37, 29, 1), (1, 2, 30, 33, 4)])
def test_kept_duals_give_the_same_gradients(cs, B, Z, H, W, every):
    """keep_duals reads the dual iterates the segment recompute stored instead of
    recomputing them per slice: the gradients must not change by a bit."""
    logits, b, _ = _problem(9 + H, B, Z, H, W)
    vbar = torch.randn(B, Z, H, W, generator=torch.Generator().manual_seed(7)).cuda()
    out = []
    for keep in (False, True):
        lg = logits.cuda().requires_grad_(True)
        r, l_, gm = _scalars()
        v = cs.unrolled_admm(lg, b.cuda(), r, l_, gm,
                             **dict(CFG, ckpt_every=every, keep_duals=keep))
        (v * vbar).sum().backward()
        out.append((v.detach().cpu().numpy(), lg.grad.cpu().numpy(), float(r.grad),
                    float(l_.grad), float(gm.grad)))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2:] == out[1][2:]


def test_full_length_gradient_matches_fp64_oracle(cs):
    """The full-length unrolled map (30 iterations, 20 Huber-TV steps, checkpoints
    every 5) at the reduced oracle size 64 x 64 x 8, batch 1: v and every gradient
    against the FP64 oracle's autograd gradient."""
    B, Z, H, W = 1, 8, 64, 64
    logits, b, x = _problem(21, B, Z, H, W)
    cfg = dict(iters=30, tv_steps=20, tv_tau=0.125, huber_eps=1e-3, ckpt_every=5)
    lg = logits.cuda().requires_grad_(True)
    r, l_, gm = _scalars(1.0, 0.05, 0.2)
    v = cs.unrolled_admm(lg, b.cuda(), r, l_, gm, **cfg)
    (0.5 * ((v - x.cuda()) ** 2).sum()).backward()
    lg64 = logits.double().requires_grad_(True)
    r64, l64, g64 = _scalars(1.0, 0.05, 0.2, dev="cpu", dtype=torch.float64)
    v64 = un.unrolled_admm(lg64, b.double(), r64, l64, g64, iters=cfg["iters"],
                           T=cfg["tv_steps"], tau=cfg["tv_tau"], eps=cfg["huber_eps"])
    (0.5 * ((v64 - x.double()) ** 2).sum()).backward()
    assert rel_l2(v.detach().cpu().numpy(), v64.detach().numpy()) <= 1e-5
    assert rel_l2(lg.grad.cpu().numpy(), lg64.grad.numpy()) <= 1e-3
    for a, e in ((r, r64), (l_, l64), (gm, g64)):
        ga, ge = float(a.grad), float(e.grad)
        assert abs(ga - ge) <= 1e-3 * max(abs(ge), 1e-3), (ga, ge)


def test_finite_differences_on_gpu(cs):
    """Central differences with 1e-4 relative perturbations of rho, lambda, gamma."""
    logits, b, x = _problem(8, 1, 4, 32, 28)
    lgc, bc, xc = logits.cuda(), b.cuda(), x.cuda()

    def loss(rho, lam, gamma, lg=lgc):
        r, l_, gm = _scalars(rho, lam, gamma)
        v = cs.unrolled_admm(lg, bc, r, l_, gm, **CFG)
        return 0.5 * ((v - xc) ** 2).sum(), (r, l_, gm)

    L, ps = loss(0.9, 0.05, 0.2)
    L.backward()
    base = (0.9, 0.05, 0.2)
    for k in range(3):
        h = 1e-4 * base[k]
        up = list(base)
        dn = list(base)
        up[k] += h
        dn[k] -= h
        with torch.no_grad():
            fd = (float(loss(*up)[0]) - float(loss(*dn)[0])) / (2 * h)
        an = float(ps[k].grad)
        assert abs(fd - an) <= 2e-2 * max(abs(an), 1e-2), (k, fd, an)


def test_full_size_batch8(cs):
    """Batch 8 of 512 x 512 x 16, 30 iterations, checkpoint every 5: finite gradients,
    a directional finite-difference check along lambda, and the same gradients with
    the dual iterates kept."""
    B, Z, H, W = 8, 16, 512, 512
    g = torch.Generator(device="cuda").manual_seed(11)
    logits = torch.randn(B, Z, H, W, generator=g, device="cuda")
    x = torch.rand(B, Z, H, W, generator=g, device="cuda")
    b = (torch.sigmoid(logits) * x).sum(1)
    cfg = dict(iters=30, tv_steps=20, tv_tau=0.125, huber_eps=1e-3, ckpt_every=5)
    lg = logits.clone().requires_grad_(True)
    r, l_, gm = _scalars(1.0, 0.05, 0.2)
    v = cs.unrolled_admm(lg, b, r, l_, gm, **cfg)
    L = 0.5 * ((v - x) ** 2).mean()
    L.backward()
    assert torch.isfinite(lg.grad).all()
    assert all(np.isfinite(float(t.grad)) for t in (r, l_, gm))
    h = 1e-3 * 0.05
    with torch.no_grad():
        lp = 0.5 * ((cs.unrolled_admm(logits, b, *_scalars(1.0, 0.05 + h, 0.2), **cfg) - x) ** 2).mean()
        lm = 0.5 * ((cs.unrolled_admm(logits, b, *_scalars(1.0, 0.05 - h, 0.2), **cfg) - x) ** 2).mean()
    fd = (float(lp) - float(lm)) / (2 * h)
    assert abs(fd - float(l_.grad)) <= 5e-2 * max(abs(float(l_.grad)), 1e-6), (fd, float(l_.grad))
    # and along rho and gamma
    for k, (base, an) in enumerate(((1.0, float(r.grad)), (0.2, float(gm.grad)))):
        h = 1e-3 * base
        vals = [[1.0, 0.05, 0.2], [1.0, 0.05, 0.2]]
        idx = 0 if k == 0 else 2
        vals[0][idx] += h
        vals[1][idx] -= h
        with torch.no_grad():
            lp, lm = (0.5 * ((cs.unrolled_admm(logits, b, *_scalars(*vv), **cfg) - x) ** 2).mean()
                      for vv in vals)
        fd = (float(lp) - float(lm)) / (2 * h)
        assert abs(fd - an) <= 5e-2 * max(abs(an), 1e-6), (("rho", "gamma")[k], fd, an)
    # the same gradients with the dual iterates kept (about 29 GB of workspace)
    lg2 = logits.clone().requires_grad_(True)
    r2, l2, g2 = _scalars(1.0, 0.05, 0.2)
    v2 = cs.unrolled_admm(lg2, b, r2, l2, g2, **dict(cfg, keep_duals=True))
    (0.5 * ((v2 - x) ** 2).mean()).backward()
    assert torch.equal(lg2.grad, lg.grad)
    assert [float(t.grad) for t in (r2, l2, g2)] == [float(t.grad) for t in (r, l_, gm)]
