"""The C-ABI library: it builds, loads, exports every declared entry point, and
rejects bad arguments on the host before any GPU work (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cslsm.h")


@pytest.fixture(scope="module")
def L():
    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as cs

    return cs.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cslsm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("cslsm_plan_create", "cslsm_plan_destroy", "cslsm_forward", "cslsm_adjoint",
              "cslsm_admm_solve", "cslsm_denoise", "cslsm_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in include/cslsm.h but not exported"


def test_status_strings_and_version(L):
    assert L.cslsm_abi_version() == 4
    for code, name in [(0, b"CSLSM_OK"), (1, b"CSLSM_ERR_INVALID_ARG"), (2, b"CSLSM_ERR_CUDA"),
                       (3, b"CSLSM_ERR_TIMEOUT"), (4, b"CSLSM_ERR_UNSUPPORTED"),
                       (5, b"CSLSM_ERR_OOM")]:
        assert L.cslsm_status_string(code) == name


def _params(**kw):
    import paper_2511_03093_gb300 as cs

    p = cs.Params(**{k: v for k, v in kw.items() if k != "init_user"})
    return p.to_c(kw.get("init_user", False))


def test_invalid_arguments_rejected_on_host(L):
    import paper_2511_03093_gb300 as cs

    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: rejected before any GPU work
    INVALID = 1
    assert L.cslsm_plan_create(ctypes.byref(h), 0, 8, 1, 4, fake, 1, None) == INVALID
    assert b"H and W" in L.cslsm_last_error()
    assert L.cslsm_plan_create(ctypes.byref(h), 8, 8, 1, 33, fake, 1, None) == INVALID
    assert L.cslsm_plan_create(ctypes.byref(h), 8, 8, 1, 4, None, 1, None) == INVALID
    assert L.cslsm_plan_create(ctypes.byref(h), 1 << 16, 1 << 16, 1, 1, fake, 1, None) == INVALID
    assert L.cslsm_plan_create(None, 8, 8, 1, 4, fake, 1, None) == INVALID
    assert L.cslsm_forward(None, fake, fake, None) == INVALID
    assert L.cslsm_adjoint(None, fake, fake, None) == INVALID
    st = cs.AdmmStats()
    p = _params()
    assert L.cslsm_admm_solve(None, fake, ctypes.byref(p), fake, None, None,
                              ctypes.byref(st), None) == INVALID
    # parameter checks of the denoiser entry point
    for bad in (dict(rho=0.0), dict(rho=float("nan")), dict(lam=-1.0), dict(tv_tau=0.3),
                dict(tv_inner=0), dict(denoiser="bm3d", bm3d_sigma=0.0)):
        p = _params(**bad)
        assert L.cslsm_denoise(p.denoiser, fake, ctypes.c_void_p(0x100000), 1, 8, 8,
                               ctypes.byref(p), None) == INVALID, bad
    p = _params()
    # overlapping in/out for TV
    assert L.cslsm_denoise(1, fake, ctypes.c_void_p(0x1000 + 4), 1, 8, 8, ctypes.byref(p),
                           None) == INVALID
    assert b"overlap" in L.cslsm_last_error()
    assert L.cslsm_denoise(0, fake, fake, 0, 8, 8, ctypes.byref(p), None) == INVALID
    assert L.cslsm_psnr(fake, fake, 0, fake, None) == INVALID
    assert L.cslsm_plan_destroy(None) == 0


def test_newer_entry_points_reject_bad_arguments_on_host(L):
    """3-D SSIM, the batch, the unrolled solver and the allocation-free BM3D refuse
    empty, oversized or inconsistent arguments before any GPU work."""
    import paper_2511_03093_gb300 as cs

    fake = ctypes.c_void_p(0x1000)  # never dereferenced
    INVALID = 1
    for Z, H, W in ((0, 8, 8), (4, 0, 8), (4, 8, -1), (1 << 11, 1 << 10, 1 << 10)):
        assert L.cslsm_ssim3d(fake, fake, Z, H, W, fake, None) == INVALID, (Z, H, W)
    assert L.cslsm_ssim3d(None, fake, 4, 8, 8, fake, None) == INVALID
    b = ctypes.c_void_p()
    p = _params()
    assert L.cslsm_batch_create(ctypes.byref(b), None, 0, ctypes.byref(p), None) == INVALID
    assert b"at least one item" in L.cslsm_last_error()
    # unrolled solver parameters: the workspace query returns 0 for invalid ones
    good = dict(rho=1.0, lam=0.05, gamma=0.2, cfg=dict(iters=4, tv_steps=8, tv_tau=0.125,
                                                       huber_eps=1e-3, ckpt_every=2))
    up = cs._unrolled_params(good["rho"], good["lam"], good["gamma"], good["cfg"])
    assert L.cslsm_unrolled_workspace_bytes(1, 4, 16, 16, ctypes.byref(up)) > 0
    for field, value in (("keep_duals", 2), ("tv_tau", 0.2), ("iters", 0), ("ckpt_every", 0),
                         ("rho", 0.0), ("lambda_", -1.0), ("huber_eps", -1.0)):
        bad = cs._unrolled_params(good["rho"], good["lam"], good["gamma"], good["cfg"])
        setattr(bad, field, value)
        assert L.cslsm_unrolled_workspace_bytes(1, 4, 16, 16, ctypes.byref(bad)) == 0, field
    assert L.cslsm_unrolled_workspace_bytes(0, 4, 16, 16, ctypes.byref(up)) == 0
    # keep_duals grows the workspace by ckpt_every x Z x (2 tv_steps + 3) x B H W floats
    kp = cs._unrolled_params(1.0, 0.05, 0.2, dict(good["cfg"], keep_duals=True))
    grow = L.cslsm_unrolled_workspace_bytes(1, 4, 16, 16, ctypes.byref(kp)) - \
        L.cslsm_unrolled_workspace_bytes(1, 4, 16, 16, ctypes.byref(up))
    assert 2 * 4 * (2 * 8 + 3) * 16 * 16 * 4 <= grow <= 2 * 4 * (2 * 8 + 3) * 16 * 16 * 4 + 512
    # batch phase length: a process-wide setting, negative values rejected
    L.cslsm_set_batch_steps_per_phase.argtypes = [ctypes.c_int]
    assert L.cslsm_set_batch_steps_per_phase(-1) == INVALID
    assert L.cslsm_set_batch_steps_per_phase(0) == 0
    L.cslsm_set_tv_route.argtypes = [ctypes.c_int]
    for bad in (-1, 3):
        assert L.cslsm_set_tv_route(bad) == INVALID
    assert L.cslsm_set_tv_route(0) == 0
    # the allocation-free BM3D: bad sizes and sigma, overlap
    assert L.cslsm_denoise_bm3d_noalloc(fake, ctypes.c_void_p(0x10000000), 0, 8, 8,
                                        ctypes.c_float(0.05), None) == INVALID
    assert L.cslsm_denoise_bm3d_noalloc(fake, ctypes.c_void_p(0x10000000), 1, 8, 8,
                                        ctypes.c_float(0.0), None) == INVALID
    assert L.cslsm_denoise_bm3d_noalloc(fake, ctypes.c_void_p(0x1004), 1, 8, 8,
                                        ctypes.c_float(0.05), None) == INVALID
    assert b"overlap" in L.cslsm_last_error()


def test_binding_refuses_cpu_tensors():
    import torch

    import paper_2511_03093_gb300 as cs

    with pytest.raises(ValueError):
        cs.denoise(torch.zeros(1, 8, 8), cs.Params())
