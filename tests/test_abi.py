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


def test_binding_refuses_cpu_tensors():
    import torch

    import paper_2511_03093_gb300 as cs

    with pytest.raises(ValueError):
        cs.denoise(torch.zeros(1, 8, 8), cs.Params())
