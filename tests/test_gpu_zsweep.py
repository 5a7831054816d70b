"""Persistent z sweep of the TV u-step (gamma > 0): bit-identical to the
per-slice tile launches for every tiling, storage type and ragged geometry,
a bounded neighbour wait that runs out is reported as CSLSM_ERR_TIMEOUT, and
the library stays usable afterwards.  Agreement with the FP64 oracle is
covered by the parity tests, which run through the sweep by default."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    from paper_2511_03093_gb300 import build as b

    b.build()
    import paper_2511_03093_gb300 as m

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    yield m
    m.zsweep_config(True, -1, 2.0, False)
    m.set_autotune(0)


def _problem(seed, N, R, H, W):
    g = torch.Generator().manual_seed(seed)
    masks = (torch.rand(N * R, H, W, generator=g) < 0.5).to(torch.uint8)
    x = torch.rand(N * R, H, W, generator=g)
    b = (masks.float() * x).view(N, R, H, W).sum(1)
    return masks.cuda(), b.cuda()


def _solve(cs, plan, b, storage, iters, T, enable, tiling=-1):
    cs.zsweep_config(enable, tiling, 2.0, False)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.25, iters=iters, denoiser="tv", tv_inner=T,
                    storage=storage)
    sd = cs.STORAGE_DTYPE[storage]
    u = torch.empty(plan.vol_shape, dtype=sd, device="cuda")
    d = torch.empty(plan.vol_shape, dtype=sd, device="cuda")
    v = plan.solve(b, prm, u=u, d=d)
    torch.cuda.synchronize()
    return v.cpu(), u.float().cpu(), d.float().cpu()


GEOMS = [(1, 5, 100, 77, 20), (2, 3, 37, 200, 7), (1, 4, 64, 64, 1), (1, 2, 150, 9, 13),
         (1, 16, 128, 128, 20)]


@pytest.mark.parametrize("N,R,H,W,T", GEOMS)
@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_sweep_matches_per_slice_launches_bitwise(cs, N, R, H, W, T, storage):
    masks, b = _problem(H + W + T, N, R, H, W)
    plan = cs.Plan(H, W, N, R, masks)
    ref = _solve(cs, plan, b, storage, 3, T, enable=False)
    got = _solve(cs, plan, b, storage, 3, T, enable=True)
    for r, g_ in zip(ref, got):
        assert torch.equal(r, g_)
    plan.close()


@pytest.mark.parametrize("H,W,T", [(96, 130, 20), (300, 64, 9)])
def test_every_tiling_is_bitwise_identical(cs, H, W, T):
    masks, b = _problem(7, 1, 4, H, W)
    plan = cs.Plan(H, W, 1, 4, masks)
    ref = _solve(cs, plan, b, "fp32", 2, T, enable=False)
    used = 0
    for t in range(cs.zsweep_num_tilings()):
        cs.zsweep_config(True, t, 2.0, False)
        try:
            cs.zsweep_shape(H, W, 4, T)
        except cs.CslsmError:
            continue  # this tiling does not fit the geometry
        got = _solve(cs, plan, b, "fp32", 2, T, enable=True, tiling=t)
        for r, g_ in zip(ref, got):
            assert torch.equal(r, g_), t
        used += 1
    assert used >= 8
    plan.close()


def test_timed_tiling_choice_keeps_results(cs):
    masks, b = _problem(3, 1, 8, 200, 180)
    plan = cs.Plan(200, 180, 1, 8, masks)
    ref = _solve(cs, plan, b, "fp32", 4, 20, enable=False)
    cs.set_autotune(1)
    try:
        got = _solve(cs, plan, b, "fp32", 4, 20, enable=True)
        shp = cs.zsweep_shape(200, 180, 8, 20)
    finally:
        cs.set_autotune(0)
    for r, g_ in zip(ref, got):
        assert torch.equal(r, g_)
    assert shp["tiles"] >= 1 and 0 <= shp["tiling"] < cs.zsweep_num_tilings()
    plan.close()


def test_shape_query(cs):
    s = cs.zsweep_shape(512, 512, 16, 20)
    props = torch.cuda.get_device_properties(0)
    assert 1 <= s["tiles"] <= 2 * props.multi_processor_count
    assert s["tile_cols"] == 64 - 2 * (s["steps_per_phase"] + 1)
    assert s["region_rows"] >= s["tile_rows"] + 2 * (s["steps_per_phase"] + 1)
    assert s["region_rows"] == s["warps"] * s["rows_per_warp"] + 2
    with pytest.raises(cs.CslsmError):
        cs.zsweep_config(True, cs.zsweep_num_tilings(), 2.0, False)
    with pytest.raises(cs.CslsmError):
        cs.zsweep_config(True, -1, 0.0, False)


def test_wait_timeout_is_reported_and_recovers(cs):
    masks, b = _problem(11, 1, 4, 120, 100)
    plan = cs.Plan(120, 100, 1, 4, masks)
    ref = _solve(cs, plan, b, "fp32", 2, 20, enable=True)
    cs.zsweep_config(True, -1, 0.2, True)
    prm = cs.Params(rho=1.0, lam=0.05, gamma=0.25, iters=2, denoiser="tv", tv_inner=20)
    with pytest.raises(cs.CslsmError) as ei:
        plan.solve(b, prm)
    assert ei.value.status == 3  # CSLSM_ERR_TIMEOUT
    cs.zsweep_config(True, -1, 2.0, False)
    again = _solve(cs, plan, b, "fp32", 2, 20, enable=True)
    for r, g_ in zip(ref, again):
        assert torch.equal(r, g_)
    plan.close()
