"""Single-volume partition over several ranks (x/y rectangles with halo
exchange): the host-side plan on its own, and world-size 2 and 4 gloo runs in
which every rank solves its rectangle of one volume (Algorithm 1, TV + z term)
with the halo of each slice's prox input exchanged once per slice, and the
assembled reconstruction equals the FP64 oracle's whole-volume solve.

The per-rank arithmetic in the gloo runs is the FP64 oracle's (v-update and
TV prox of a rectangle); what is under test is the partition: ownership, the
halo width T + 1, the exchange plan and the Gauss-Seidel order across ranks.
No GPU is involved (the partitioned path is unmeasured on hardware)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2511_03093_gb300.partition import Partition


@pytest.mark.parametrize("H,W,ry,rx", [(40, 36, 2, 1), (40, 36, 1, 2), (17, 23, 2, 2),
                                       (9, 50, 3, 1), (30, 30, 2, 3)])
@pytest.mark.parametrize("halo", [1, 4, 11])
def test_plan_tiles_the_image_and_pairs_match(H, W, ry, rx, halo):
    part = Partition(H, W, ry, rx)
    cover = np.zeros((H, W), int)
    for r in range(part.world):
        o = part.owned(r)
        cover[o.y0:o.y1, o.x0:o.x1] += 1
        e = part.extended(r, halo)
        assert (e.y0, e.x0) == (max(0, o.y0 - halo), max(0, o.x0 - halo))
        assert (e.y1, e.x1) == (min(H, o.y1 + halo), min(W, o.x1 + halo))
    assert np.all(cover == 1)
    for r in range(part.world):
        sends, recvs = part.exchange_plan(r, halo)
        # what r receives covers exactly its halo (extended minus owned)
        got = np.zeros((H, W), int)
        for _, q in recvs:
            got[q.y0:q.y1, q.x0:q.x1] += 1
        e, o = part.extended(r, halo), part.owned(r)
        want = np.zeros((H, W), int)
        want[e.y0:e.y1, e.x0:e.x1] = 1
        want[o.y0:o.y1, o.x0:o.x1] = 0
        np.testing.assert_array_equal(got, want)
        # every send is the matching receive of the peer
        for peer, q in sends:
            assert (r, q) in part.exchange_plan(peer, halo)[1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    import synth

    w = synth.Workload("part", 4, 40, 36, drift=True, mask_p=0.3, peak=50.0, sigma_g=0.02,
                       seed=3131, n_blobs=30)
    return synth.generate(w)


PRM = dict(rho=1.0, lam=0.05, gamma=0.2, iters=3, T=10, tau=0.125)


def _rank_solve(rank, world, port, ry, rx, q):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2511_03093_gb300.partition import halo_exchange

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = _problem()
        b, masks = data["b64"], data["masks"].astype(np.float64)
        Z, H, W = masks.shape
        part = Partition(H, W, ry, rx)
        o = part.owned(rank)
        halo = PRM["T"] + 1
        e = part.extended(rank, halo)
        rho, lam, gam = PRM["rho"], PRM["lam"], PRM["gamma"]
        bo = np.ascontiguousarray(b[:, o.y0:o.y1, o.x0:o.x1])
        mo = np.ascontiguousarray(masks[:, o.y0:o.y1, o.x0:o.x1])
        u = np.zeros((Z,) + o.shape)
        d = np.zeros_like(u)
        for _ in range(PRM["iters"]):
            v = oracle.vupdate(bo, u, d, mo, rho)  # pixel-local: no exchange
            for n in range(Z):  # Gauss-Seidel in z, newest neighbours
                g = (rho * (v[n] + d[n]) + gam * (u[(n - 1) % Z] + u[(n + 1) % Z])) / (rho + 2 * gam)
                gx = halo_exchange(torch.from_numpy(g), part, rank, halo).numpy()
                ux = oracle.tv_prox(gx, lam / (rho + 2 * gam), PRM["T"], PRM["tau"])
                u[n] = ux[o.y0 - e.y0:o.y1 - e.y0, o.x0 - e.x0:o.x1 - e.x0]
            d = d + v - u
        q.put((rank, (o.y0, o.y1, o.x0, o.x1), v))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ry,rx", [(2, 1), (1, 2), (2, 2)])
def test_partitioned_solve_equals_whole_volume_oracle(ry, rx):
    import oracle

    world = ry * rx
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_solve, args=(r, world, port, ry, rx, q))
             for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    data = _problem()
    Z, H, W = data["masks"].shape
    v = np.full((Z, H, W), np.nan)
    for _, (y0, y1, x0, x1), vr in parts:
        v[:, y0:y1, x0:x1] = vr
    ref, *_ = oracle.admm(data["b64"], data["masks"], Z, rho=PRM["rho"], lam=PRM["lam"],
                          gamma=PRM["gamma"], iters=PRM["iters"], denoiser="tv",
                          tv_inner=PRM["T"], tv_tau=PRM["tau"])
    # the owned pixels run the same FP64 operations in the same order as the
    # whole-volume solve, so the values agree to the last bit
    np.testing.assert_array_equal(v, ref)
